// pt_api.cu -- the C ABI of libpt.so (include/pt.h): contexts, trees,
// workspace management, host/device staging and the call sequence.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <new>
#include <vector>

#include "../../include/pt.h"
#include "pt_kernels.cuh"

using namespace pt;

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------

struct pt_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;   // private stream used only to capture graphs
    // private stream that copies host results while the stream's last
    // kernels (energy sums, neighbour CSR) run, and the event it waits on
    cudaStream_t out_stream = nullptr;
    cudaEvent_t ev_out = nullptr;
    char err[512] = {0};
    Status *h_status = nullptr;      // pinned
    cudaEvent_t ev[8] = {};
    pt_tree *batch_tree = nullptr;   // reused by pt_batch_longrange_force
    // trees built in this context and not yet freed: pt_ctx_destroy releases
    // their device memory and detaches them, so a later pt_tree_free never
    // touches the destroyed context
    std::vector<pt_tree *> trees;
    // device and pinned host blocks given up by buffers that grew: freed when
    // the context is destroyed (or once they pass kRetiredMax), because a
    // cudaFree / cudaFreeHost waits for the whole device, which would stall
    // the streams of every other context (a server's other workers)
    std::vector<void *> retired_dev, retired_host;
    size_t retired_bytes = 0;
    struct TuneEntry {
        int nsets, nbucket, mbucket, order, precision;
        double theta;
        int n_leaf, n_group;
        double ms;
    };
    std::vector<TuneEntry> tune_cache;   // autotuner results of this context
};

namespace {

int fail(pt_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof ctx->err, fmt, ap);
        va_end(ap);
    }
    return code;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? PT_ERR_OOM : PT_ERR_CUDA, \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define TRY(expr)                \
    do {                         \
        int r_ = (expr);         \
        if (r_ != PT_OK) return r_; \
    } while (0)

// Grow-only device buffer.
struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <typename T>
    T *as() const { return static_cast<T *>(p); }
};

constexpr size_t kRetiredMax = 2ull << 30;

void free_retired(pt_ctx *ctx) {
    for (void *q : ctx->retired_dev) cudaFree(q);
    for (void *q : ctx->retired_host) cudaFreeHost(q);
    ctx->retired_dev.clear();
    ctx->retired_host.clear();
    ctx->retired_bytes = 0;
}

void retire(pt_ctx *ctx, void *p, size_t bytes, bool host) {
    if (!p) return;
    (host ? ctx->retired_host : ctx->retired_dev).push_back(p);
    ctx->retired_bytes += bytes;
    if (ctx->retired_bytes > kRetiredMax) free_retired(ctx);
}

// A buffer that has to grow keeps a quarter of head room, and its old block
// is retired rather than freed (see pt_ctx::retired_dev).
int ensure(pt_ctx *ctx, Buf &b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return PT_OK;
    if (b.p) {
        bytes = std::max(bytes, b.bytes + b.bytes / 4);
        retire(ctx, b.p, b.bytes, false);
        b.p = nullptr;
        b.bytes = 0;
    }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        (void)cudaGetLastError();
        return fail(ctx, PT_ERR_OOM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    }
    b.bytes = bytes;
    return PT_OK;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// ---------------------------------------------------------------------------
// Tree
// ---------------------------------------------------------------------------

struct pt_tree {
    pt_ctx *ctx = nullptr;
    unsigned n = 0;
    int nsets = 0;
    pt_params prm{};
    std::vector<SetInfo> h_sets;
    // capacities
    unsigned cap_n = 0, cap_nodes = 0, cap_sets = 0;
    unsigned long long cap_cells = 0, cap_pp = 0, cap_pairs = 0, cap_sort = 0;
    // device buffers
    Buf status, sets, set_of, bmin, bmax, n_dev;
    Buf in_pos, in_mass;                                   // staging for host inputs
    Buf keys_in, vals_in, qbuf, skey, perm, sp64, spH, spL, sq;
    Buf nd_a, nd_b, nd_r, nd_c, nd_q, nd_t, nd_f, nd_bnd, nd_int, topo_bs, tmp_a, tmp_b, lcp;
    Buf gflag, gbegin, gr_r, gr_a, gr_b, gr_nc, gr_np, gr_co, gr_po, gr_nf, gr_fo, gr_ord, gpart, red_part;
    Buf cells, pp;
    Buf pairs, nb_keys, nb_keys_s, nb_vals, nb_vals_s, nb_off, nb_idx, npairs_dev;
    Buf sort_k2, sort_v2, sort_counts, scan_sums;
    Buf in_scale, scale_buf, set_mean, ssc, nd_thr, gr_thr;   // mass-dependent radii
    Buf orb_vel, orb_sv, orb_rnbf, orb_ndr, orb_ndthr, orb_grthr, orb_ctr, orb_rnb;   // orbit-dependent search
    Buf walk_spill;                                        // spill areas of the walk stacks
    Buf out_acc, out_pot;                                  // staging for host outputs
    // batch state (the context's batch tree only)
    Buf d_tab, d_totals, d_acc, d_pot;
    BatchTab *h_tab = nullptr;                 // pinned, cap_tab entries
    SetInfo *h_sets_pin = nullptr;             // pinned, cap_tab entries
    long long *h_totals = nullptr;             // pinned, cap_tab entries
    unsigned *h_n = nullptr;                   // pinned
    int cap_tab = 0;
    double *h_io = nullptr;                    // pinned host staging (4 doubles per particle)
    long long *h_nboff = nullptr;              // pinned, n + 1
    int *h_nbidx = nullptr;                    // pinned, cap_h_nb
    size_t cap_h_io = 0, cap_h_nboff = 0, cap_h_nb = 0;
    cudaGraphExec_t gexec = nullptr;           // captured launch sequence
    // single-tree builds: the build's launch sequence, captured once its
    // arguments (sizes, buffers, inputs) repeat, then replayed
    cudaGraphExec_t gbuild = nullptr;
    BuildArgs gbuild_args{}, last_build_args{};
    bool have_last_build = false;
    std::vector<unsigned> gkey_n;
    std::vector<double> gkey_r;
    pt_params gkey_p{};
    int gkey_mode = -1;
    // last results
    Status h{};
    unsigned walk_stack = kWalkStackSmall;
    unsigned walk_spill_cap = 0;               // spill entries per warp allocated (0: none yet)
    // list sizes of the last successful walk of this tree: the one-pass walk
    // sizes its arrays from them (0: no estimate yet, walk in two passes)
    unsigned long long est_cells = 0, est_pp = 0;
    unsigned long long chunk_cells = kWalkChunkEntries, chunk_pp = kWalkChunkEntries;
    const double *scale_in = nullptr;          // device radius factors of the current build
    bool built = false, lists_valid = false;
    float ms_build = 0.f;
    int launches_build = 0, launches_force = 0;

    void release() {
        Buf *all[] = {&status, &sets, &set_of, &bmin, &bmax, &n_dev, &in_pos, &in_mass, &keys_in,
                      &vals_in, &qbuf, &skey, &perm, &sp64, &spH, &spL, &sq, &nd_a, &nd_b, &nd_r,
                      &nd_c, &nd_q, &nd_t, &nd_f, &nd_bnd, &nd_int, &topo_bs, &tmp_a, &tmp_b, &lcp, &gflag, &gbegin, &gr_r, &gr_a,
                      &gr_b, &gr_nc, &gr_np, &gr_co, &gr_po, &gr_nf, &gr_fo, &gr_ord, &gpart, &red_part, &cells, &pp, &pairs,
                      &nb_keys, &nb_keys_s, &nb_vals, &nb_vals_s, &nb_off, &nb_idx, &npairs_dev,
                      &sort_k2, &sort_v2, &sort_counts, &scan_sums, &out_acc, &out_pot,
                      &in_scale, &scale_buf, &set_mean, &ssc, &nd_thr, &gr_thr, &orb_vel, &orb_sv, &orb_rnbf, &walk_spill,
                      &orb_ndr, &orb_ndthr, &orb_grthr, &orb_ctr, &orb_rnb};
        for (Buf *b : all) b->release();
        d_tab.release(); d_totals.release(); d_acc.release(); d_pot.release();
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
        if (gbuild) cudaGraphExecDestroy(gbuild);
        gbuild = nullptr;
        have_last_build = false;
        void *pinned[] = {h_tab, h_sets_pin, h_totals, h_n, h_io, h_nboff, h_nbidx};
        for (void *q : pinned)
            if (q) cudaFreeHost(q);
        h_tab = nullptr; h_sets_pin = nullptr; h_totals = nullptr; h_n = nullptr;
        h_io = nullptr; h_nboff = nullptr; h_nbidx = nullptr;
        cap_tab = 0; cap_h_io = cap_h_nboff = cap_h_nb = 0;
    }
};

namespace {

int check_params(pt_ctx *ctx, const pt_params *p) {
    if (!p) return fail(ctx, PT_ERR_ARG, "params is NULL");
    if (!(p->theta >= 0.0) || !std::isfinite(p->theta))
        return fail(ctx, PT_ERR_ARG, "theta must be finite and >= 0 (got %g)", p->theta);
    if (!(p->G > 0.0) || !std::isfinite(p->G)) return fail(ctx, PT_ERR_ARG, "G must be > 0");
    if (p->n_leaf < 1) return fail(ctx, PT_ERR_ARG, "n_leaf must be >= 1");
    if (p->n_group < 1) return fail(ctx, PT_ERR_ARG, "n_group must be >= 1");
    if (p->order != 0 && p->order != 2) return fail(ctx, PT_ERR_ARG, "order must be 0 or 2");
    if (p->precision != PT_FP64 && p->precision != PT_MIXED)
        return fail(ctx, PT_ERR_ARG, "precision must be PT_FP64 or PT_MIXED");
    if (p->mass_dependent != 0 && p->mass_dependent != 1)
        return fail(ctx, PT_ERR_ARG, "mass_dependent must be 0 or 1");
    return PT_OK;
}

int check_radii(pt_ctx *ctx, double r_in, double r_out) {
    if (!(r_in >= 0.0) || !(r_out > r_in) || !std::isfinite(r_out))
        return fail(ctx, PT_ERR_ARG, "need 0 <= r_in < r_out (got r_in=%g r_out=%g)", r_in, r_out);
    return PT_OK;
}

// Integer form of the opening test: the smallest d2 with s^2 < fl(theta^2 * d2)
// for every level (see pt.h); INT64_MAX when no d2 in range qualifies.
void walk_thresholds(double theta, WalkParams &wp) {
    const double theta2 = theta * theta;
    for (int l = 0; l < kLevels; l++) {
        const double s = std::ldexp(1.0, kBits + 1 - l);
        const double s2 = s * s;
        long long thr = 0x7fffffffffffffffll;
        if (theta2 > 0.0) {
            const double est = s2 / theta2;
            if (est < 1.0e15) {
                long long d = (long long)std::floor(est) - 8;
                if (d < 0) d = 0;
                while (!(s2 < theta2 * (double)d)) d++;
                thr = d;
            }
        }
        wp.ithr[l] = thr;
    }
}

ScanTmp scan_tmp_of(pt_tree *t) { return ScanTmp{t->scan_sums.as<unsigned long long>()}; }
SortTmp sort_tmp_of(pt_tree *t) {
    return SortTmp{t->sort_k2.as<unsigned long long>(), t->sort_v2.as<unsigned>(),
                   t->sort_counts.as<unsigned>()};
}

int alloc_build(pt_tree *t, unsigned n, int nsets) {
    pt_ctx *ctx = t->ctx;
    // node capacity: at least the estimate for this build's size (a tree
    // reused for a larger set, e.g. a batch tree, grows here; overflows of
    // the estimate double it in run_build)
    {
        const unsigned long long c = 2ull * n / (unsigned)std::max(1, std::min(t->prm.n_leaf, 8)) +
                                     (unsigned long long)kLevels * nsets + 1024;
        const unsigned est = (unsigned)std::min<unsigned long long>(c, 0x7fffffffull);
        if (t->cap_nodes < est) t->cap_nodes = est;
    }
    if (t->cap_nodes < (unsigned)nsets + 1024) t->cap_nodes = nsets + 1024;
    const size_t N = n, C = t->cap_nodes, S = nsets;
    TRY(ensure(ctx, t->status, sizeof(Status)));
    TRY(ensure(ctx, t->sets, S * sizeof(SetInfo)));
    TRY(ensure(ctx, t->set_of, nsets > 1 ? N * 4 : 16));
    TRY(ensure(ctx, t->bmin, 3 * S * 8));
    TRY(ensure(ctx, t->bmax, 3 * S * 8));
    TRY(ensure(ctx, t->n_dev, 16));
    TRY(ensure(ctx, t->keys_in, N * 8));
    TRY(ensure(ctx, t->vals_in, N * 4));
    TRY(ensure(ctx, t->qbuf, N * 16));
    TRY(ensure(ctx, t->skey, N * 8));
    TRY(ensure(ctx, t->perm, N * 4));
    TRY(ensure(ctx, t->sp64, N * 32));
    TRY(ensure(ctx, t->spH, N * 16));
    TRY(ensure(ctx, t->spL, N * 16));
    TRY(ensure(ctx, t->sq, N * 16));
    TRY(ensure(ctx, t->nd_a, C * 16));
    TRY(ensure(ctx, t->nd_b, C * 16));
    TRY(ensure(ctx, t->nd_r, C * 8));
    TRY(ensure(ctx, t->nd_c, C * 32));
    TRY(ensure(ctx, t->nd_q, C * 64));
    TRY(ensure(ctx, t->nd_t, C * 64));
    TRY(ensure(ctx, t->nd_f, C * 48));
    TRY(ensure(ctx, t->nd_bnd, C * 32));
    TRY(ensure(ctx, t->nd_int, C * 4));
    TRY(ensure(ctx, t->topo_bs, (size_t)sm_count() * 8 * 4));   // one per block of the topology grid
    TRY(ensure(ctx, t->lcp, N + 32));
    TRY(ensure(ctx, t->tmp_a, std::max(C, N) * 4));
    TRY(ensure(ctx, t->tmp_b, std::max(C, N) * 4));
    TRY(ensure(ctx, t->gflag, N * 4));
    TRY(ensure(ctx, t->gbegin, N * 4));
    TRY(ensure(ctx, t->gr_r, N * 8));
    TRY(ensure(ctx, t->gr_a, N * 16));
    TRY(ensure(ctx, t->gr_b, N * 16));
    TRY(ensure(ctx, t->gr_nc, N * 4));
    TRY(ensure(ctx, t->gr_np, N * 4));
    TRY(ensure(ctx, t->gr_nf, N * 4));
    TRY(ensure(ctx, t->gr_fo, (N + 1) * 8));
    TRY(ensure(ctx, t->gr_ord, N * 4));
    TRY(ensure(ctx, t->gr_co, (N + 1) * 8));
    TRY(ensure(ctx, t->gr_po, (N + 1) * 8));
    TRY(ensure(ctx, t->gpart, N * 32));
    TRY(ensure(ctx, t->red_part, (size_t)kRedBlocksMax * 48));     // reduction partials, one per block
    TRY(ensure(ctx, t->ssc, N * 8));
    TRY(ensure(ctx, t->set_mean, S * 8));
    if (t->prm.mass_dependent) {
        TRY(ensure(ctx, t->scale_buf, N * 8));
        TRY(ensure(ctx, t->nd_thr, C * 8));
        TRY(ensure(ctx, t->gr_thr, N * 8));
    }
    TRY(ensure(ctx, t->scan_sums, (kScanBlocks + 1) * 8));
    TRY(ensure(ctx, t->sort_counts, (size_t)kSortCountsLen * 4));
    t->cap_sort = std::max<unsigned long long>(t->cap_sort, N);
    TRY(ensure(ctx, t->sort_k2, t->cap_sort * 8));
    TRY(ensure(ctx, t->sort_v2, t->cap_sort * 4));
    t->cap_n = n;
    t->cap_sets = nsets;
    return PT_OK;
}

BuildArgs build_args(pt_tree *t, const double *pos, const double *mass) {
    BuildArgs A;
    std::memset(&A, 0, sizeof A);        // padding too: whole records are compared (build graph key)
    A.n = t->n;
    A.n_dev = t->n_dev.as<unsigned>();
    A.nsets = t->nsets;
    A.pos = pos;
    A.mass = mass;
    A.sets = t->sets.as<SetInfo>();
    A.set_of = t->set_of.as<unsigned>();
    A.bmin = t->bmin.as<unsigned long long>();
    A.bmax = t->bmax.as<unsigned long long>();
    A.keys_in = t->keys_in.as<unsigned long long>();
    A.vals_in = t->vals_in.as<unsigned>();
    A.qbuf = t->qbuf.as<uint4>();
    A.skey = t->skey.as<unsigned long long>();
    A.perm = t->perm.as<unsigned>();
    A.sp64 = t->sp64.as<double4>();
    A.spH = t->spH.as<float4>();
    A.spL = t->spL.as<float4>();
    A.sq = t->sq.as<uint4>();
    A.cap_nodes = t->cap_nodes;
    A.nd_a = t->nd_a.as<uint4>();
    A.nd_b = t->nd_b.as<uint4>();
    A.nd_r = t->nd_r.as<uint2>();
    A.nd_c = t->nd_c.as<double4>();
    A.nd_q = t->nd_q.as<double4>();
    A.nd_t = t->nd_t.as<double4>();
    A.nd_f = t->nd_f.as<float4>();
    A.nd_bnd = t->nd_bnd.as<uint4>();
    A.nd_int = t->nd_int.as<unsigned>();
    A.topo_bsum = t->topo_bs.as<unsigned>();
    A.lcp = t->lcp.as<unsigned char>();
    A.tmp_u32a = t->tmp_a.as<unsigned>();
    A.tmp_u32b = t->tmp_b.as<unsigned>();
    A.gflag = t->gflag.as<unsigned>();
    A.gbegin = t->gbegin.as<unsigned>();
    A.gr_r = t->gr_r.as<uint2>();
    A.gr_a = t->gr_a.as<uint4>();
    A.gr_b = t->gr_b.as<uint4>();
    A.n_leaf = t->prm.n_leaf;
    A.n_group = t->prm.n_group;
    A.scale = t->scale_in;
    A.massdep = t->prm.mass_dependent;
    A.scale_buf = t->scale_buf.as<double>();
    A.set_mean = t->set_mean.as<double>();
    A.ssc = t->ssc.as<double>();
    A.nd_thr = t->nd_thr.as<long long>();
    A.gr_thr = t->gr_thr.as<long long>();
    A.status = t->status.as<Status>();
    A.scan_tmp = scan_tmp_of(t);
    A.sort_tmp = sort_tmp_of(t);
    return A;
}

int read_status(pt_tree *t) {
    pt_ctx *ctx = t->ctx;
    CK(cudaMemcpyAsync(ctx->h_status, t->status.p, sizeof(Status), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    t->h = *ctx->h_status;
    return PT_OK;
}

// Build over t->n particles in t->nsets sets; pos/mass are device pointers.
// Enqueues the build between events ev[0] and ev[1]. Its ~105 short kernels
// are bound by the host's launch rate, so a build whose arguments equal the
// previous one's is captured into a CUDA graph (on the context's private
// stream) and replayed from then on.
int launch_build(pt_tree *t, const BuildArgs &A) {
    pt_ctx *ctx = t->ctx;
    const bool same_graph = t->gbuild && std::memcmp(&A, &t->gbuild_args, sizeof A) == 0;
    const bool repeat = t->have_last_build && std::memcmp(&A, &t->last_build_args, sizeof A) == 0;
    if (!same_graph && repeat) {
        if (t->gbuild) cudaGraphExecDestroy(t->gbuild);
        t->gbuild = nullptr;
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        const int nk = build_launch(A, ctx->cap_stream);
        cudaError_t ec = cudaStreamEndCapture(ctx->cap_stream, &g);
        if (ec == cudaSuccess) ec = cudaGraphInstantiate(&t->gbuild, g, 0);
        if (g) cudaGraphDestroy(g);
        if (ec != cudaSuccess) {
            (void)cudaGetLastError();
            t->gbuild = nullptr;
            return fail(ctx, PT_ERR_CUDA, "build graph capture: %s", cudaGetErrorString(ec));
        }
        t->gbuild_args = A;
        t->launches_build = nk;
    }
    CK(cudaEventRecord(ctx->ev[0], ctx->stream));
    if (t->gbuild && std::memcmp(&A, &t->gbuild_args, sizeof A) == 0) {
        CK(cudaGraphLaunch(t->gbuild, ctx->stream));
    } else {
        t->launches_build = build_launch(A, ctx->stream);
        t->last_build_args = A;
        t->have_last_build = true;
    }
    CK(cudaGetLastError());
    CK(cudaEventRecord(ctx->ev[1], ctx->stream));
    return PT_OK;
}

int run_build(pt_tree *t, const double *pos, const double *mass) {
    pt_ctx *ctx = t->ctx;
    for (int attempt = 0; attempt < 8; attempt++) {
        TRY(alloc_build(t, t->n, t->nsets));
        CK(cudaMemcpyAsync(t->sets.p, t->h_sets.data(), t->nsets * sizeof(SetInfo),
                           cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(t->n_dev.p, &t->n, 4, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemsetAsync(t->status.p, 0, sizeof(Status), ctx->stream));
        const BuildArgs A = build_args(t, pos, mass);
        TRY(launch_build(t, A));
        TRY(read_status(t));
        cudaEventElapsedTime(&t->ms_build, ctx->ev[0], ctx->ev[1]);
        const unsigned f = t->h.flags;
        if (f & kErrNonFinite) return fail(ctx, PT_ERR_ARG, "non-finite position or mass in the input");
        if (f & kErrNegMass) return fail(ctx, PT_ERR_ARG, "negative mass in the input");
        if (f & kErrBadScale) return fail(ctx, PT_ERR_ARG, "radius factor not finite and positive");
        if (f & kErrNodeCap) {
            unsigned long long c = 2ull * t->cap_nodes;
            if (c > 0x7fffffffull) return fail(ctx, PT_ERR_INTERNAL, "tree node count exceeds 2^31");
            t->cap_nodes = (unsigned)c;
            // node arrays are re-allocated for the new capacity by alloc_build
            continue;
        }
        t->built = true;
        t->lists_valid = false;
        return PT_OK;
    }
    return fail(ctx, PT_ERR_INTERNAL, "tree build did not converge on a node capacity");
}

WalkArgs walk_args(pt_tree *t) {
    WalkArgs A{};
    A.nd_a = t->nd_a.as<uint4>();
    A.nd_b = t->nd_b.as<uint4>();
    A.nd_r = t->nd_r.as<uint2>();
    A.gr_r = t->gr_r.as<uint2>();
    A.gr_a = t->gr_a.as<uint4>();
    A.gr_b = t->gr_b.as<uint4>();
    A.sets = t->sets.as<SetInfo>();
    A.nd_thr = t->nd_thr.as<long long>();
    A.gr_thr = t->gr_thr.as<long long>();
    A.massdep = t->prm.mass_dependent;
    walk_thresholds(t->prm.theta, A.wp);
    A.gr_nc = t->gr_nc.as<unsigned>();
    A.gr_np = t->gr_np.as<unsigned>();
    A.gr_co = t->gr_co.as<unsigned long long>();
    A.gr_po = t->gr_po.as<unsigned long long>();
    A.gr_nf = t->gr_nf.as<unsigned>();
    A.gr_fo = t->gr_fo.as<unsigned long long>();
    A.cells = t->cells.as<unsigned>();
    A.pp = t->pp.as<unsigned>();
    A.cap_cells = t->cap_cells;
    A.cap_pp = t->cap_pp;
    A.chunk_cells = t->chunk_cells;
    A.chunk_pp = t->chunk_pp;
    A.stack_cap = t->walk_stack;
    A.spill = t->walk_spill.as<unsigned>();
    A.spill_cap = t->walk_spill_cap;
    A.st = t->status.as<Status>();
    A.scan_tmp = scan_tmp_of(t);
    return A;
}

ForceArgs force_args(pt_tree *t, double *acc, double *pot, bool want_nb) {
    ForceArgs A{};
    A.gr_r = t->gr_r.as<uint2>();
    A.gr_a = t->gr_a.as<uint4>();
    A.gr_b = t->gr_b.as<uint4>();
    A.gr_nc = t->gr_nc.as<unsigned>();
    A.gr_np = t->gr_np.as<unsigned>();
    A.gr_co = t->gr_co.as<unsigned long long>();
    A.gr_po = t->gr_po.as<unsigned long long>();
    A.gr_nf = t->gr_nf.as<unsigned>();
    A.gr_fo = t->gr_fo.as<unsigned long long>();
    A.gr_ord = t->gr_ord.as<unsigned>();
    A.cells = t->cells.as<unsigned>();
    A.pp = t->pp.as<unsigned>();
    A.sp64 = t->sp64.as<double4>();
    A.spH = t->spH.as<float4>();
    A.spL = t->spL.as<float4>();
    A.nd_c = t->nd_c.as<double4>();
    A.nd_q = t->nd_q.as<double4>();
    A.nd_f = t->nd_f.as<float4>();
    A.sets = t->sets.as<SetInfo>();
    A.perm = t->perm.as<unsigned>();
    A.ssc = t->ssc.as<double>();
    A.massdep = t->prm.mass_dependent;
    A.acc = acc;
    A.pot = pot;
    A.G = t->prm.G;
    A.order = t->prm.order;
    A.want_nb = want_nb ? 1 : 0;
    A.pairs = t->pairs.as<uint2>();
    A.pair_cap = t->cap_pairs;
    A.gpart = t->gpart.as<double4>();
    A.red_e = t->red_part.as<double4>();
    A.red_c = reinterpret_cast<unsigned long long *>(t->red_part.as<double4>() + kRedBlocksMax);
    A.st = t->status.as<Status>();
    return A;
}

int key_bits_for(unsigned n) {
    unsigned long long nn = (unsigned long long)n * n;
    int b = 1;
    while (b < 64 && (1ull << b) < nn) b++;
    return b;
}

NbArgs nb_args(pt_tree *t) {
    NbArgs A{};
    A.n = t->n;
    A.perm = t->perm.as<unsigned>();
    A.pairs = t->pairs.as<uint2>();
    A.pair_cap = t->cap_pairs;
    A.npairs_dev = t->npairs_dev.as<unsigned>();
    A.keys = t->nb_keys.as<unsigned long long>();
    A.keys_sorted = t->nb_keys_s.as<unsigned long long>();
    A.vals = t->nb_vals.as<unsigned>();
    A.vals_sorted = t->nb_vals_s.as<unsigned>();
    A.nb_off = t->nb_off.as<long long>();
    A.nb_idx = t->nb_idx.as<int>();
    A.key_bits = key_bits_for(t->n);
    A.st = t->status.as<Status>();
    A.sort_tmp = sort_tmp_of(t);
    return A;
}

int alloc_pairs(pt_tree *t, unsigned long long cap) {
    pt_ctx *ctx = t->ctx;
    if (cap < 1024) cap = 1024;
    if (cap > 0x7fffffffull) cap = 0x7fffffffull;
    if (t->cap_pairs >= cap && t->pairs.p) return PT_OK;
    t->cap_pairs = cap;
    TRY(ensure(ctx, t->pairs, cap * 8));
    TRY(ensure(ctx, t->nb_keys, cap * 8));
    TRY(ensure(ctx, t->nb_keys_s, cap * 8));
    TRY(ensure(ctx, t->nb_vals, cap * 4));
    TRY(ensure(ctx, t->nb_vals_s, cap * 4));
    TRY(ensure(ctx, t->nb_idx, cap * 4));
    TRY(ensure(ctx, t->npairs_dev, 16));
    if (t->cap_sort < cap) {
        t->cap_sort = cap;
        TRY(ensure(ctx, t->sort_k2, cap * 8));
        TRY(ensure(ctx, t->sort_v2, cap * 4));
    }
    return PT_OK;
}

// Sizes the list arrays and chunk granules of a one-pass walk from the last
// walk's totals: chunks of about four groups' lists (about one move of a
// partial list per four groups); arrays for the estimate plus a quarter (the
// moves leave up to an eighth behind) and per active warp one and a half
// chunks left unused at the end (three for the PP array: a warp holds a near
// and a far chunk).
int size_onepass(pt_tree *t) {
    pt_ctx *ctx = t->ctx;
    const unsigned long long ngr = std::max<unsigned long long>(t->h.ngroups, 1);
    auto granule = [&](unsigned long long est) {
        unsigned long long c = 4 * (est / ngr + 1);
        return std::min<unsigned long long>(std::max<unsigned long long>(c, kWalkChunkEntries), 1ull << 22);
    };
    t->chunk_cells = granule(t->est_cells);
    t->chunk_pp = granule(t->est_pp);
    const unsigned long long warps =
        std::min<unsigned long long>((unsigned long long)walk_warps(t->walk_stack), ngr);
    const unsigned long long need_c = t->est_cells + t->est_cells / 4 + warps * t->chunk_cells * 3 / 2;
    const unsigned long long need_p = t->est_pp + t->est_pp / 4 + warps * t->chunk_pp * 3;
    if (need_c > t->cap_cells || !t->cells.p) {
        t->cap_cells = need_c;
        TRY(ensure(ctx, t->cells, t->cap_cells * 4));
    }
    if (need_p > t->cap_pp || !t->pp.p) {
        t->cap_pp = need_p;
        TRY(ensure(ctx, t->pp, t->cap_pp * 4));
    }
    return PT_OK;
}

// A walk stack overflowed: first give the warps spill areas in global memory
// (sized for the launch with the small stack, the widest), then a larger
// shared stack.
int on_walk_overflow(pt_tree *t) {
    pt_ctx *ctx = t->ctx;
    if (t->walk_spill_cap == 0) {
        TRY(ensure(ctx, t->walk_spill, (size_t)walk_warps(kWalkStackSmall) * kWalkSpill * 4));
        t->walk_spill_cap = kWalkSpill;
        return PT_OK;
    }
    if (t->walk_stack < kWalkStackLarge) {
        t->walk_stack = kWalkStackLarge;
        return PT_OK;
    }
    return fail(ctx, PT_ERR_INTERNAL, "walk stack overflow (more than %u pending nodes)",
                kWalkStackLarge + kWalkSpill);
}

// Walk + force (+ neighbour CSR) on a built tree; acc/pot are device
// pointers in input order.  On return t->h holds the status.
int run_force(pt_tree *t, double *acc, double *pot, bool want_nb, unsigned long long nb_cap_hint,
              float *ms, double *acc_host = nullptr, double *pot_host = nullptr) {
    pt_ctx *ctx = t->ctx;
    cudaStream_t st = ctx->stream;
    // host outputs: copied on the private stream as soon as the force kernel
    // has written them, while the energy sums and the neighbour CSR run (a
    // retried attempt copies again after its own force kernel)
    auto copy_out = [&]() -> int {
        if (!acc_host && !pot_host) return PT_OK;
        CK(cudaEventRecord(ctx->ev_out, st));
        CK(cudaStreamWaitEvent(ctx->out_stream, ctx->ev_out, 0));
        if (acc_host) CK(cudaMemcpyAsync(acc_host, acc, (size_t)t->n * 24, cudaMemcpyDeviceToHost, ctx->out_stream));
        if (pot_host) CK(cudaMemcpyAsync(pot_host, pot, (size_t)t->n * 8, cudaMemcpyDeviceToHost, ctx->out_stream));
        return PT_OK;
    };
    Status *dS = t->status.as<Status>();
    TRY(ensure(ctx, t->nb_off, ((size_t)t->n + 1) * 8));
    TRY(alloc_pairs(t, std::max<unsigned long long>(nb_cap_hint, 2ull * t->n)));
    bool onepass = t->est_cells > 0 && t->est_pp > 0;
    for (int attempt = 0; attempt < 6; attempt++) {
        CK(cudaMemsetAsync(&dS->flags, 0, sizeof(unsigned), st));
        CK(cudaMemsetAsync(&dS->max_stack, 0, sizeof(unsigned), st));
        CK(cudaMemsetAsync(&dS->work, 0, sizeof(dS->work), st));
        CK(cudaMemsetAsync(&dS->npairs, 0, 3 * sizeof(unsigned long long), st));   // npairs, pp_full, pp_fast
        if (onepass) {
            TRY(size_onepass(t));
            CK(cudaMemsetAsync(&dS->cell_total, 0, 2 * sizeof(unsigned long long), st));   // cell, pp totals
            CK(cudaEventRecord(ctx->ev[2], st));
            WalkArgs W = walk_args(t);
            int nk = walk_launch(W, 2, st);
            CK(cudaEventRecord(ctx->ev[3], st));
            ForceArgs F = force_args(t, acc, pot, want_nb);
            F.direct_groups = t->h.ngroups;           // known since the build's status read
            nk += force_launch(F, t->prm.precision, st);
            CK(cudaEventRecord(ctx->ev[4], st));
            TRY(copy_out());
            nk += force_reduce_launch(F, st);
            if (want_nb) nk += nb_launch(nb_args(t), st);
            t->launches_force = nk;
            CK(cudaGetLastError());
            CK(cudaEventRecord(ctx->ev[5], st));
            TRY(read_status(t));
            const unsigned f = t->h.flags;
            if (f & (kErrStack | kErrListCap)) {
                if (f & kErrStack) TRY(on_walk_overflow(t));
                onepass = false;                         // size the lists exactly
                continue;
            }
            if (want_nb && t->h.npairs > t->cap_pairs && t->h.npairs <= nb_cap_hint) {
                TRY(alloc_pairs(t, t->h.npairs + t->h.npairs / 8));
                continue;
            }
            cudaEventElapsedTime(&ms[0], ctx->ev[2], ctx->ev[3]);
            cudaEventElapsedTime(&ms[1], ctx->ev[3], ctx->ev[4]);
            cudaEventElapsedTime(&ms[2], ctx->ev[2], ctx->ev[5]);
            t->est_cells = t->h.cell_total;
            t->est_pp = t->h.pp_total;
            t->lists_valid = true;
            return PT_OK;
        }
        CK(cudaEventRecord(ctx->ev[2], st));
        WalkArgs W = walk_args(t);
        int nk = walk_launch(W, 0, st);
        CK(cudaGetLastError());
        TRY(read_status(t));
        if (t->h.flags & kErrStack) {
            TRY(on_walk_overflow(t));
            continue;
        }
        if (t->h.cell_total > t->cap_cells || !t->cells.p) {
            t->cap_cells = t->h.cell_total + t->h.cell_total / 8 + 1024;
            TRY(ensure(ctx, t->cells, t->cap_cells * 4));
        }
        if (t->h.pp_total > t->cap_pp || !t->pp.p) {
            t->cap_pp = t->h.pp_total + t->h.pp_total / 8 + 1024;
            TRY(ensure(ctx, t->pp, t->cap_pp * 4));
        }
        W = walk_args(t);
        nk += walk_launch(W, 1, st);
        CK(cudaEventRecord(ctx->ev[3], st));
        ForceArgs F = force_args(t, acc, pot, want_nb);
        F.direct_groups = t->h.ngroups;
        nk += force_launch(F, t->prm.precision, st);
        CK(cudaEventRecord(ctx->ev[4], st));
        TRY(copy_out());
        nk += force_reduce_launch(F, st);
        if (want_nb) nk += nb_launch(nb_args(t), st);
        t->launches_force = nk;
        CK(cudaGetLastError());
        CK(cudaEventRecord(ctx->ev[5], st));
        TRY(read_status(t));
        const unsigned f = t->h.flags;
        if (f & kErrStack) {                            // cannot happen after the counting pass
            TRY(on_walk_overflow(t));
            continue;
        }
        if (f & kErrListCap) continue;                  // cannot happen after sizing; retry
        if (want_nb && t->h.npairs > t->cap_pairs && t->h.npairs <= nb_cap_hint) {
            TRY(alloc_pairs(t, t->h.npairs + t->h.npairs / 8));
            continue;
        }
        cudaEventElapsedTime(&ms[0], ctx->ev[2], ctx->ev[3]);
        cudaEventElapsedTime(&ms[1], ctx->ev[3], ctx->ev[4]);
        cudaEventElapsedTime(&ms[2], ctx->ev[2], ctx->ev[5]);
        t->est_cells = t->h.cell_total;
        t->est_pp = t->h.pp_total;
        t->lists_valid = true;
        return PT_OK;
    }
    return fail(ctx, PT_ERR_INTERNAL, "force evaluation did not converge on buffer capacities");
}

void fill_stats(pt_tree *t, pt_stats *s, const float *ms) {
    if (!s) return;
    const Status &h = t->h;
    s->n = t->n;
    s->nodes = h.nnodes;
    s->groups = h.ngroups;
    s->max_level = h.max_level;
    s->cell_list_total = (int64_t)h.cell_total;
    s->pp_list_total = (int64_t)h.pp_total;
    s->cell_interactions = (int64_t)h.cell_inter;
    s->pp_interactions = (int64_t)h.pp_inter;
    s->neighbours = (int64_t)h.npairs;
    s->energy = h.energy;
    s->momentum[0] = h.mom[0];
    s->momentum[1] = h.mom[1];
    s->momentum[2] = h.mom[2];
    s->ms_build = t->ms_build;
    s->ms_walk = ms ? ms[0] : 0.0;
    s->ms_force = ms ? ms[1] : 0.0;
    s->ms_total = ms ? ms[2] : 0.0;
    s->pp_changeover_interactions = (int64_t)h.pp_full;
    s->max_walk_stack = h.max_stack;
    s->launches_build = t->launches_build;
    s->launches_force = t->launches_force;
}


// ---------------------------------------------------------------------------
// Batches (pt_batch_longrange_force): one forest over all sets.
// ---------------------------------------------------------------------------

template <typename T>
int ensure_pinned(pt_ctx *ctx, T *&p, size_t &cap, size_t n) {
    if (n <= cap && p) return PT_OK;
    if (p) {
        n = std::max(n, cap + cap / 4);
        retire(ctx, p, cap * sizeof(T), true);
    }
    p = nullptr;
    cap = 0;
    if (cudaMallocHost((void **)&p, n * sizeof(T)) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(ctx, PT_ERR_OOM, "cudaMallocHost(%zu bytes) failed", n * sizeof(T));
    }
    cap = n;
    return PT_OK;
}

int batch_tables(pt_tree *t, int nsets) {
    pt_ctx *ctx = t->ctx;
    if (t->cap_tab < nsets) {
        retire(ctx, t->h_tab, t->cap_tab * sizeof(BatchTab), true);
        retire(ctx, t->h_sets_pin, t->cap_tab * sizeof(SetInfo), true);
        retire(ctx, t->h_totals, t->cap_tab * sizeof(long long), true);
        if (t->cap_tab > 0) nsets = std::max(nsets, t->cap_tab + t->cap_tab / 4);
        t->h_tab = nullptr; t->h_sets_pin = nullptr; t->h_totals = nullptr; t->cap_tab = 0;
        if (cudaMallocHost((void **)&t->h_tab, nsets * sizeof(BatchTab)) != cudaSuccess ||
            cudaMallocHost((void **)&t->h_sets_pin, nsets * sizeof(SetInfo)) != cudaSuccess ||
            cudaMallocHost((void **)&t->h_totals, nsets * sizeof(long long)) != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(ctx, PT_ERR_OOM, "pinned batch tables");
        }
        t->cap_tab = nsets;
    }
    if (!t->h_n && cudaMallocHost((void **)&t->h_n, 16) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(ctx, PT_ERR_OOM, "pinned batch tables");
    }
    TRY(ensure(ctx, t->d_tab, (size_t)nsets * sizeof(BatchTab)));
    TRY(ensure(ctx, t->d_totals, (size_t)nsets * 8));
    TRY(ensure(ctx, t->d_acc, (size_t)t->n * 24));
    TRY(ensure(ctx, t->d_pot, (size_t)t->n * 8));
    return PT_OK;
}

// Everything a batch enqueues after the tables are filled, without any host
// synchronisation (this is what a CUDA graph captures).
int enqueue_batch(pt_tree *t, cudaStream_t st, bool host_io, bool want_nb) {
    pt_ctx *ctx = t->ctx;
    const unsigned n = t->n;
    const int C = t->nsets;
    Status *dS = t->status.as<Status>();
    BatchTab *dtab = t->d_tab.as<BatchTab>();
    SetInfo *dsets = t->sets.as<SetInfo>();
    double *ip = t->in_pos.as<double>(), *im = t->in_mass.as<double>();
    CK(cudaMemcpyAsync(dtab, t->h_tab, C * sizeof(BatchTab), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dsets, t->h_sets_pin, C * sizeof(SetInfo), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(t->n_dev.p, t->h_n, 4, cudaMemcpyHostToDevice, st));
    int nk = 0;
    double *isc = t->scale_in ? t->in_scale.as<double>() : nullptr;
    if (host_io) {
        CK(cudaMemcpyAsync(ip, t->h_io, (size_t)n * 24, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(im, t->h_io + 3ull * n, (size_t)n * 8, cudaMemcpyHostToDevice, st));
        if (isc) CK(cudaMemcpyAsync(isc, t->h_io + 4ull * n, (size_t)n * 8, cudaMemcpyHostToDevice, st));
    } else {
        nk += batch_gather_launch(dtab, dsets, C, n, ip, im, isc, st);
    }
    CK(cudaMemsetAsync(dS, 0, sizeof(Status), st));
    nk += build_launch(build_args(t, ip, im), st);
    CK(cudaMemsetAsync(&dS->flags, 0, sizeof(unsigned), st));
    WalkArgs W = walk_args(t);
    nk += walk_launch(W, 2, st);              // one pass (arrays sized before the capture)
    ForceArgs F = force_args(t, t->d_acc.as<double>(), t->d_pot.as<double>(), want_nb);
    // this step's group count is on the device: a grid sized from the last
    // step's, with head room (groups beyond it are taken from a counter)
    const unsigned long long hint = t->h.ngroups ? t->h.ngroups + t->h.ngroups / 8 + 64 : 0;
    F.direct_groups = (unsigned)std::min<unsigned long long>(hint, 0x7fffffffull);
    F.count_hint = 1;
    nk += force_launch(F, t->prm.precision, st);
    nk += force_reduce_launch(F, st);
    if (want_nb) {
        nk += nb_launch(nb_args(t), st);
        nk += batch_nb_launch(dtab, dsets, C, n, t->nb_off.as<long long>(), t->nb_idx.as<int>(),
                              t->d_totals.as<long long>(), !host_io, st);
    }
    if (host_io) {
        CK(cudaMemcpyAsync(t->h_io, t->d_acc.p, (size_t)n * 24, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(t->h_io + 3ull * n, t->d_pot.p, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
    } else {
        nk += batch_scatter_launch(dtab, dsets, C, n, t->d_acc.as<double>(), t->d_pot.as<double>(), st);
    }
    if (want_nb)
        CK(cudaMemcpyAsync(t->h_totals, t->d_totals.p, C * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ctx->h_status, dS, sizeof(Status), cudaMemcpyDeviceToHost, st));
    t->launches_force = nk;
    t->launches_build = 0;
    return PT_OK;
}

bool graph_matches(pt_tree *t, int C, const pt_cluster_desc *d, const pt_params *p, int mode) {
    if (!t->gexec || t->gkey_mode != mode || (int)t->gkey_n.size() != C) return false;
    if (std::memcmp(&t->gkey_p, p, sizeof(pt_params)) != 0) return false;
    for (int c = 0; c < C; c++)
        if (t->gkey_n[c] != (unsigned)d[c].n || t->gkey_r[2 * c] != d[c].r_in ||
            t->gkey_r[2 * c + 1] != d[c].r_out)
            return false;
    return true;
}

int batch_impl(pt_ctx *ctx, int C, pt_cluster_desc *d, const pt_params *params, int flags,
               pt_stats *stats) {
    if (C < 1 || !d) return fail(ctx, PT_ERR_ARG, "n_clusters must be >= 1");
    TRY(check_params(ctx, params));
    unsigned long long ntot = 0;
    bool want_nb = false, any_dev = false, any_host = false, any_scale = false;
    for (int c = 0; c < C; c++) {
        if (d[c].radius_scale) any_scale = true;
        if (d[c].n < 1) return fail(ctx, PT_ERR_ARG, "cluster %d: n must be >= 1", c);
        if (!d[c].pos || !d[c].mass || !d[c].acc || !d[c].pot)
            return fail(ctx, PT_ERR_ARG, "cluster %d: NULL buffer", c);
        TRY(check_radii(ctx, d[c].r_in, d[c].r_out));
        if (d[c].nb_offsets) {
            want_nb = true;
            if (d[c].nb_capacity < 0 || (d[c].nb_capacity > 0 && !d[c].nb_idx))
                return fail(ctx, PT_ERR_ARG, "cluster %d: bad neighbour buffers", c);
        }
        ntot += (unsigned long long)d[c].n;
        (is_device_ptr(d[c].pos) ? any_dev : any_host) = true;
    }
    if (any_dev && any_host) return fail(ctx, PT_ERR_ARG, "mixing host and device buffers in one batch");
    if (any_scale && !params->mass_dependent)
        return fail(ctx, PT_ERR_ARG, "radius_scale needs params->mass_dependent = 1");
    if (ntot > 0x7fffffffull) return fail(ctx, PT_ERR_ARG, "batch holds more than 2^31 particles");
    const bool host_io = any_host;
    CK(cudaSetDevice(ctx->device));
    pt_tree *t = ctx->batch_tree;
    if (!t) {
        t = new (std::nothrow) pt_tree;
        if (!t) return fail(ctx, PT_ERR_OOM, "out of host memory");
        ctx->batch_tree = t;
        t->ctx = ctx;
    }
    const unsigned n = (unsigned)ntot;
    t->n = n;
    t->nsets = C;
    t->prm = *params;
    t->h_sets.resize(C);
    unsigned long long nb_hint = 0;
    {
        unsigned b = 0;
        for (int c = 0; c < C; c++) {
            SetInfo si{};
            si.r_in = d[c].r_in;
            si.r_out = d[c].r_out;
            si.begin = b;
            si.n = (unsigned)d[c].n;
            t->h_sets[c] = si;
            b += (unsigned)d[c].n;
            nb_hint += d[c].nb_offsets ? (unsigned long long)d[c].nb_capacity : 0ull;
        }
    }
    TRY(alloc_build(t, n, C));
    TRY(batch_tables(t, C));
    TRY(ensure(ctx, t->in_pos, (size_t)n * 24));
    TRY(ensure(ctx, t->in_mass, (size_t)n * 8));
    TRY(ensure(ctx, t->nb_off, ((size_t)n + 1) * 8));
    if (any_scale) TRY(ensure(ctx, t->in_scale, (size_t)n * 8));
    t->scale_in = any_scale ? t->in_scale.as<double>() : nullptr;
    if (host_io) TRY(ensure_pinned(ctx, t->h_io, t->cap_h_io, (any_scale ? 5ull : 4ull) * n));
    // tables (pinned) and host inputs
    for (int c = 0; c < C; c++) {
        BatchTab e{};
        e.pos = d[c].pos;
        e.mass = d[c].mass;
        e.scale = d[c].radius_scale;
        e.acc = d[c].acc;
        e.pot = d[c].pot;
        e.nb_off = (long long *)d[c].nb_offsets;
        e.nb_idx = (int *)d[c].nb_idx;
        e.nb_cap = d[c].nb_offsets ? (unsigned long long)d[c].nb_capacity : 0ull;
        t->h_tab[c] = e;
        t->h_sets_pin[c] = t->h_sets[c];
        t->h_totals[c] = 0;
        if (host_io) {
            const size_t b = t->h_sets[c].begin, m = (size_t)d[c].n;
            std::memcpy(t->h_io + 3 * b, d[c].pos, m * 24);
            std::memcpy(t->h_io + 3ull * n + b, d[c].mass, m * 8);
            if (any_scale) {
                double *dst = t->h_io + 4ull * n + b;
                if (d[c].radius_scale) std::memcpy(dst, d[c].radius_scale, m * 8);
                else for (size_t k = 0; k < m; k++) dst[k] = 1.0;
            }
        }
    }
    *t->h_n = n;
    const int mode = (host_io ? 1 : 0) | (want_nb ? 2 : 0) | (any_scale ? 4 : 0);
    cudaStream_t st = ctx->stream;
    bool done = false;
    float ms[3] = {0, 0, 0};
    if ((flags & PT_BATCH_GRAPH) && graph_matches(t, C, d, params, mode)) {
        CK(cudaEventRecord(ctx->ev[6], st));
        CK(cudaGraphLaunch(t->gexec, st));
        CK(cudaEventRecord(ctx->ev[7], st));
        CK(cudaStreamSynchronize(st));
        t->h = *ctx->h_status;
        const unsigned f = t->h.flags;
        const bool pair_short = want_nb && t->h.npairs > t->cap_pairs && t->h.npairs <= nb_hint;
        if (f & (kErrNonFinite | kErrNegMass | kErrBadScale))
            return fail(ctx, PT_ERR_ARG, "non-finite position, negative mass or radius factor not finite and positive");
        if (!(f & (kErrNodeCap | kErrStack | kErrListCap)) && !pair_short) {
            done = true;
            cudaEventElapsedTime(&ms[2], ctx->ev[6], ctx->ev[7]);
        } else {
            cudaGraphExecDestroy(t->gexec);   // capacities outgrown: rebuild below
            t->gexec = nullptr;
        }
    }
    if (!done) {
        // uncaptured path: sizes every buffer, then (optionally) captures a graph
        CK(cudaMemcpyAsync(t->d_tab.p, t->h_tab, C * sizeof(BatchTab), cudaMemcpyHostToDevice, st));
        double *ip = t->in_pos.as<double>(), *im = t->in_mass.as<double>();
        double *isc = any_scale ? t->in_scale.as<double>() : nullptr;
        if (host_io) {
            CK(cudaMemcpyAsync(ip, t->h_io, (size_t)n * 24, cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(im, t->h_io + 3ull * n, (size_t)n * 8, cudaMemcpyHostToDevice, st));
            if (isc) CK(cudaMemcpyAsync(isc, t->h_io + 4ull * n, (size_t)n * 8, cudaMemcpyHostToDevice, st));
        } else {
            CK(cudaMemcpyAsync(t->sets.p, t->h_sets_pin, C * sizeof(SetInfo), cudaMemcpyHostToDevice, st));
            batch_gather_launch(t->d_tab.as<BatchTab>(), t->sets.as<SetInfo>(), C, n, ip, im, isc, st);
        }
        TRY(run_build(t, ip, im));
        TRY(run_force(t, t->d_acc.as<double>(), t->d_pot.as<double>(), want_nb, nb_hint, ms));
        BatchTab *dtab = t->d_tab.as<BatchTab>();
        SetInfo *dsets = t->sets.as<SetInfo>();
        if (want_nb)
            batch_nb_launch(dtab, dsets, C, n, t->nb_off.as<long long>(), t->nb_idx.as<int>(),
                            t->d_totals.as<long long>(), !host_io, st);
        if (host_io) {
            CK(cudaMemcpyAsync(t->h_io, t->d_acc.p, (size_t)n * 24, cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(t->h_io + 3ull * n, t->d_pot.p, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
        } else {
            batch_scatter_launch(dtab, dsets, C, n, t->d_acc.as<double>(), t->d_pot.as<double>(), st);
        }
        if (want_nb) CK(cudaMemcpyAsync(t->h_totals, t->d_totals.p, C * 8, cudaMemcpyDeviceToHost, st));
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(st));
        if (flags & PT_BATCH_GRAPH) {
            // the captured walk runs in one pass: lists sized from this step's
            // totals with head room, so that later steps of the same shape fit
            t->est_cells = t->h.cell_total;
            t->est_pp = t->h.pp_total;
            TRY(size_onepass(t));
            if (t->h.nnodes + t->h.nnodes / 4 > t->cap_nodes) {
                t->cap_nodes = t->h.nnodes + t->h.nnodes / 4 + 1024;
                TRY(alloc_build(t, n, C));
            }
            if (want_nb) TRY(alloc_pairs(t, std::max<unsigned long long>(t->cap_pairs, t->h.npairs * 2 + 1024)));
            if (t->gexec) cudaGraphExecDestroy(t->gexec);
            t->gexec = nullptr;
            const Status keep = t->h;
            cudaGraph_t g = nullptr;
            // captured on the context's private stream (the caller's stream
            // may be the legacy default stream, which cannot be captured); the
            // graph is later launched on the caller's stream
            cudaStream_t cs = ctx->cap_stream;
            CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            int rc = enqueue_batch(t, cs, host_io, want_nb);
            cudaError_t ec = cudaStreamEndCapture(cs, &g);
            if (rc != PT_OK) {
                if (g) cudaGraphDestroy(g);
                (void)cudaGetLastError();
                return rc;
            }
            if (ec != cudaSuccess) return fail(ctx, PT_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ec));
            ec = cudaGraphInstantiate(&t->gexec, g, 0);
            cudaGraphDestroy(g);
            if (ec != cudaSuccess) {
                t->gexec = nullptr;
                return fail(ctx, PT_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ec));
            }
            t->gkey_mode = mode;
            t->gkey_p = *params;
            t->gkey_n.resize(C);
            t->gkey_r.resize(2 * C);
            for (int c = 0; c < C; c++) {
                t->gkey_n[c] = (unsigned)d[c].n;
                t->gkey_r[2 * c] = d[c].r_in;
                t->gkey_r[2 * c + 1] = d[c].r_out;
            }
            t->h = keep;
        }
    }
    // outputs
    int rc = PT_OK;
    if (host_io) {
        for (int c = 0; c < C; c++) {
            const size_t b = t->h_sets[c].begin, m = (size_t)d[c].n;
            std::memcpy(d[c].acc, t->h_io + 3 * b, m * 24);
            std::memcpy(d[c].pot, t->h_io + 3ull * n + b, m * 8);
        }
    }
    if (want_nb) {
        if (host_io) {
            const unsigned long long np = std::min<unsigned long long>(t->h.npairs, t->cap_pairs);
            TRY(ensure_pinned(ctx, t->h_nboff, t->cap_h_nboff, (size_t)n + 1));
            TRY(ensure_pinned(ctx, t->h_nbidx, t->cap_h_nb, std::max<size_t>(np, 1)));
            CK(cudaMemcpyAsync(t->h_nboff, t->nb_off.p, ((size_t)n + 1) * 8, cudaMemcpyDeviceToHost, st));
            if (np) CK(cudaMemcpyAsync(t->h_nbidx, t->nb_idx.p, np * 4, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
        }
        for (int c = 0; c < C; c++) {
            d[c].nb_total = d[c].nb_offsets ? t->h_totals[c] : 0;
            if (!d[c].nb_offsets) continue;
            if (d[c].nb_total > d[c].nb_capacity || t->h.npairs > t->cap_pairs) {
                rc = fail(ctx, PT_ERR_CAPACITY, "cluster %d: neighbour lists need %lld entries, capacity %lld",
                          c, (long long)d[c].nb_total, (long long)d[c].nb_capacity);
                continue;
            }
            if (host_io) {
                const size_t b = t->h_sets[c].begin, m = (size_t)d[c].n;
                const long long o0 = t->h_nboff[b];
                for (size_t k = 0; k <= m; k++) d[c].nb_offsets[k] = t->h_nboff[b + k] - o0;
                for (long long e = 0; e < d[c].nb_total; e++) d[c].nb_idx[e] = t->h_nbidx[o0 + e] - (int)b;
            }
        }
    } else {
        for (int c = 0; c < C; c++) d[c].nb_total = 0;
    }
    fill_stats(t, stats, ms);
    return rc;
}


// ---------------------------------------------------------------------------
// Autotuner: times every (n_leaf, n_group) candidate on the caller's batch
// (device time of build + force, best of `reps`) and keeps the fastest; the
// result is cached per (sets, size buckets, theta, order, precision).
// ---------------------------------------------------------------------------

int bucket_of(unsigned long long v) {
    int b = 0;
    while ((1ull << b) < v && b < 62) b++;
    return b;
}

int autotune_impl(pt_ctx *ctx, int C, pt_cluster_desc *d, const pt_params *base, const int *leafs,
                  int nl, const int *groups, int ng, int reps, pt_params *best, double *best_ms) {
    if (C < 1 || !d || !base || !best) return fail(ctx, PT_ERR_ARG, "autotune: bad arguments");
    TRY(check_params(ctx, base));
    static const int kLeafDefault[] = {4, 8, 16, 32};
    static const int kGroupDefault[] = {32, 48, 64, 96, 128};
    if (!leafs || nl <= 0) { leafs = kLeafDefault; nl = 4; }
    if (!groups || ng <= 0) { groups = kGroupDefault; ng = 5; }
    if (reps < 1) reps = 2;
    unsigned long long ntot = 0;
    for (int c = 0; c < C; c++) ntot += (unsigned long long)(d[c].n > 0 ? d[c].n : 0);
    const int nb = bucket_of(ntot), mb = bucket_of(ntot / (unsigned long long)C);
    for (const auto &e : ctx->tune_cache)
        if (e.nsets == C && e.nbucket == nb && e.mbucket == mb && e.order == base->order &&
            e.precision == base->precision && e.theta == base->theta) {
            *best = *base;
            best->n_leaf = e.n_leaf;
            best->n_group = e.n_group;
            if (best_ms) *best_ms = e.ms;
            return PT_OK;
        }
    double bms = 1e300;
    pt_params bp = *base;
    for (int i = 0; i < nl; i++)
        for (int j = 0; j < ng; j++) {
            pt_params p = *base;
            p.n_leaf = leafs[i];
            p.n_group = groups[j];
            double ms = 1e300;
            for (int r = 0; r <= reps; r++) {        // first run sizes the buffers
                pt_stats st{};
                int rc = batch_impl(ctx, C, d, &p, 0, &st);
                if (rc != PT_OK && rc != PT_ERR_CAPACITY) return rc;
                if (r > 0) ms = std::min(ms, st.ms_build + st.ms_total);
            }
            if (ms < bms) {
                bms = ms;
                bp = p;
            }
        }
    *best = bp;
    if (best_ms) *best_ms = bms;
    ctx->tune_cache.push_back({C, nb, mb, base->order, base->precision, base->theta, bp.n_leaf,
                               bp.n_group, bms});
    return PT_OK;
}

}  // namespace

namespace pt {
int sm_count() {
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        (void)cudaGetLastError();
        return 152;
    }
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
        (void)cudaGetLastError();
        v = 152;      // grid sizing only: any positive count gives the same results
    }
    cache[dev].store(v, std::memory_order_relaxed);
    return v;
}
}  // namespace pt

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

int pt_abi_version(void) { return 1; }

int pt_ctx_create(pt_ctx **out, int device, void *stream) {
    if (!out) return PT_ERR_ARG;
    *out = nullptr;
    pt_ctx *ctx = new (std::nothrow) pt_ctx;
    if (!ctx) return PT_ERR_OOM;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
        (void)cudaGetLastError();
        delete ctx;
        return PT_ERR_CUDA;
    }
    if (device < 0 || device >= ndev) {
        delete ctx;
        return PT_ERR_ARG;
    }
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(stream);
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaMallocHost(&ctx->h_status, sizeof(Status)) != cudaSuccess) {
        (void)cudaGetLastError();
        delete ctx;
        return PT_ERR_CUDA;
    }
    for (auto &e : ctx->ev) cudaEventCreate(&e);
    if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->out_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        walk_init() != 0 || sm_count() <= 0) {
        (void)cudaGetLastError();
        pt_ctx_destroy(ctx);
        return PT_ERR_CUDA;
    }
    *out = ctx;
    return PT_OK;
}

int pt_ctx_destroy(pt_ctx *ctx) {
    if (!ctx) return PT_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->batch_tree) pt_tree_free(ctx->batch_tree);
    for (pt_tree *t : ctx->trees) {      // still alive: free their memory, detach them
        t->release();
        t->built = false;
        t->lists_valid = false;
        t->ctx = nullptr;
    }
    ctx->trees.clear();
    for (auto &e : ctx->ev)
        if (e) cudaEventDestroy(e);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->out_stream) cudaStreamDestroy(ctx->out_stream);
    if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    free_retired(ctx);
    delete ctx;
    return PT_OK;
}

const char *pt_last_error(const pt_ctx *ctx) { return ctx ? ctx->err : "no context"; }

}  // extern "C"

namespace pt {
cudaStream_t ctx_enter(pt_ctx *ctx) {
    cudaSetDevice(ctx->device);
    return ctx->stream;
}
int ctx_fail(pt_ctx *ctx, int code, const char *msg) {
    snprintf(ctx->err, sizeof ctx->err, "%s", msg);
    return code;
}
}  // namespace pt

extern "C" {

int pt_tree_build(pt_ctx *ctx, int64_t n, const double *pos, const double *mass,
                  const pt_params *params, pt_tree **tree) {
    return pt_tree_build_scaled(ctx, n, pos, mass, nullptr, params, tree);
}

int pt_tree_build_scaled(pt_ctx *ctx, int64_t n, const double *pos, const double *mass,
                         const double *radius_scale, const pt_params *params, pt_tree **tree) {
    if (!ctx) return PT_ERR_ARG;
    ctx->err[0] = 0;
    if (!tree) return fail(ctx, PT_ERR_ARG, "tree is NULL");
    if (n < 1 || n > 0x7fffffffll) return fail(ctx, PT_ERR_ARG, "n must be in [1, 2^31) (got %lld)", (long long)n);
    if (!pos || !mass) return fail(ctx, PT_ERR_ARG, "pos and mass must not be NULL");
    TRY(check_params(ctx, params));
    TRY(check_radii(ctx, params->r_in, params->r_out));
    CK(cudaSetDevice(ctx->device));
    pt_tree *t = *tree;
    if (!t) {
        t = new (std::nothrow) pt_tree;
        if (!t) return fail(ctx, PT_ERR_OOM, "out of host memory");
        *tree = t;
    }
    if (t->ctx != ctx) {
        if (t->ctx) {
            auto &v = t->ctx->trees;
            v.erase(std::remove(v.begin(), v.end(), t), v.end());
        }
        ctx->trees.push_back(t);
        t->ctx = ctx;
    }
    t->n = (unsigned)n;
    t->nsets = 1;
    t->prm = *params;
    SetInfo si{};
    si.r_in = params->r_in;
    si.r_out = params->r_out;
    si.begin = 0;
    si.n = (unsigned)n;
    t->h_sets.assign(1, si);
    if (radius_scale && !params->mass_dependent)
        return fail(ctx, PT_ERR_ARG, "radius_scale needs params->mass_dependent = 1");
    const double *dpos = pos, *dmass = mass;
    t->scale_in = nullptr;
    if (radius_scale) {
        if (is_device_ptr(radius_scale)) {
            t->scale_in = radius_scale;
        } else {
            TRY(ensure(ctx, t->in_scale, (size_t)n * 8));
            CK(cudaMemcpyAsync(t->in_scale.p, radius_scale, (size_t)n * 8, cudaMemcpyHostToDevice,
                               ctx->stream));
            t->scale_in = t->in_scale.as<double>();
        }
    }
    if (!is_device_ptr(pos)) {
        TRY(ensure(ctx, t->in_pos, (size_t)n * 24));
        CK(cudaMemcpyAsync(t->in_pos.p, pos, (size_t)n * 24, cudaMemcpyHostToDevice, ctx->stream));
        dpos = t->in_pos.as<double>();
    }
    if (!is_device_ptr(mass)) {
        TRY(ensure(ctx, t->in_mass, (size_t)n * 8));
        CK(cudaMemcpyAsync(t->in_mass.p, mass, (size_t)n * 8, cudaMemcpyHostToDevice, ctx->stream));
        dmass = t->in_mass.as<double>();
    }
    return run_build(t, dpos, dmass);
}

int pt_longrange_force(pt_ctx *ctx, pt_tree *t, double *acc, double *pot, int64_t *nb_offsets,
                       int32_t *nb_idx, int64_t nb_capacity, int64_t *nb_total, pt_stats *stats) {
    if (!ctx) return PT_ERR_ARG;
    ctx->err[0] = 0;
    if (!t || !t->built) return fail(ctx, PT_ERR_ARG, "tree is NULL or not built");
    if (!acc || !pot) return fail(ctx, PT_ERR_ARG, "acc and pot must not be NULL");
    if (nb_offsets && (!nb_idx && nb_capacity > 0)) return fail(ctx, PT_ERR_ARG, "nb_idx is NULL");
    if (nb_capacity < 0) return fail(ctx, PT_ERR_ARG, "nb_capacity < 0");
    CK(cudaSetDevice(ctx->device));
    const size_t n = t->n;
    const bool dacc = is_device_ptr(acc), dpot = is_device_ptr(pot);
    double *a = acc, *p = pot;
    if (!dacc) {
        TRY(ensure(ctx, t->out_acc, n * 24));
        a = t->out_acc.as<double>();
    }
    if (!dpot) {
        TRY(ensure(ctx, t->out_pot, n * 8));
        p = t->out_pot.as<double>();
    }
    const bool want_nb = nb_offsets != nullptr;
    float ms[3] = {0, 0, 0};
    const int rf = run_force(t, a, p, want_nb, (unsigned long long)nb_capacity, ms, dacc ? nullptr : acc,
                             dpot ? nullptr : pot);
    // no copy into the caller's host buffers may outlive the call
    if (rf != PT_OK) {
        if (!dacc || !dpot) cudaStreamSynchronize(ctx->out_stream);
        return rf;
    }
    cudaStream_t st = ctx->stream;
    int rc = PT_OK;
    const unsigned long long npairs = t->h.npairs;
    if (nb_total) *nb_total = want_nb ? (int64_t)npairs : 0;
    if (want_nb) {
        if (npairs > (unsigned long long)nb_capacity || npairs > t->cap_pairs) {
            rc = fail(ctx, PT_ERR_CAPACITY, "neighbour lists need %llu entries, capacity %lld",
                      npairs, (long long)nb_capacity);
        } else {
            cudaMemcpyKind k1 = is_device_ptr(nb_offsets) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
            CK(cudaMemcpyAsync(nb_offsets, t->nb_off.p, (n + 1) * 8, k1, st));
            if (npairs) {
                cudaMemcpyKind k2 = is_device_ptr(nb_idx) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
                CK(cudaMemcpyAsync(nb_idx, t->nb_idx.p, npairs * 4, k2, st));
            }
        }
    }
    CK(cudaStreamSynchronize(st));
    if (!dacc || !dpot) CK(cudaStreamSynchronize(ctx->out_stream));
    fill_stats(t, stats, ms);
    return rc;
}

int pt_orbit_neighbours(pt_tree *t, const double *vel, const pt_orbit_params *op, int64_t *nb_offsets,
                        int32_t *nb_idx, int64_t nb_capacity, int64_t *nb_total, int64_t *n_candidates,
                        double *r_nb) {
    if (!t || !t->ctx) return PT_ERR_ARG;
    pt_ctx *ctx = t->ctx;
    ctx->err[0] = 0;
    if (!t->built) return fail(ctx, PT_ERR_ARG, "tree is not built");
    if (!vel || !op) return fail(ctx, PT_ERR_ARG, "vel and params must not be NULL");
    if (!(op->dt >= 0.0) || !std::isfinite(op->dt) || !(op->C_r >= 0.0) || !std::isfinite(op->C_r) ||
        !(op->C_v >= 0.0) || !std::isfinite(op->C_v))
        return fail(ctx, PT_ERR_ARG, "need finite dt, C_r, C_v >= 0");
    if (op->mode < PT_ORBIT_ROUT || op->mode > PT_ORBIT_CANDIDATES)
        return fail(ctx, PT_ERR_ARG, "unknown orbit mode %d", op->mode);
    if (nb_capacity < 0) return fail(ctx, PT_ERR_ARG, "nb_capacity < 0");
    if (nb_offsets && !nb_idx && nb_capacity > 0) return fail(ctx, PT_ERR_ARG, "nb_idx is NULL");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const size_t n = t->n;
    const double *dvel = vel;
    if (!is_device_ptr(vel)) {
        TRY(ensure(ctx, t->orb_vel, n * 24));
        CK(cudaMemcpyAsync(t->orb_vel.p, vel, n * 24, cudaMemcpyHostToDevice, st));
        dvel = t->orb_vel.as<double>();
    }
    double *drnb = nullptr;
    if (r_nb) {
        if (is_device_ptr(r_nb)) {
            drnb = r_nb;
        } else {
            TRY(ensure(ctx, t->orb_rnb, n * 8));
            drnb = t->orb_rnb.as<double>();
        }
    }
    TRY(ensure(ctx, t->orb_sv, n * 32));
    TRY(ensure(ctx, t->orb_rnbf, n * 4));
    TRY(ensure(ctx, t->orb_ndr, (size_t)t->cap_nodes * 8));
    TRY(ensure(ctx, t->orb_ndthr, (size_t)t->cap_nodes * 8));
    TRY(ensure(ctx, t->orb_grthr, n * 8));
    TRY(ensure(ctx, t->orb_ctr, 16));
    TRY(ensure(ctx, t->nb_off, (n + 1) * 8));
    const bool want_nb = nb_offsets != nullptr;
    TRY(alloc_pairs(t, std::max<unsigned long long>((unsigned long long)nb_capacity, 2ull * n)));
    Status *dS = t->status.as<Status>();
    unsigned stack = kOrbitStack;
    unsigned long long ctr[2] = {0, 0};
    for (int attempt = 0; attempt < 6; attempt++) {
        CK(cudaMemsetAsync(&dS->flags, 0, sizeof(unsigned), st));
        CK(cudaMemsetAsync(&dS->npairs, 0, sizeof(unsigned long long), st));
        CK(cudaMemsetAsync(t->orb_ctr.p, 0, 16, st));
        OrbitArgs A{};
        A.n = t->n;
        A.perm = t->perm.as<unsigned>();
        A.sp64 = t->sp64.as<double4>();
        A.spH = t->spH.as<float4>();
        A.spL = t->spL.as<float4>();
        A.sq = t->sq.as<uint4>();
        A.ssc = t->ssc.as<double>();
        A.massdep = t->prm.mass_dependent;
        A.sets = t->sets.as<SetInfo>();
        A.nd_a = t->nd_a.as<uint4>();
        A.nd_b = t->nd_b.as<uint4>();
        A.nd_r = t->nd_r.as<uint2>();
        A.gr_r = t->gr_r.as<uint2>();
        A.gr_a = t->gr_a.as<uint4>();
        A.gr_b = t->gr_b.as<uint4>();
        A.vel = dvel;
        A.dt = op->dt;
        A.C_r = op->C_r;
        A.C_v = op->C_v;
        A.G = t->prm.G;
        A.mode = op->mode;
        A.sv = t->orb_sv.as<double4>();
        A.rnbf = t->orb_rnbf.as<float>();
        A.nd_rnb = t->orb_ndr.as<double>();
        A.nd_thr = t->orb_ndthr.as<long long>();
        A.gr_thr = t->orb_grthr.as<long long>();
        A.rnb_out = drnb;
        A.pairs = t->pairs.as<uint2>();
        A.pair_cap = t->cap_pairs;
        A.ctr = t->orb_ctr.as<unsigned long long>();
        A.stack_cap = stack;
        A.cap_nodes = t->cap_nodes;
        A.st = dS;
        if (orbit_launch(A, st) < 0) return fail(ctx, PT_ERR_CUDA, "orbit search: kernel attribute refused");
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(ctx->h_status, t->orb_ctr.p, 16, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        memcpy(ctr, ctx->h_status, 16);
        TRY(read_status(t));
        if (t->h.flags & kErrStack) {
            if (stack < kWalkStackLarge) {
                stack = kWalkStackLarge;
                continue;
            }
            return fail(ctx, PT_ERR_INTERNAL, "orbit search stack overflow (more than %u pending nodes)", stack);
        }
        if (want_nb && t->h.npairs > t->cap_pairs && t->h.npairs <= (unsigned long long)nb_capacity) {
            TRY(alloc_pairs(t, t->h.npairs + t->h.npairs / 8));
            continue;
        }
        break;
    }
    if (t->h.flags & kErrStack) return fail(ctx, PT_ERR_INTERNAL, "orbit search did not converge");
    const unsigned long long npairs = t->h.npairs;
    if (n_candidates) *n_candidates = (int64_t)ctr[1];
    if (nb_total) *nb_total = (int64_t)npairs;
    int rc = PT_OK;
    if (drnb && drnb != r_nb) CK(cudaMemcpyAsync(r_nb, drnb, n * 8, cudaMemcpyDeviceToHost, st));
    if (want_nb) {
        if (npairs > (unsigned long long)nb_capacity || npairs > t->cap_pairs) {
            rc = fail(ctx, PT_ERR_CAPACITY, "orbit neighbour lists need %llu entries, capacity %lld",
                      npairs, (long long)nb_capacity);
        } else {
            nb_launch(nb_args(t), st);
            CK(cudaGetLastError());
            cudaMemcpyKind k1 = is_device_ptr(nb_offsets) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
            CK(cudaMemcpyAsync(nb_offsets, t->nb_off.p, (n + 1) * 8, k1, st));
            if (npairs) {
                cudaMemcpyKind k2 = is_device_ptr(nb_idx) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
                CK(cudaMemcpyAsync(nb_idx, t->nb_idx.p, npairs * 4, k2, st));
            }
        }
    }
    CK(cudaStreamSynchronize(st));
    return rc;
}

int pt_tree_free(pt_tree *t) {
    if (!t) return PT_OK;
    if (t->ctx) {
        cudaSetDevice(t->ctx->device);
        cudaStreamSynchronize(t->ctx->stream);
        auto &v = t->ctx->trees;
        v.erase(std::remove(v.begin(), v.end(), t), v.end());
    }
    t->release();
    delete t;
    return PT_OK;
}

// ---- introspection --------------------------------------------------------

int pt_tree_info(pt_tree *t, int64_t *info, double *box) {
    if (!t || !t->built) return PT_ERR_ARG;
    pt_ctx *ctx = t->ctx;
    if (info) {
        info[0] = t->n;
        info[1] = t->h.nnodes;
        info[2] = t->h.ngroups;
        info[3] = t->h.max_level;
        info[4] = t->nsets;
    }
    if (box) {
        std::vector<SetInfo> s(t->nsets);
        CK(cudaMemcpy(s.data(), t->sets.p, t->nsets * sizeof(SetInfo), cudaMemcpyDeviceToHost));
        for (int k = 0; k < t->nsets; k++) {
            for (int d = 0; d < 3; d++) box[5 * k + d] = s[k].origin[d];
            box[5 * k + 3] = s[k].S;
            box[5 * k + 4] = s[k].scale;
        }
    }
    return PT_OK;
}

int pt_tree_keys(pt_tree *t, uint64_t *keys, uint32_t *perm) {
    if (!t || !t->built) return PT_ERR_ARG;
    pt_ctx *ctx = t->ctx;
    if (keys) CK(cudaMemcpy(keys, t->skey.p, (size_t)t->n * 8, cudaMemcpyDeviceToHost));
    if (perm) CK(cudaMemcpy(perm, t->perm.p, (size_t)t->n * 4, cudaMemcpyDeviceToHost));
    return PT_OK;
}

int pt_tree_nodes(pt_tree *t, int64_t *ints, uint32_t *q, double *mom) {
    if (!t || !t->built) return PT_ERR_ARG;
    pt_ctx *ctx = t->ctx;
    const size_t nn = t->h.nnodes;
    std::vector<uint4> a(nn), b(nn);
    std::vector<uint2> r(nn);
    std::vector<double4> c(nn), qq(2 * nn);
    CK(cudaMemcpy(a.data(), t->nd_a.p, nn * 16, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(b.data(), t->nd_b.p, nn * 16, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(r.data(), t->nd_r.p, nn * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(c.data(), t->nd_c.p, nn * 32, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(qq.data(), t->nd_q.p, nn * 64, cudaMemcpyDeviceToHost));
    for (size_t v = 0; v < nn; v++) {
        if (ints) {
            int64_t *o = ints + 8 * v;
            o[0] = r[v].x;
            o[1] = r[v].y;
            o[2] = meta_level(a[v].w);
            o[3] = meta_leaf(a[v].w);
            o[4] = meta_leaf(a[v].w) ? -1 : (int64_t)b[v].w;
            o[5] = meta_nchild(a[v].w);
            o[6] = 0;
            o[7] = 0;
        }
        if (q) {
            uint32_t *o = q + 6 * v;
            o[0] = a[v].x; o[1] = a[v].y; o[2] = a[v].z;
            o[3] = b[v].x; o[4] = b[v].y; o[5] = b[v].z;
        }
        if (mom) {
            double *o = mom + 10 * v;
            o[0] = c[v].w; o[1] = c[v].x; o[2] = c[v].y; o[3] = c[v].z;
            o[4] = qq[2 * v].x; o[5] = qq[2 * v].y; o[6] = qq[2 * v].z; o[7] = qq[2 * v].w;
            o[8] = qq[2 * v + 1].x; o[9] = qq[2 * v + 1].y;
        }
    }
    return PT_OK;
}

int pt_tree_groups(pt_tree *t, int64_t *g) {
    if (!t || !t->built || !g) return PT_ERR_ARG;
    pt_ctx *ctx = t->ctx;
    const size_t ng = t->h.ngroups;
    std::vector<uint2> r(ng);
    std::vector<uint4> a(ng), b(ng);
    CK(cudaMemcpy(r.data(), t->gr_r.p, ng * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(a.data(), t->gr_a.p, ng * 16, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(b.data(), t->gr_b.p, ng * 16, cudaMemcpyDeviceToHost));
    for (size_t k = 0; k < ng; k++) {
        int64_t *o = g + 8 * k;
        o[0] = r[k].x; o[1] = r[k].y;
        o[2] = a[k].x; o[3] = a[k].y; o[4] = a[k].z;
        o[5] = b[k].x; o[6] = b[k].y; o[7] = b[k].z;
    }
    return PT_OK;
}

// Group-order CSR copy of one list kind; the device arrays hold each group's
// entries contiguously at its offset (in group order after a two-pass walk,
// in allocation order after a one-pass walk).
// Per-group lists as CSR: each group's segment (off_b, cnt_b) followed by its
// second segment (off2_b, cnt2_b) when given (the far PP entries).
static int lists_csr(pt_tree *t, const Buf &off_b, const Buf &cnt_b, const Buf *off2_b, const Buf *cnt2_b,
                     const Buf &arr, int64_t *off_out, uint32_t *out) {
    pt_ctx *ctx = t->ctx;
    const size_t ng = t->h.ngroups;
    const int nseg = off2_b ? 2 : 1;
    std::vector<unsigned long long> off(nseg * ng);
    std::vector<unsigned> cnt(nseg * ng);
    CK(cudaMemcpy(off.data(), off_b.p, ng * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(cnt.data(), cnt_b.p, ng * 4, cudaMemcpyDeviceToHost));
    if (off2_b) {
        CK(cudaMemcpy(off.data() + ng, off2_b->p, ng * 8, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(cnt.data() + ng, cnt2_b->p, ng * 4, cudaMemcpyDeviceToHost));
    }
    unsigned long long extent = 0, total = 0;
    for (size_t k = 0; k < nseg * ng; k++) {
        extent = std::max(extent, off[k] + cnt[k]);
        total += cnt[k];
    }
    if (off_out) {
        int64_t acc = 0;
        for (size_t k = 0; k < ng; k++) {
            off_out[k] = acc;
            for (int q = 0; q < nseg; q++) acc += cnt[q * ng + k];
        }
        off_out[ng] = acc;
    }
    if (out && total) {
        std::vector<uint32_t> all(extent);
        CK(cudaMemcpy(all.data(), arr.p, extent * 4, cudaMemcpyDeviceToHost));
        size_t at = 0;
        for (size_t k = 0; k < ng; k++)
            for (int q = 0; q < nseg; q++)
                for (unsigned e = 0; e < cnt[q * ng + k]; e++) out[at++] = all[off[q * ng + k] + e];
    }
    return PT_OK;
}

int pt_tree_lists(pt_tree *t, int64_t *cell_off, uint32_t *cells, int64_t *pp_off, uint32_t *pp) {
    if (!t || !t->lists_valid) return PT_ERR_ARG;
    TRY(lists_csr(t, t->gr_co, t->gr_nc, nullptr, nullptr, t->cells, cell_off, cells));
    TRY(lists_csr(t, t->gr_po, t->gr_np, &t->gr_fo, &t->gr_nf, t->pp, pp_off, pp));
    return PT_OK;
}

int pt_batch_longrange_force(pt_ctx *ctx, int n_clusters, pt_cluster_desc *desc,
                             const pt_params *params, int flags, pt_stats *stats) {
    if (!ctx) return PT_ERR_ARG;
    ctx->err[0] = 0;
    return batch_impl(ctx, n_clusters, desc, params, flags, stats);
}

int pt_autotune(pt_ctx *ctx, int n_clusters, pt_cluster_desc *desc, const pt_params *base,
                const int *leaf_candidates, int n_leaf_candidates, const int *group_candidates,
                int n_group_candidates, int reps, pt_params *best, double *best_ms) {
    if (!ctx) return PT_ERR_ARG;
    ctx->err[0] = 0;
    return autotune_impl(ctx, n_clusters, desc, base, leaf_candidates, n_leaf_candidates,
                         group_candidates, n_group_candidates, reps, best, best_ms);
}

}  // extern "C"
