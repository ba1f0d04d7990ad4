// pt_kernels.cuh -- launch arguments of the build, walk and force stages
// (internal to libpt.so).
#pragma once

#include "pt_internal.cuh"

struct pt_ctx;

namespace pt {

constexpr unsigned kWalkStackSmall = 768;    // per-warp walk stack entries (shared memory)
constexpr unsigned kWalkStackLarge = 12288;  // retry size after an overflow
constexpr unsigned kOrbitStack = 2048;       // per-warp stack of the orbit-dependent search
constexpr unsigned kWalkMaxIters = 1u << 24;   // safety cap on walk iterations per group
constexpr unsigned long long kWalkChunkEntries = 8192;   // one-pass list allocation granule

struct BuildArgs {
    unsigned n;                      // particles (all sets)
    const unsigned *n_dev;           // device copy of n
    int nsets;
    const double *pos, *mass;        // input order (device)
    SetInfo *sets;                   // nsets
    unsigned *set_of;                // n (only when nsets > 1)
    unsigned long long *bmin, *bmax; // 3 * nsets
    unsigned long long *keys_in;     // n
    unsigned *vals_in;               // n
    uint4 *qbuf;                     // n
    unsigned long long *skey;        // n
    unsigned *perm;                  // n
    double4 *sp64;
    float4 *spH, *spL;
    uint4 *sq;
    // nodes
    unsigned cap_nodes;
    uint4 *nd_a, *nd_b;
    uint2 *nd_r;
    double4 *nd_c, *nd_q, *nd_t;
    float4 *nd_f;
    uint4 *nd_bnd;                   // 2 per node: child boundaries of split nodes (build only)
    unsigned *nd_int;                // per level from lvl_begin: its internal nodes (build only)
    unsigned *topo_bsum;             // children counted per block of the topology grid (build only)
    unsigned char *lcp;              // n + 32 bytes: shared key digits of neighbours (build only)
    unsigned *tmp_u32a, *tmp_u32b;   // max(cap_nodes, n) each
    // groups
    unsigned *gflag, *gbegin;        // n each
    uint2 *gr_r;
    uint4 *gr_a, *gr_b;
    int n_leaf, n_group;
    // mass-dependent changeover radii (Eq. 12): per-particle factors in input
    // order (NULL: computed from the masses when massdep, else all 1)
    const double *scale;
    int massdep;
    double *scale_buf;               // n (device-computed factors)
    double *set_mean;                // nsets
    double *ssc;                     // n, sorted factors
    long long *nd_thr, *gr_thr;      // gap thresholds per node / group
    Status *status;
    ScanTmp scan_tmp;
    SortTmp sort_tmp;
};

struct WalkArgs {
    const uint4 *nd_a, *nd_b;
    const uint2 *nd_r;
    const uint2 *gr_r;
    const uint4 *gr_a, *gr_b;
    const SetInfo *sets;
    const long long *nd_thr, *gr_thr;    // per node / group gap thresholds (massdep)
    int massdep;
    WalkParams wp;
    unsigned *gr_nc, *gr_np;
    unsigned long long *gr_co, *gr_po;   // ngroups + 1
    // PP entries of leaves whose box is at least r_out from the group's box
    // (opened for the opening angle only: no pair within r_out), kept apart
    unsigned *gr_nf;
    unsigned long long *gr_fo;
    unsigned *cells, *pp;
    unsigned long long cap_cells, cap_pp;
    unsigned long long chunk_cells, chunk_pp;   // one-pass allocation granules (entries)
    unsigned stack_cap;                  // stack entries per warp
    unsigned *spill;                     // per-warp spill areas of the stack (global memory)
    unsigned spill_cap;                  // entries per warp in the spill area
    Status *st;
    ScanTmp scan_tmp;
};

struct ForceArgs {
    const uint2 *gr_r;
    const uint4 *gr_a, *gr_b;        // group grid boxes (qmin, set), (qmax, -)
    const unsigned *gr_nc, *gr_np;
    const unsigned long long *gr_co, *gr_po;
    const unsigned *gr_nf;           // far PP segment (no pair within r_out)
    const unsigned long long *gr_fo;
    unsigned *gr_ord;                // mixed kernel: group processing order (written per launch)
    const unsigned *cells, *pp;
    const double4 *sp64;
    const float4 *spH, *spL;
    const double4 *nd_c, *nd_q;
    const float4 *nd_f;
    const SetInfo *sets;
    const unsigned *perm;
    const double *ssc;               // sorted radius factors (massdep)
    int massdep;
    double *acc, *pot;               // input (caller) order, device
    double G;
    int order;                       // 0 or 2
    int want_nb;
    uint2 *pairs;                    // (sorted i, sorted j)
    unsigned long long pair_cap;
    // CTAs of the launch, each first taking the group of its own index: the
    // group count when the host knows it (after the build), else a hint (a
    // batch's count from its previous step, with head room: the count is on
    // the device when a step is enqueued or captured); groups beyond the grid
    // go to CTAs that take them from an atomic counter.  0: a persistent
    // launch taking every group from the counter.
    unsigned direct_groups;
    unsigned count_hint;             // 1: direct_groups is a hint (take groups beyond it)
    double4 *gpart;                  // per group: sum m phi / 2, sum m a
    double4 *red_e;                  // per reduction block: partial sums of gpart
    unsigned long long *red_c;       // per reduction block: cell and PP interaction counts
    Status *st;
};

struct NbArgs {
    unsigned n;                      // particles (all sets)
    const unsigned *perm;
    const uint2 *pairs;
    unsigned long long pair_cap;
    unsigned *npairs_dev;            // clamped pair count (device)
    unsigned long long *keys, *keys_sorted;
    unsigned *vals, *vals_sorted;
    long long *nb_off;               // n + 1 (global CSR, input order)
    int *nb_idx;                     // pair_cap
    int key_bits;
    Status *st;
    SortTmp sort_tmp;
};

// Orbit-dependent neighbour search (Sec. 6.3.1, Eq. 24) on a built tree.
struct OrbitArgs {
    unsigned n;
    const unsigned *perm;
    const double4 *sp64;
    const float4 *spH, *spL;             // float-float split of the sorted positions
    const uint4 *sq;
    const double *ssc;
    int massdep;
    const SetInfo *sets;
    const uint4 *nd_a, *nd_b;
    const uint2 *nd_r;
    const uint2 *gr_r;
    const uint4 *gr_a, *gr_b;
    const double *vel;                   // input order, n x 3 (device)
    double dt, C_r, C_v, G;
    int mode;                            // 0 r_out reference, 1 r_nb reference, 2 candidates
    double4 *sv;                         // sorted (v, r_nb)
    float *rnbf;                         // sorted r_nb as float (prefilter)
    double *nd_rnb;                      // per node: largest r_nb
    long long *nd_thr, *gr_thr;          // gap thresholds from r_nb
    double *rnb_out;                     // optional: r_nb in input order
    uint2 *pairs;
    unsigned long long pair_cap;
    unsigned long long *ctr;             // [0] work counter, [1] candidates
    unsigned stack_cap;
    unsigned cap_nodes;
    Status *st;
};
int orbit_launch(const OrbitArgs &A, cudaStream_t st);

// Per-set pointer table of a batch (device resident).
struct BatchTab {
    const double *pos, *mass;
    const double *scale;             // radius factors or NULL
    double *acc, *pot;
    long long *nb_off;
    int *nb_idx;
    unsigned long long nb_cap;
};

int batch_gather_launch(const BatchTab *tab, const SetInfo *sets, int nsets, unsigned n,
                        double *pos, double *mass, double *scale, cudaStream_t st);
int batch_scatter_launch(const BatchTab *tab, const SetInfo *sets, int nsets, unsigned n,
                         const double *acc, const double *pot, cudaStream_t st);
int batch_nb_launch(const BatchTab *tab, const SetInfo *sets, int nsets, unsigned n,
                    const long long *off, const int *idx, long long *totals, bool split,
                    cudaStream_t st);
int build_launch(const BuildArgs &A, cudaStream_t st);   // returns kernels launched
int walk_init();   // once per context: kernel attributes of the walk
// Context access for the auxiliary entry points outside pt_api.cu: selects the
// context's device and returns its stream; ctx_fail records a message.
cudaStream_t ctx_enter(pt_ctx *ctx);
int ctx_fail(pt_ctx *ctx, int code, const char *msg);
int walk_warps(unsigned stack_cap);   // warps of a walk launch with this stack size
constexpr unsigned kWalkSpill = 4096;    // per-warp spill entries of the walk stack (global memory)
int walk_launch(const WalkArgs &A, int phase, cudaStream_t st);    // 0 count+scan, 1 fill, 2 one pass
int force_launch(const ForceArgs &A, int precision, cudaStream_t st);
constexpr int kRedBlocksMax = 256;    // partial-sum slots of the force's energy / momentum reduction
int force_reduce_launch(const ForceArgs &A, cudaStream_t st);
int nb_launch(const NbArgs &A, cudaStream_t st);

}  // namespace pt
