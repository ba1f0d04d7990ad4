// pt_orbit.cu -- orbit-dependent neighbour search (Sec. 6.3.1, Eq. 24).
//
// Stage 1: every particle searches within r_nb,i = s_i r_out + C_r |v_i| dt_L
// and j != i is a candidate of i when r_ij < max(r_nb,i, r_nb,j).  Stage 2
// keeps a candidate when the pericentre of the pair's Kepler orbit is below
// C_v times the reference radius (r_out,ij by default, r_nb,ij in the printed
// form, which keeps every candidate because a pericentre never exceeds the
// current separation).
//
// The search runs on the octree of pt_tree_build: every node carries the
// largest r_nb of its particles (bottom-up, one launch per level) and every
// group the largest of its members; a warp walks one group and opens a node
// unless the integer gap between the group's and the node's grid boxes rules
// out every pair (the same conservative gap test as the r_out test of the
// interaction walk, with the larger of the two radii).  Candidate pairs are
// then decided in float64 with one IEEE operation at a time (no
// contraction), so the lists are bit-identical to a brute-force search.
#include "pt_kernels.cuh"

namespace pt {

constexpr int kOrbWarps = 4;
constexpr int kOrbThreads = 32 * kOrbWarps;
constexpr unsigned kOrbMaxIters = 1u << 24;   // guard against a corrupted tree

__device__ __forceinline__ long long radius_threshold(double R, double scale) {
    const double Rg = __dmul_rn(R, scale);
    const double R2 = __dmul_rn(Rg, Rg);
    return (R2 > 4.0e18) ? 4000000000000000000ll : (long long)floor(R2) + 2;
}

// Sorted velocities and Eq. 24 radii.
__global__ void k_orbit_prep(OrbitArgs A) {
    for (unsigned p = blockIdx.x * blockDim.x + threadIdx.x; p < A.n; p += gridDim.x * blockDim.x) {
        const unsigned i = A.perm[p];
        const double vx = A.vel[3ull * i], vy = A.vel[3ull * i + 1], vz = A.vel[3ull * i + 2];
        const double vv = __dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz));
        const double sp = __dsqrt_rn(vv);
        const double ro = __dmul_rn(A.sets[A.sq[p].w].r_out, A.massdep ? A.ssc[p] : 1.0);
        const double rnb = __dadd_rn(ro, __dmul_rn(A.C_r, __dmul_rn(sp, A.dt)));
        A.sv[p] = make_double4(vx, vy, vz, rnb);
        A.rnbf[p] = __double2float_rn(rnb);
        if (A.rnb_out) A.rnb_out[i] = rnb;
    }
}

// Largest r_nb per node, level l (leaves from their particles, internal
// nodes from their children, which sit one level deeper).
__global__ void k_orbit_nodes(OrbitArgs A, int l) {
    unsigned b0 = A.st->lvl_begin[l], cnt = A.st->lvl_count[l];
    if (b0 >= A.cap_nodes) return;
    if (cnt > A.cap_nodes - b0) cnt = A.cap_nodes - b0;
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
        const unsigned v = b0 + k;
        const uint4 a = A.nd_a[v];
        double R = 0.0;
        if (meta_leaf(a.w)) {
            const uint2 r = A.nd_r[v];
            for (unsigned p = r.x; p < r.x + r.y; p++) R = fmax(R, A.sv[p].w);
        } else {
            const unsigned fc = A.nd_b[v].w, nc = meta_nchild(a.w);
            if (fc >= A.cap_nodes || nc > A.cap_nodes - fc) continue;
            for (unsigned c = fc; c < fc + nc; c++) R = fmax(R, A.nd_rnb[c]);
        }
        A.nd_rnb[v] = R;
        const uint2 r = A.nd_r[v];
        A.nd_thr[v] = radius_threshold(R, A.sets[A.sq[r.x].w].scale);
    }
}

__global__ void k_orbit_groups(OrbitArgs A) {
    const unsigned ng = A.st->ngroups;
    for (unsigned g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        const uint2 r = A.gr_r[g];
        double R = 0.0;
        for (unsigned p = r.x; p < r.x + r.y; p++) R = fmax(R, A.sv[p].w);
        A.gr_thr[g] = radius_threshold(R, A.sets[A.gr_a[g].w].scale);
    }
}

// Kepler pericentre of the relative orbit (eccentricity-vector form; see pt.h).
__device__ __forceinline__ double dot3(double ax, double ay, double az, double bx, double by, double bz) {
    return __dadd_rn(__dadd_rn(__dmul_rn(ax, bx), __dmul_rn(ay, by)), __dmul_rn(az, bz));
}
__device__ __forceinline__ double pericentre(double dx, double dy, double dz, double vx, double vy,
                                             double vz, double mu) {
    const double r2 = dot3(dx, dy, dz, dx, dy, dz);
    const double v2 = dot3(vx, vy, vz, vx, vy, vz);
    if (v2 == 0.0) return __dsqrt_rn(r2);
    const double cx = __dsub_rn(__dmul_rn(dy, vz), __dmul_rn(dz, vy));
    const double cy = __dsub_rn(__dmul_rn(dz, vx), __dmul_rn(dx, vz));
    const double cz = __dsub_rn(__dmul_rn(dx, vy), __dmul_rn(dy, vx));
    const double h2 = dot3(cx, cy, cz, cx, cy, cz);
    if (mu == 0.0) return __dsqrt_rn(__ddiv_rn(h2, v2));
    const double r = __dsqrt_rn(r2);
    const double a = __dsub_rn(v2, __ddiv_rn(mu, r));
    const double b = dot3(dx, dy, dz, vx, vy, vz);
    const double ex = __dsub_rn(__dmul_rn(a, dx), __dmul_rn(b, vx));
    const double ey = __dsub_rn(__dmul_rn(a, dy), __dmul_rn(b, vy));
    const double ez = __dsub_rn(__dmul_rn(a, dz), __dmul_rn(b, vz));
    const double e = __ddiv_rn(__dsqrt_rn(dot3(ex, ey, ez, ex, ey, ez)), mu);
    return __ddiv_rn(__ddiv_rn(h2, mu), __dadd_rn(1.0, e));
}

// 0: not a candidate, 1: candidate dropped by stage 2, 2: neighbour.
__device__ __forceinline__ int orbit_pair(const OrbitArgs &A, unsigned pi, unsigned pj) {
    const double4 xi = A.sp64[pi], xj = A.sp64[pj];
    const double4 vi = A.sv[pi], vj = A.sv[pj];
    const double dx = __dsub_rn(xj.x, xi.x), dy = __dsub_rn(xj.y, xi.y), dz = __dsub_rn(xj.z, xi.z);
    const double r2 = dot3(dx, dy, dz, dx, dy, dz);
    const double R = fmax(vi.w, vj.w);
    if (!(r2 < __dmul_rn(R, R))) return 0;
    if (A.mode == 2) return 2;
    const double rp = pericentre(dx, dy, dz, __dsub_rn(vj.x, vi.x), __dsub_rn(vj.y, vi.y),
                                 __dsub_rn(vj.z, vi.z), __dmul_rn(A.G, __dadd_rn(xi.w, xj.w)));
    double Rs = R;
    if (A.mode == 0) {
        const double s = A.massdep ? fmax(A.ssc[pi], A.ssc[pj]) : 1.0;
        Rs = __dmul_rn(A.sets[A.sq[pi].w].r_out, s);
    }
    return rp < __dmul_rn(A.C_v, Rs) ? 2 : 1;
}

constexpr int kOrbChunk = 128;     // opened-leaf particles staged per warp

// Candidate tests of the staged particles against every member of group g:
// a float32 prefilter on float-float differences with a 2^-10 margin on
// r_nb^2 (it can only let extra pairs through), then the exact float64 test
// and the pericentre in orbit_pair.  The prefilter runs branch-free over 32
// staged particles at a time into a bit mask (the chunk is padded to a
// multiple of 32 with massless particles far away); only the set bits take
// the float64 path.  Candidates are counted, kept pairs appended to the
// pair buffer.
__device__ __forceinline__ void orbit_chunk(const OrbitArgs &A, const uint2 gr, int fill,
                                            float4 *cH, float4 *cL, float *cR, unsigned *cI,
                                            unsigned long long &ncand) {
    const unsigned lane = threadIdx.x & 31;
    const int fill32 = (fill + 31) & ~31;             // <= kOrbChunk, a multiple of 32
    if ((int)lane + fill < fill32) {
        const int e = fill + (int)lane;
        cH[e] = make_float4(1e15f, 1e15f, 1e15f, 0.0f);
        cL[e] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        cR[e] = 0.0f;
        cI[e] = 0xffffffffu;
    }
    __syncwarp();
    for (unsigned t0 = 0; t0 < gr.y; t0 += 32) {
        const unsigned t = t0 + lane;
        const bool valid = t < gr.y;
        const unsigned pi = gr.x + (valid ? t : 0u);
        const float4 Hi = A.spH[pi], Li = A.spL[pi];
        const float ri = A.rnbf[pi];
        for (int e0 = 0; e0 < fill32; e0 += 32) {
            unsigned hit = 0u;
#pragma unroll 8
            for (int q = 0; q < 32; q++) {
                const float4 Hj = cH[e0 + q], Lj = cL[e0 + q];
                const float dx = (Hj.x - Hi.x) + (Lj.x - Li.x);
                const float dy = (Hj.y - Hi.y) + (Lj.y - Li.y);
                const float dz = (Hj.z - Hi.z) + (Lj.z - Li.z);
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                const float R = fmaxf(ri, cR[e0 + q]);
                hit |= (r2 < R * R * (1.0f + 1.0f / 1024.0f) ? 1u : 0u) << q;
            }
            if (!valid) hit = 0u;
            while (hit) {
                const int q = __ffs(hit) - 1;
                hit &= hit - 1u;
                const unsigned pj = cI[e0 + q];
                if (pj != pi && pj != 0xffffffffu) {
                    const int state = orbit_pair(A, pi, pj);
                    ncand += state > 0;
                    if (state == 2) {
                        const unsigned long long at = atomicAdd(&A.st->npairs, 1ull);
                        if (at < A.pair_cap) A.pairs[at] = make_uint2(pi, pj);
                    }
                }
            }
        }
    }
}

__global__ void __launch_bounds__(kOrbThreads) k_orbit_search(OrbitArgs A) {
    extern __shared__ unsigned ostack[];
    __shared__ unsigned pfx[kOrbWarps][32];
    __shared__ unsigned pbeg[kOrbWarps][32];
    __shared__ float4 cH[kOrbWarps][kOrbChunk], cL[kOrbWarps][kOrbChunk];
    __shared__ float cR[kOrbWarps][kOrbChunk];
    __shared__ unsigned cI[kOrbWarps][kOrbChunk];
    const unsigned w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned ng = A.st->ngroups;
    unsigned *stk = ostack + (size_t)w * A.stack_cap;
    const int cap = (int)A.stack_cap;
    for (;;) {
        unsigned g = 0;
        if (lane == 0) g = (unsigned)atomicAdd(&A.ctr[0], 1ull);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= ng) break;
        const uint4 ga = A.gr_a[g], gb = A.gr_b[g];
        const uint2 gr = A.gr_r[g];
        const long long gthr = A.gr_thr[g];
        unsigned long long ncand = 0;
        int fill = 0;
        if (lane == 0) stk[0] = gb.w;
        __syncwarp();
        int sp = 1;
        bool overflow = false;
        unsigned iters = 0;
        while (sp > 0) {
            if (++iters > kOrbMaxIters) {
                overflow = true;
                break;
            }
            const int k = sp < 32 ? sp : 32;
            sp -= k;
            const bool valid = (int)lane < k;
            const unsigned v = valid ? stk[sp + lane] : 0u;
            __syncwarp();
            unsigned nch = 0, first = 0, pcount = 0, pbegin = 0;
            if (valid) {
                const uint4 a = A.nd_a[v], b = A.nd_b[v];
                const unsigned qmn[3] = {a.x, a.y, a.z}, qmx[3] = {b.x, b.y, b.z};
                const unsigned gmn[3] = {ga.x, ga.y, ga.z}, gmx[3] = {gb.x, gb.y, gb.z};
                long long gap2 = 0;
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    // empty grid cells between the two boxes along d
                    int gg = (int)qmn[d] - (int)gmx[d] - 1;
                    gg = max(gg, (int)gmn[d] - (int)qmx[d] - 1);
                    gg = max(gg, 0);
                    gap2 += (long long)gg * gg;
                }
                if (gap2 < max(gthr, A.nd_thr[v])) {
                    if (meta_leaf(a.w)) {
                        const uint2 r = A.nd_r[v];
                        pbegin = r.x;
                        pcount = r.y;
                    } else {
                        nch = meta_nchild(a.w);
                        first = b.w;
                    }
                }
            }
            // stage the particles of the opened leaves, testing full chunks
            const unsigned pincl = warp_incl_scan(pcount);
            const unsigned ptot = __shfl_sync(0xffffffffu, pincl, 31);
            if (ptot) {
                pfx[w][lane] = pincl - pcount;
                pbeg[w][lane] = pbegin;
                __syncwarp();
                for (unsigned done = 0; done < ptot;) {
                    const unsigned take = min(ptot - done, (unsigned)(kOrbChunk - fill));
                    for (unsigned e = lane; e < take; e += 32) {
                        const unsigned q = done + e;
                        int lo = 0, hi = 31;
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (pfx[w][mid] <= q) lo = mid; else hi = mid - 1;
                        }
                        const unsigned pj = pbeg[w][lo] + (q - pfx[w][lo]);
                        cH[w][fill + e] = A.spH[pj];
                        cL[w][fill + e] = A.spL[pj];
                        cR[w][fill + e] = A.rnbf[pj];
                        cI[w][fill + e] = pj;
                    }
                    fill += (int)take;
                    done += take;
                    __syncwarp();
                    if (fill == kOrbChunk) {
                        orbit_chunk(A, gr, fill, cH[w], cL[w], cR[w], cI[w], ncand);
                        fill = 0;
                        __syncwarp();
                    }
                }
            }
            // children of opened internal nodes
            const unsigned cincl = warp_incl_scan(nch);
            const unsigned ctot = __shfl_sync(0xffffffffu, cincl, 31);
            if (sp + (int)ctot > cap) {
                overflow = true;
                break;
            }
            for (unsigned j = 0; j < nch; j++) stk[sp + (cincl - nch) + j] = first + j;
            sp += (int)ctot;
            __syncwarp();
        }
        if (fill > 0 && !overflow) orbit_chunk(A, gr, fill, cH[w], cL[w], cR[w], cI[w], ncand);
        __syncwarp();
        ncand = warp_sum(ncand);
        if (lane == 0) {
            if (overflow) atomicOr(&A.st->flags, kErrStack);
            atomicAdd(&A.ctr[1], ncand);
        }
        __syncwarp();
    }
}

int orbit_launch(const OrbitArgs &A, cudaStream_t st) {
    const size_t smem = (size_t)kOrbWarps * A.stack_cap * sizeof(unsigned);
    if (cudaFuncSetAttribute(k_orbit_search, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
    k_orbit_prep<<<sm_count() * 8, 256, 0, st>>>(A);
    int nk = 1;
    for (int l = kLevels - 1; l >= 0; l--, nk++) k_orbit_nodes<<<sm_count() * 4, 256, 0, st>>>(A, l);
    k_orbit_groups<<<sm_count() * 4, 256, 0, st>>>(A);
    int per_sm = (int)((200u * 1024u) / (smem + 24u * 1024u));
    per_sm = per_sm < 1 ? 1 : (per_sm > 12 ? 12 : per_sm);
    k_orbit_search<<<sm_count() * per_sm, kOrbThreads, smem, st>>>(A);
    return nk + 2;
}

}  // namespace pt
