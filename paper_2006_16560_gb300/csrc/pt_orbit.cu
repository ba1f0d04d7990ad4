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
__device__ __forceinline__ double pericentre(const double dx[3], const double dv[3], double mu) {
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx[0], dx[0]), __dmul_rn(dx[1], dx[1])), __dmul_rn(dx[2], dx[2]));
    const double v2 = __dadd_rn(__dadd_rn(__dmul_rn(dv[0], dv[0]), __dmul_rn(dv[1], dv[1])), __dmul_rn(dv[2], dv[2]));
    if (v2 == 0.0) return __dsqrt_rn(r2);
    const double cx = __dsub_rn(__dmul_rn(dx[1], dv[2]), __dmul_rn(dx[2], dv[1]));
    const double cy = __dsub_rn(__dmul_rn(dx[2], dv[0]), __dmul_rn(dx[0], dv[2]));
    const double cz = __dsub_rn(__dmul_rn(dx[0], dv[1]), __dmul_rn(dx[1], dv[0]));
    const double h2 = __dadd_rn(__dadd_rn(__dmul_rn(cx, cx), __dmul_rn(cy, cy)), __dmul_rn(cz, cz));
    if (mu == 0.0) return __dsqrt_rn(__ddiv_rn(h2, v2));
    const double r = __dsqrt_rn(r2);
    const double a = __dsub_rn(v2, __ddiv_rn(mu, r));
    const double b = __dadd_rn(__dadd_rn(__dmul_rn(dx[0], dv[0]), __dmul_rn(dx[1], dv[1])), __dmul_rn(dx[2], dv[2]));
    const double ex = __dsub_rn(__dmul_rn(a, dx[0]), __dmul_rn(b, dv[0]));
    const double ey = __dsub_rn(__dmul_rn(a, dx[1]), __dmul_rn(b, dv[1]));
    const double ez = __dsub_rn(__dmul_rn(a, dx[2]), __dmul_rn(b, dv[2]));
    const double e = __ddiv_rn(__dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez))), mu);
    return __ddiv_rn(__ddiv_rn(h2, mu), __dadd_rn(1.0, e));
}

// 0: not a candidate, 1: candidate dropped by stage 2, 2: neighbour.
__device__ __forceinline__ int orbit_pair(const OrbitArgs &A, unsigned pi, unsigned pj) {
    const double4 xi = A.sp64[pi], xj = A.sp64[pj];
    const double4 vi = A.sv[pi], vj = A.sv[pj];
    const double dx[3] = {__dsub_rn(xj.x, xi.x), __dsub_rn(xj.y, xi.y), __dsub_rn(xj.z, xi.z)};
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx[0], dx[0]), __dmul_rn(dx[1], dx[1])), __dmul_rn(dx[2], dx[2]));
    const double R = fmax(vi.w, vj.w);
    if (!(r2 < __dmul_rn(R, R))) return 0;
    if (A.mode == 2) return 2;
    const double dv[3] = {__dsub_rn(vj.x, vi.x), __dsub_rn(vj.y, vi.y), __dsub_rn(vj.z, vi.z)};
    const double rp = pericentre(dx, dv, __dmul_rn(A.G, __dadd_rn(xi.w, xj.w)));
    double Rs = R;
    if (A.mode == 0) {
        const double s = A.massdep ? fmax(A.ssc[pi], A.ssc[pj]) : 1.0;
        Rs = __dmul_rn(A.sets[A.sq[pi].w].r_out, s);
    }
    return rp < __dmul_rn(A.C_v, Rs) ? 2 : 1;
}

__global__ void __launch_bounds__(kOrbThreads) k_orbit_search(OrbitArgs A) {
    extern __shared__ unsigned ostack[];
    __shared__ unsigned pfx[kOrbWarps][32];
    __shared__ unsigned pbeg[kOrbWarps][32];
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
            // pairs (group member, particle of an opened leaf)
            const unsigned pincl = warp_incl_scan(pcount);
            const unsigned ptot = __shfl_sync(0xffffffffu, pincl, 31);
            if (ptot) {
                pfx[w][lane] = pincl - pcount;
                pbeg[w][lane] = pbegin;
                __syncwarp();
                const unsigned long long total = (unsigned long long)ptot * gr.y;
                for (unsigned long long e0 = 0; e0 < total; e0 += 32) {
                    const unsigned long long e = e0 + lane;
                    int state = 0;
                    unsigned pi = 0, pj = 0;
                    if (e < total) {
                        const unsigned il = (unsigned)(e / ptot), jl = (unsigned)(e % ptot);
                        int lo = 0, hi = 31;
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (pfx[w][mid] <= jl) lo = mid; else hi = mid - 1;
                        }
                        pi = gr.x + il;
                        pj = pbeg[w][lo] + (jl - pfx[w][lo]);
                        if (pi != pj) state = orbit_pair(A, pi, pj);
                    }
                    ncand += __popc(__ballot_sync(0xffffffffu, state > 0));
                    const unsigned kmask = __ballot_sync(0xffffffffu, state == 2);
                    if (kmask) {
                        unsigned long long base = 0;
                        if (lane == 0) base = atomicAdd(&A.st->npairs, (unsigned long long)__popc(kmask));
                        base = __shfl_sync(0xffffffffu, base, 0);
                        if (state == 2) {
                            const unsigned long long at = base + __popc(kmask & lanemask_lt());
                            if (at < A.pair_cap) A.pairs[at] = make_uint2(pi, pj);
                        }
                    }
                }
                __syncwarp();
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
    k_orbit_prep<<<152 * 8, 256, 0, st>>>(A);
    int nk = 1;
    for (int l = kLevels - 1; l >= 0; l--, nk++) k_orbit_nodes<<<152 * 4, 256, 0, st>>>(A, l);
    k_orbit_groups<<<152 * 4, 256, 0, st>>>(A);
    int per_sm = (int)((200u * 1024u) / (smem + 2048));
    per_sm = per_sm < 1 ? 1 : (per_sm > 12 ? 12 : per_sm);
    k_orbit_search<<<152 * per_sm, kOrbThreads, smem, st>>>(A);
    return nk + 2;
}

}  // namespace pt
