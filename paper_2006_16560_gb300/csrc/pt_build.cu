// pt_build.cu -- tree build kernels: root box, Morton keys, gather, octree
// topology, bottom-up multipoles and walk groups.
//
// Every kernel reads its element count from device memory and runs on a
// fixed grid (grid-stride loops), so the whole build is one data-independent
// launch sequence on the context stream.
#include "pt_kernels.cuh"

namespace pt {

constexpr int kT = 256;
constexpr unsigned kTopoBig = 16;     // nodes above this size get a warp in the topology count

// ---------------------------------------------------------------------------
// Sets (clusters) and the root box
// ---------------------------------------------------------------------------

// set_of[i] for every input particle (binary search over set begins).
__global__ void k_set_of(const SetInfo *sets, int nsets, unsigned n, unsigned *set_of) {
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int lo = 0, hi = nsets - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (sets[mid].begin <= i) lo = mid; else hi = mid - 1;
        }
        set_of[i] = (unsigned)lo;
    }
}

__global__ void k_box_init(unsigned long long *bmin, unsigned long long *bmax, int nsets) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * nsets; i += gridDim.x * blockDim.x) {
        bmin[i] = ~0ull;
        bmax[i] = 0ull;
    }
}

// Per-set minimum and maximum of each coordinate (exact: min / max do not
// depend on the order of reduction) plus input validation.
__global__ void __launch_bounds__(kT) k_box(const double *pos, const double *mass, unsigned n,
                                            const unsigned *set_of, unsigned long long *bmin,
                                            unsigned long long *bmax, Status *st) {
    unsigned bad = 0;
    if (!set_of) {
        // one set: per-thread extrema over the grid-stride loop, reduced over
        // the warp and the block, then one atomic per block and component
        __shared__ unsigned long long sb[kT / 32][6];
        unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
        for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
            const double x[3] = {pos[3ull * i], pos[3ull * i + 1], pos[3ull * i + 2]};
            const double m = mass[i];
            if (!isfinite(x[0]) || !isfinite(x[1]) || !isfinite(x[2]) || !isfinite(m)) bad |= kErrNonFinite;
            if (m < 0.0) bad |= kErrNegMass;
#pragma unroll
            for (int d = 0; d < 3; d++) {
                const unsigned long long o = dbl_to_ordered(x[d]);
                lo[d] = o < lo[d] ? o : lo[d];
                hi[d] = o > hi[d] ? o : hi[d];
            }
        }
#pragma unroll
        for (int d = 0; d < 3; d++) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long a = __shfl_xor_sync(0xffffffffu, lo[d], o);
                const unsigned long long b = __shfl_xor_sync(0xffffffffu, hi[d], o);
                lo[d] = a < lo[d] ? a : lo[d];
                hi[d] = b > hi[d] ? b : hi[d];
            }
        }
        const unsigned w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) {
#pragma unroll
            for (int d = 0; d < 3; d++) {
                sb[w][d] = lo[d];
                sb[w][3 + d] = hi[d];
            }
        }
        __syncthreads();
        if (threadIdx.x < 6 && blockIdx.x * blockDim.x < n) {
            const int c = threadIdx.x;
            unsigned long long v = sb[0][c];
            for (int k = 1; k < kT / 32; k++) {
                const unsigned long long u = sb[k][c];
                v = c < 3 ? (u < v ? u : v) : (u > v ? u : v);
            }
            if (c < 3) atomicMin(&bmin[c], v);
            else atomicMax(&bmax[c - 3], v);
        }
        bad = __reduce_or_sync(0xffffffffu, bad);
        if ((threadIdx.x & 31) == 0 && bad) atomicOr(&st->flags, bad);
        return;
    }
    for (unsigned base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        unsigned i = base + threadIdx.x;
        bool valid = i < n;
        unsigned s = valid ? (set_of ? set_of[i] : 0u) : 0xffffffffu;
        double x[3] = {0, 0, 0};
        if (valid) {
            x[0] = pos[3ull * i];
            x[1] = pos[3ull * i + 1];
            x[2] = pos[3ull * i + 2];
            double m = mass[i];
            if (!isfinite(x[0]) || !isfinite(x[1]) || !isfinite(x[2]) || !isfinite(m)) bad |= kErrNonFinite;
            if (m < 0.0) bad |= kErrNegMass;
        }
        unsigned s0 = __shfl_sync(0xffffffffu, s, 0);
        bool uniform = __all_sync(0xffffffffu, s == s0);
        for (int d = 0; d < 3; d++) {
            unsigned long long lo = valid ? dbl_to_ordered(x[d]) : ~0ull;
            unsigned long long hi = valid ? dbl_to_ordered(x[d]) : 0ull;
            if (uniform) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    unsigned long long a = __shfl_xor_sync(0xffffffffu, lo, o);
                    unsigned long long b = __shfl_xor_sync(0xffffffffu, hi, o);
                    lo = a < lo ? a : lo;
                    hi = b > hi ? b : hi;
                }
                if ((threadIdx.x & 31) == 0 && s0 != 0xffffffffu) {
                    atomicMin(&bmin[3 * s0 + d], lo);
                    atomicMax(&bmax[3 * s0 + d], hi);
                }
            } else if (valid) {
                atomicMin(&bmin[3 * s + d], lo);
                atomicMax(&bmax[3 * s + d], hi);
            }
        }
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && bad) atomicOr(&st->flags, bad);
}

// S = largest extent (1 if zero), scale = 2^21 / S (IEEE division), and the
// r_out gap threshold floor((r_out * scale)^2) + 2.
__global__ void k_box_finalize(SetInfo *sets, int nsets, const unsigned long long *bmin,
                               const unsigned long long *bmax) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsets) return;
    double S = 0.0;
    for (int d = 0; d < 3; d++) {
        double lo = ordered_to_dbl(bmin[3 * s + d]);
        double hi = ordered_to_dbl(bmax[3 * s + d]);
        sets[s].origin[d] = lo;
        double e = __dsub_rn(hi, lo);
        if (e > S) S = e;
    }
    if (S == 0.0) S = 1.0;
    sets[s].S = S;
    double scale = __ddiv_rn((double)kGrid, S);
    sets[s].scale = scale;
    double R = __dmul_rn(sets[s].r_out, scale);
    double R2 = __dmul_rn(R, R);
    sets[s].r2thr = (R2 > 4.0e18) ? 4000000000000000000ll : (long long)floor(R2) + 2;
}

// ---------------------------------------------------------------------------
// Keys
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long spread3(unsigned v) {
    // place bit b of v at bit 3b (21 bits)
    unsigned long long x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__global__ void __launch_bounds__(kT) k_keys(const double *pos, unsigned n, const unsigned *set_of,
                                             const SetInfo *sets, unsigned long long *keys,
                                             unsigned *vals, uint4 *qbuf) {
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        unsigned s = set_of ? set_of[i] : 0u;
        const SetInfo &S = sets[s];
        unsigned q[3];
        for (int d = 0; d < 3; d++) {
            // floor((x - origin) scale) clamped to the grid: the conversion
            // rounds down and saturates, the clamp is integer
            const long long u = __double2ll_rd(__dmul_rn(__dsub_rn(pos[3ull * i + d], S.origin[d]), S.scale));
            q[d] = (unsigned)min(max(u, 0ll), (long long)(kGrid - 1));
        }
        keys[i] = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
        vals[i] = i;
        qbuf[i] = make_uint4(q[0], q[1], q[2], s);
    }
}

// Sorted particle records: float64 (x, y, z, m), float-float split of the
// position for the mixed-precision path, and grid coordinates.
__global__ void __launch_bounds__(kT) k_gather(const double *pos, const double *mass, unsigned n,
                                               const unsigned *perm, const uint4 *qbuf,
                                               const double *scale, double *ssc,
                                               double4 *sp64, float4 *spH, float4 *spL, uint4 *sq,
                                               Status *st) {
    for (unsigned p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        unsigned i = perm[p];
        const double sc = scale ? scale[i] : 1.0;
        if (!(sc > 0.0 && isfinite(sc))) atomicOr(&st->flags, kErrBadScale);   // rare: no aggregation
        const float inv_sc = scale ? __double2float_rn(1.0 / sc) : 1.0f;
        ssc[p] = sc;
        double x = pos[3ull * i], y = pos[3ull * i + 1], z = pos[3ull * i + 2], m = mass[i];
        sp64[p] = make_double4(x, y, z, m);
        float xh = __double2float_rn(x), yh = __double2float_rn(y), zh = __double2float_rn(z);
        spH[p] = make_float4(xh, yh, zh, __double2float_rn(m));
        spL[p] = make_float4(__double2float_rn(x - (double)xh), __double2float_rn(y - (double)yh),
                             __double2float_rn(z - (double)zh), inv_sc);
        sq[p] = qbuf[i];
    }
}

// ---------------------------------------------------------------------------
// Mass-dependent radii (Sec. 6.1, Eq. 12): s_i = max(1, m_i/<m>)^(1/3), with
// <m> the set's mean mass (one block per set, fixed summation order).
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kT) k_set_mean_mass(const double *mass, const SetInfo *sets,
                                                      double *mean) {
    __shared__ double sh[kT];
    const SetInfo S = sets[blockIdx.x];
    double v = 0.0;
    for (unsigned k = threadIdx.x; k < S.n; k += blockDim.x) v += mass[S.begin + k];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = kT / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) mean[blockIdx.x] = sh[0] / (double)S.n;
}

__global__ void __launch_bounds__(kT) k_eq12_scale(const double *mass, unsigned n, const unsigned *set_of,
                                                   const double *mean, double *scale) {
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double q = mass[i] / mean[set_of ? set_of[i] : 0u];
        scale[i] = cbrt(q > 1.0 ? q : 1.0);
    }
}

// floor(((r_out s) scale)^2) + 2, the gap threshold of the walk (see pt.h).
__device__ __forceinline__ long long gap_threshold(const SetInfo &S, double s) {
    const double R = __dmul_rn(__dmul_rn(S.r_out, s), S.scale);
    const double R2 = __dmul_rn(R, R);
    return (R2 > 4.0e18) ? 4000000000000000000ll : (long long)floor(R2) + 2;
}

// ---------------------------------------------------------------------------
// Topology, level by level
// ---------------------------------------------------------------------------

__device__ __forceinline__ void level_range(const Status *st, int l, unsigned cap, unsigned &b,
                                            unsigned &c) {
    b = st->lvl_begin[l];
    c = st->lvl_count[l];
    if (b >= cap) { c = 0; return; }
    if (c > cap - b) c = cap - b;
}

__global__ void k_topo_roots(const SetInfo *sets, int nsets, uint4 *nd_a, uint4 *nd_b,
                             uint2 *nd_r, Status *st) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nsets) {
        nd_r[s] = make_uint2(sets[s].begin, sets[s].n);
        nd_a[s] = make_uint4(0, 0, 0, make_meta(0, 0, 0));
        nd_b[s] = make_uint4(0, 0, 0, 0);
    }
    if (s == 0) {
        st->lvl_begin[0] = 0;
        st->lvl_count[0] = (unsigned)nsets;
        for (int l = 1; l <= kLevels; l++) {
            st->lvl_begin[l] = 0;
            st->lvl_count[l] = 0;
        }
        for (int l = 0; l <= kLevels; l++) st->lvl_int[l] = 0;
        for (int b = 0; b < kLeafBuckets; b++) st->leaf_hist[b] = st->leaf_fill[b] = 0;
    }
}

// lcp[p] = number of leading key digits (levels) that sorted keys p - 1 and
// p share (21 when equal; lcp[0] is unused).  Inside a node of level l the
// children start exactly at the positions with lcp == l.
__global__ void __launch_bounds__(kT) k_lcp(const unsigned long long *skey, const unsigned *n_dev,
                                            unsigned char *lcp) {
    const unsigned n = *n_dev;
    for (unsigned p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        unsigned d = 0xffu;
        if (p > 0) {
            const unsigned long long x = skey[p - 1] ^ skey[p];
            d = x == 0ull ? (unsigned)kBits : (unsigned)(62 - (63 - __clzll((long long)x))) / 3u;
        }
        lcp[p] = (unsigned char)d;
    }
}

// Boundaries of the 8 key digits of level l+1 inside [b, b+c), c <= kTopoBig:
// B[k] is the first position whose digit is >= k, found by scanning lcp 16
// bytes at a time for the children's starts.  (Larger nodes take a warp whose
// lanes bisect the keys for the seven boundaries at once: measured faster
// than one thread per node for every node above 16 particles.)
__device__ __forceinline__ void child_bounds(const unsigned long long *skey, const unsigned char *lcp,
                                             unsigned b, unsigned c, int l, unsigned B[9]) {
    const int sh = 3 * (kBits - 1 - l);
    const unsigned e = b + c;
    B[0] = b;
    B[8] = e;
#pragma unroll
    for (unsigned k = 1; k < 8; k++) B[k] = e;
    // children start in increasing digit order: a start with digit dg is
    // the first position for every k <= dg not yet placed
    auto place = [&](unsigned pos) {
        const unsigned dg = (unsigned)(skey[pos] >> sh) & 7u;
#pragma unroll
        for (unsigned k = 1; k < 8; k++)
            if (k <= dg && B[k] == e) B[k] = pos;
    };
    place(b);
    const unsigned pat = (unsigned)l * 0x01010101u;
    for (unsigned q = (b + 1) & ~15u; q < e; q += 16) {
        const uint4 w = *reinterpret_cast<const uint4 *>(lcp + q);
        const unsigned words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int t = 0; t < 4; t++) {
            unsigned eq = __vcmpeq4(words[t], pat);          // 0xff in each equal byte
            while (eq) {
                const int bit = __ffs(eq) - 1;
                eq &= ~(0xffu << bit);
                const unsigned pos = q + 4u * t + (unsigned)(bit >> 3);
                if (pos > b && pos < e) place(pos);
            }
        }
    }
}

// Block sum and exclusive block scan (kT threads, every thread calls).
__device__ __forceinline__ unsigned block_sum(unsigned v, unsigned *sh) {
    v = __reduce_add_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned t = 0;
#pragma unroll
    for (int i = 0; i < kT / 32; i++) t += sh[i];
    __syncthreads();
    return t;
}

__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned *sh, unsigned &total) {
    const unsigned inc = warp_incl_scan(v);
    const unsigned w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 31) sh[w] = inc;
    __syncthreads();
    unsigned before = 0, t = 0;
#pragma unroll
    for (int i = 0; i < kT / 32; i++) {
        const unsigned x = sh[i];
        before += (unsigned)i < w ? x : 0u;
        t += x;
    }
    __syncthreads();
    total = t;
    return before + inc - v;
}

// The level's nodes in even contiguous chunks, one per block (the same
// partition in k_topo_count and k_topo_emit: both run on the same grid).
__device__ __forceinline__ void topo_chunk(unsigned cnt, unsigned &k0, unsigned &k1) {
    const unsigned C = (cnt + gridDim.x - 1) / gridDim.x;
    k0 = min(blockIdx.x * C, cnt);
    k1 = min(k0 + C, cnt);
}

// Number of children of every node of level l (0 for a leaf); writes meta,
// keeps the child boundaries of split nodes for k_topo_emit and the block's
// total of children in bsum.  Nodes of up to kTopoBig particles take a
// thread; larger ones a warp, whose lanes 1..7 bisect for the seven digit
// boundaries at once (a thread doing them one after another waits on ~140
// dependent loads at the top levels).
__global__ void __launch_bounds__(kT) k_topo_count(int l, const unsigned long long *skey,
                                                   const unsigned char *lcp, uint4 *nd_a,
                                                   const uint2 *nd_r, unsigned *nch, uint4 *bnd,
                                                   unsigned *bsum, int n_leaf, unsigned cap,
                                                   const Status *st) {
    __shared__ unsigned sh[kT / 32];
    unsigned b0, cnt, k0, k1;
    level_range(st, l, cap, b0, cnt);
    topo_chunk(cnt, k0, k1);
    const bool can_split = l < kMaxLevel;
    for (unsigned k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const unsigned v = b0 + k;
        const uint2 r = nd_r[v];
        const bool split = can_split && (int)r.y > n_leaf;
        if (split && r.y > kTopoBig) continue;            // a warp's, below
        unsigned nc = 0;
        if (split) {
            unsigned B[9];
            child_bounds(skey, lcp, r.x, r.y, l, B);
            for (int j = 0; j < 8; j++) nc += (B[j + 1] > B[j]) ? 1u : 0u;
            bnd[2 * v] = make_uint4(B[0], B[1], B[2], B[3]);
            bnd[2 * v + 1] = make_uint4(B[4], B[5], B[6], B[7]);
        }
        nch[k] = nc;
        uint4 a = nd_a[v];
        a.w = make_meta((unsigned)l, nc == 0 ? 1u : 0u, nc);
        nd_a[v] = a;
    }
    if (can_split) {
        const unsigned lane = threadIdx.x & 31;
        const int sh3 = 3 * (kBits - 1 - l);
        for (unsigned k = k0 + (threadIdx.x >> 5); k < k1; k += kT / 32) {
            const unsigned v = b0 + k;
            const uint2 r = nd_r[v];
            if (r.y <= kTopoBig || (int)r.y <= n_leaf) continue;   // uniform across the warp
            const unsigned e = r.x + r.y;
            unsigned pos = r.x;                              // lane 0: B[0]
            if (lane >= 1 && lane < 8) {                     // first p with digit >= lane
                unsigned lo = r.x, hi = e;
                while (lo < hi) {
                    const unsigned mid = lo + ((hi - lo) >> 1);
                    const unsigned dg = (unsigned)(skey[mid] >> sh3) & 7u;
                    if (dg >= lane) hi = mid; else lo = mid + 1;
                }
                pos = lo;
            }
            unsigned B[9];
#pragma unroll
            for (int j = 0; j < 8; j++) B[j] = __shfl_sync(0xffffffffu, pos, j);
            B[8] = e;
            if (lane == 0) {
                unsigned nc = 0;
                for (int j = 0; j < 8; j++) nc += (B[j + 1] > B[j]) ? 1u : 0u;
                bnd[2 * v] = make_uint4(B[0], B[1], B[2], B[3]);
                bnd[2 * v + 1] = make_uint4(B[4], B[5], B[6], B[7]);
                nch[k] = nc;
                uint4 a = nd_a[v];
                a.w = make_meta((unsigned)l, nc == 0 ? 1u : 0u, nc);
                nd_a[v] = a;
            }
        }
    }
    __syncthreads();                  // the block's nch entries are in place
    unsigned s = 0;
    for (unsigned k = k0 + threadIdx.x; k < k1; k += blockDim.x) s += nch[k];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) bsum[blockIdx.x] = s;
}

// Creates the children of level l's split nodes and lists the split nodes
// themselves, in any order, in nd_int from lvl_begin[l] on (the multipole
// pass then takes one internal node per thread with no leaves in between:
// float64 instructions cost the same for a warp with few lanes).  A block's
// children follow those of the blocks before it (the sum of their bsum) in
// the order of its chunk (a block scan), so level l+1 is in key order.
__global__ void __launch_bounds__(kT) k_topo_emit(int l, const uint4 *bnd,
                                                  uint4 *nd_a, uint4 *nd_b, uint2 *nd_r,
                                                  const unsigned *nch, const unsigned *bsum,
                                                  unsigned *nd_int, unsigned cap, Status *st) {
    __shared__ unsigned sh[kT / 32];
    unsigned b0, cnt, k0, k1;
    level_range(st, l, cap, b0, cnt);
    topo_chunk(cnt, k0, k1);
    const unsigned next = st->lvl_begin[l] + st->lvl_count[l];
    unsigned s = 0;
    for (unsigned i = threadIdx.x; i < blockIdx.x; i += blockDim.x) s += bsum[i];
    const unsigned base = block_sum(s, sh);
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        // only this thread touches level l+1's entries; the kernels that
        // read them are later launches
        const unsigned total = base + bsum[blockIdx.x];
        st->lvl_begin[l + 1] = next;
        unsigned c = total;
        if ((unsigned long long)next + total > cap) {
            atomicOr(&st->flags, kErrNodeCap);
            c = next < cap ? cap - next : 0u;
        }
        st->lvl_count[l + 1] = c;
    }
    const unsigned lane = threadIdx.x & 31;
    unsigned carry = 0;
    for (unsigned r0 = k0; r0 < k1; r0 += blockDim.x) {      // uniform across the block
        const unsigned k = r0 + threadIdx.x;
        const unsigned nc = k < k1 ? nch[k] : 0u;
        unsigned tot;
        const unsigned excl = block_excl_scan(nc, sh, tot);
        const unsigned m = __ballot_sync(0xffffffffu, nc != 0);
        unsigned slot = 0;
        if (m) {                      // list slots: one atomic per warp
            if (lane == 0) slot = atomicAdd(&st->lvl_int[l], (unsigned)__popc(m));
            slot = __shfl_sync(0xffffffffu, slot, 0) + __popc(m & lanemask_lt());
        }
        if (nc) {
            const unsigned v = b0 + k;
            if (b0 + slot < cap) nd_int[b0 + slot] = v;
            const uint2 r = nd_r[v];
            const uint4 b1 = bnd[2 * v], b2 = bnd[2 * v + 1];
            const unsigned B[9] = {b1.x, b1.y, b1.z, b1.w, b2.x, b2.y, b2.z, b2.w, r.x + r.y};
            const unsigned first = next + base + carry + excl;
            unsigned c = first;
            for (int j = 0; j < 8; j++) {
                if (B[j + 1] == B[j]) continue;
                if (c < cap) {
                    nd_r[c] = make_uint2(B[j], B[j + 1] - B[j]);
                    nd_a[c] = make_uint4(0, 0, 0, make_meta((unsigned)l + 1, 1, 0));
                    nd_b[c] = make_uint4(0, 0, 0, 0);
                }
                c++;
            }
            uint4 bb = nd_b[v];
            bb.w = first;
            nd_b[v] = bb;
        }
        carry += tot;
    }
}

__global__ void k_topo_finish(Status *st, unsigned cap) {
    unsigned total = 0, maxl = 0;
    for (int l = 0; l < kLevels; l++) {
        if (st->lvl_count[l]) maxl = (unsigned)l;
        total += st->lvl_count[l];
    }
    if (total > cap) {
        atomicOr(&st->flags, kErrNodeCap);
        total = cap;
    }
    st->nnodes = total;
    st->max_level = maxl;
}

// ---------------------------------------------------------------------------
// Multipoles, bottom-up one level at a time.  Leaves sum their particles
// about the first particle, internal nodes combine their children with the
// parallel-axis shift; T is the central second moment sum m d d^T and the
// stored quadrupole is Q = 3T - tr(T) I (twice the traceless A' of Eq. 31).
// ---------------------------------------------------------------------------

// max of two non-negative doubles on the integer pipe (their bit patterns
// order like their values); GB300's float64 pipe is the build's slow unit
__device__ __forceinline__ double dmax_pos(double a, double b) {
    return __longlong_as_double(max(__double_as_longlong(a), __double_as_longlong(b)));
}

// Writes node v's multipole records: COM and mass, Q = 3T - tr(T) I, T with
// the largest radius factor, the grid box, the walk's gap threshold (f1) and
// the float record of the mixed kernel.
__device__ __forceinline__ void store_moments(unsigned v, uint4 a, uint4 bb, unsigned p0, double M,
                                              const double com[3], const double T[6], double smax,
                                              const unsigned qmn[3], const unsigned qmx[3],
                                              const uint4 *sq, uint4 *nd_a, uint4 *nd_b, double4 *nd_c,
                                              double4 *nd_q, double4 *nd_t, float4 *nd_f,
                                              const SetInfo *sets, long long *nd_thr) {
    double tr = T[0] + T[1] + T[2];
    double Q[6] = {3 * T[0] - tr, 3 * T[1] - tr, 3 * T[2] - tr, 3 * T[3], 3 * T[4], 3 * T[5]};
    nd_c[v] = make_double4(com[0], com[1], com[2], M);
    nd_q[2 * v] = make_double4(Q[0], Q[1], Q[2], Q[3]);
    nd_q[2 * v + 1] = make_double4(Q[4], Q[5], 0.0, 0.0);
    nd_t[2 * v] = make_double4(T[0], T[1], T[2], T[3]);
    nd_t[2 * v + 1] = make_double4(T[4], T[5], smax, 0.0);
    if (nd_thr) nd_thr[v] = gap_threshold(sets[sq[p0].w], smax);
    a.x = qmn[0]; a.y = qmn[1]; a.z = qmn[2];
    bb.x = qmx[0]; bb.y = qmx[1]; bb.z = qmx[2];
    nd_a[v] = a;
    nd_b[v] = bb;
    // float record of the mixed kernel: float-float COM, M and -Q without its
    // zz element (Q is traceless: -Qzz = Qxx + Qyy)
    float hx = __double2float_rn(com[0]), hy = __double2float_rn(com[1]), hz = __double2float_rn(com[2]);
    nd_f[3 * v] = make_float4(hx, hy, hz, __double2float_rn(M));
    nd_f[3 * v + 1] = make_float4(__double2float_rn(com[0] - (double)hx),
                                  __double2float_rn(com[1] - (double)hy),
                                  __double2float_rn(com[2] - (double)hz), __double2float_rn(-Q[0]));
    nd_f[3 * v + 2] = make_float4(__double2float_rn(-Q[1]), __double2float_rn(-Q[3]),
                                  __double2float_rn(-Q[4]), __double2float_rn(-Q[5]));
}

// Moments of leaf v: its particles summed about the first particle (whose own
// offset is zero).
__device__ __forceinline__ void leaf_moments(unsigned v, const double4 *sp64, const uint4 *sq, uint4 *nd_a,
                                             uint4 *nd_b, const uint2 *nd_r, double4 *nd_c, double4 *nd_q,
                                             double4 *nd_t, float4 *nd_f, const double *ssc,
                                             const SetInfo *sets, long long *nd_thr) {
    const uint4 a = nd_a[v], bb = nd_b[v];
    const uint2 r = nd_r[v];
    double s1[3] = {0, 0, 0}, s2[6] = {0, 0, 0, 0, 0, 0}, T[6] = {0, 0, 0, 0, 0, 0}, com[3];
    const double4 p0 = sp64[r.x];
    const uint4 q0 = sq[r.x];
    const double x0[3] = {p0.x, p0.y, p0.z};
    double M = p0.w, smax = ssc[r.x];
    unsigned qmn[3] = {q0.x, q0.y, q0.z}, qmx[3] = {q0.x, q0.y, q0.z};
    for (unsigned p = r.x + 1; p < r.x + r.y; p++) {
        const double4 P = sp64[p];
        const uint4 q = sq[p];
        const double d0 = P.x - x0[0], d1 = P.y - x0[1], d2 = P.z - x0[2], m = P.w;
        // float64 is GB300's slow pipe: m d formed once, reused by both sums
        const double md0 = m * d0, md1 = m * d1, md2 = m * d2;
        M += m;
        s1[0] += md0; s1[1] += md1; s1[2] += md2;
        s2[0] = fma(md0, d0, s2[0]); s2[1] = fma(md1, d1, s2[1]); s2[2] = fma(md2, d2, s2[2]);
        s2[3] = fma(md0, d1, s2[3]); s2[4] = fma(md0, d2, s2[4]); s2[5] = fma(md1, d2, s2[5]);
        qmn[0] = min(qmn[0], q.x); qmn[1] = min(qmn[1], q.y); qmn[2] = min(qmn[2], q.z);
        qmx[0] = max(qmx[0], q.x); qmx[1] = max(qmx[1], q.y); qmx[2] = max(qmx[2], q.z);
        smax = dmax_pos(smax, ssc[p]);
    }
    if (M > 0.0) {
        // one reciprocal for the three offsets; T = S2 - s1 dc^T (s1 = M dc)
        const double iM = 1.0 / M;
        const double dc[3] = {s1[0] * iM, s1[1] * iM, s1[2] * iM};
        for (int d = 0; d < 3; d++) com[d] = x0[d] + dc[d];
        T[0] = fma(-s1[0], dc[0], s2[0]);
        T[1] = fma(-s1[1], dc[1], s2[1]);
        T[2] = fma(-s1[2], dc[2], s2[2]);
        T[3] = fma(-s1[0], dc[1], s2[3]);
        T[4] = fma(-s1[0], dc[2], s2[4]);
        T[5] = fma(-s1[1], dc[2], s2[5]);
    } else {
        for (int d = 0; d < 3; d++) com[d] = x0[d];
    }
    store_moments(v, a, bb, r.x, M, com, T, smax, qmn, qmx, sq, nd_a, nd_b, nd_c, nd_q, nd_t, nd_f, sets,
                  nd_thr);
}

// Moments of internal node v from its (complete) children: mass and COM about
// the first child's COM, then T = sum of the children's T shifted to the COM
// (parallel axes).  The child loops are unrolled over the at most eight
// children, so their loads are issued together.
__device__ __forceinline__ void internal_moments(unsigned v, const uint4 *sq, uint4 *nd_a, uint4 *nd_b,
                                                 const uint2 *nd_r, double4 *nd_c, double4 *nd_q,
                                                 double4 *nd_t, float4 *nd_f, const SetInfo *sets,
                                                 long long *nd_thr, unsigned cap) {
    const uint4 a = nd_a[v], bb = nd_b[v];
    const unsigned fc = bb.w, nc = meta_nchild(a.w);
    if (nc < 1 || nc > 8 || fc >= cap || nc > cap - fc) return;   // truncated build (flag is set)
    double4 C[8];
#pragma unroll
    for (int j = 0; j < 8; j++) C[j] = j < (int)nc ? nd_c[fc + j] : make_double4(0.0, 0.0, 0.0, 0.0);
    const double x0[3] = {C[0].x, C[0].y, C[0].z};
    double M = C[0].w, s1[3] = {0, 0, 0}, T[6] = {0, 0, 0, 0, 0, 0}, com[3], smax = 0.0;
    unsigned qmn[3] = {kGrid, kGrid, kGrid}, qmx[3] = {0, 0, 0};
#pragma unroll
    for (int j = 0; j < 8; j++) {
        if (j >= (int)nc) break;
        const unsigned c = fc + j;
        if (j > 0) {
            M += C[j].w;
            s1[0] += C[j].w * (C[j].x - x0[0]);
            s1[1] += C[j].w * (C[j].y - x0[1]);
            s1[2] += C[j].w * (C[j].z - x0[2]);
        }
        const uint4 ca = nd_a[c], cb = nd_b[c];
        smax = dmax_pos(smax, nd_t[2 * c + 1].z);
        qmn[0] = min(qmn[0], ca.x); qmn[1] = min(qmn[1], ca.y); qmn[2] = min(qmn[2], ca.z);
        qmx[0] = max(qmx[0], cb.x); qmx[1] = max(qmx[1], cb.y); qmx[2] = max(qmx[2], cb.z);
    }
    if (M > 0.0) {
        const double iM = 1.0 / M;
        for (int d = 0; d < 3; d++) com[d] = x0[d] + s1[d] * iM;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            if (j >= (int)nc) break;
            const unsigned c = fc + j;
            const double4 t0 = nd_t[2 * c], t1 = nd_t[2 * c + 1];
            const double e0 = C[j].x - com[0], e1 = C[j].y - com[1], e2 = C[j].z - com[2], m = C[j].w;
            const double me0 = m * e0, me1 = m * e1, me2 = m * e2;
            T[0] += fma(me0, e0, t0.x);
            T[1] += fma(me1, e1, t0.y);
            T[2] += fma(me2, e2, t0.z);
            T[3] += fma(me0, e1, t0.w);
            T[4] += fma(me0, e2, t1.x);
            T[5] += fma(me1, e2, t1.y);
        }
    } else {
        for (int d = 0; d < 3; d++) com[d] = x0[d];
    }
    store_moments(v, a, bb, nd_r[v].x, M, com, T, smax, qmn, qmx, sq, nd_a, nd_b, nd_c, nd_q, nd_t, nd_f,
                  sets, nd_thr);
}

// Leaves in order of their particle count, so that the threads of a warp in
// the leaf multipole pass loop over leaves of one size (in node order a warp
// runs as many float64 iterations as its largest leaf, ~3x the mean).  The
// order within a size class is the atomics' and does not matter: each leaf
// is still summed by one thread, particle by particle.
__device__ __forceinline__ unsigned leaf_bucket(unsigned count) {
    return count < (unsigned)kLeafBuckets - 1 ? count : (unsigned)kLeafBuckets - 1;
}

__global__ void __launch_bounds__(kT) k_leaf_hist(const uint4 *nd_a, const uint2 *nd_r, unsigned cap,
                                                  Status *st) {
    __shared__ unsigned h[kLeafBuckets];
    for (int b = threadIdx.x; b < kLeafBuckets; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const unsigned nn = min(st->nnodes, cap);
    for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < nn; v += gridDim.x * blockDim.x)
        if (meta_leaf(nd_a[v].w)) atomicAdd(&h[leaf_bucket(nd_r[v].y)], 1u);
    __syncthreads();
    for (int b = threadIdx.x; b < kLeafBuckets; b += blockDim.x)
        if (h[b]) atomicAdd(&st->leaf_hist[b], h[b]);
}

// list[off[b] ..] = the leaves of class b; each block round takes its
// classes' slots with one global atomic per class.
__global__ void __launch_bounds__(kT) k_leaf_scatter(const uint4 *nd_a, const uint2 *nd_r, unsigned cap,
                                                     unsigned *list, Status *st) {
    __shared__ unsigned off[kLeafBuckets], cnt[kLeafBuckets], base[kLeafBuckets];
    if (threadIdx.x == 0) {
        unsigned o = 0;
        for (int b = 0; b < kLeafBuckets; b++) {
            off[b] = o;
            o += st->leaf_hist[b];
        }
    }
    const unsigned nn = min(st->nnodes, cap);
    for (unsigned r0 = blockIdx.x * blockDim.x; r0 < nn; r0 += gridDim.x * blockDim.x) {
        for (int b = threadIdx.x; b < kLeafBuckets; b += blockDim.x) cnt[b] = 0;
        __syncthreads();
        const unsigned v = r0 + threadIdx.x;
        const bool leaf = v < nn && meta_leaf(nd_a[v].w);
        unsigned b = 0, local = 0;
        if (leaf) {
            b = leaf_bucket(nd_r[v].y);
            local = atomicAdd(&cnt[b], 1u);
        }
        __syncthreads();
        for (int c = threadIdx.x; c < kLeafBuckets; c += blockDim.x)
            if (cnt[c]) base[c] = atomicAdd(&st->leaf_fill[c], cnt[c]);
        __syncthreads();
        if (leaf) {
            const unsigned at = off[b] + base[b] + local;
            if (at < cap) list[at] = v;
        }
        __syncthreads();
    }
}

// Multipoles bottom-up: every leaf at once (k_moments_leaves), then the
// internal nodes one level at a time, deepest first (k_moments_level), so
// that each level finds its children complete.  (A single launch in which
// the last child to arrive computes its parent was measured slower: its
// climb is a 21-step chain of dependent loads.)
__global__ void __launch_bounds__(kT) k_moments_leaves(const double4 *sp64, const uint4 *sq, uint4 *nd_a,
                                                       uint4 *nd_b, const uint2 *nd_r, double4 *nd_c,
                                                       double4 *nd_q, double4 *nd_t, float4 *nd_f,
                                                       const double *ssc, const SetInfo *sets,
                                                       long long *nd_thr, const unsigned *list, unsigned cap,
                                                       const Status *st) {
    __shared__ unsigned nl;
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int b = 0; b < kLeafBuckets; b++) t += st->leaf_hist[b];
        nl = min(t, cap);
    }
    __syncthreads();
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < nl; k += gridDim.x * blockDim.x)
        leaf_moments(list[k], sp64, sq, nd_a, nd_b, nd_r, nd_c, nd_q, nd_t, nd_f, ssc, sets, nd_thr);
}

// The internal nodes of level l, from the list the topology pass wrote.
__global__ void __launch_bounds__(kT) k_moments_level(int l, const uint4 *sq, uint4 *nd_a, uint4 *nd_b,
                                                      const uint2 *nd_r, double4 *nd_c, double4 *nd_q,
                                                      double4 *nd_t, float4 *nd_f, const SetInfo *sets,
                                                      long long *nd_thr, const unsigned *nd_int, unsigned cap,
                                                      const Status *st) {
    unsigned b0, cnt;
    level_range(st, l, cap, b0, cnt);
    const unsigned ni = min(st->lvl_int[l], cnt);
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < ni; k += gridDim.x * blockDim.x)
        internal_moments(nd_int[b0 + k], sq, nd_a, nd_b, nd_r, nd_c, nd_q, nd_t, nd_f, sets, nd_thr, cap);
}

// ---------------------------------------------------------------------------
// Groups: mark the first particle of every group, compact, then describe.
// A node with at most n_group particles (or a leaf) is a group; a larger
// node's children are taken in key order, each larger child on its own (its
// thread marks its children; a leaf that large is a group).  The smaller
// children of a node with at most 8 n_group particles form runs of
// consecutive children, each cut into groups of exactly n_group particles
// (the last one of a run smaller), so most groups fill the force kernel's
// 64-target pass; those of a larger node are packed whole and greedily into
// groups of at most n_group (cutting there could join sparse children of a
// wide node into one group whose box reaches far).
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kT) k_group_mark(const uint4 *nd_a, const uint4 *nd_b,
                                                   const uint2 *nd_r, unsigned *gflag,
                                                   int n_group, const Status *st) {
    const unsigned nn = st->nnodes;
    const unsigned G = (unsigned)n_group;
    for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < nn; v += gridDim.x * blockDim.x) {
        uint4 a = nd_a[v];
        uint2 r = nd_r[v];
        bool leaf = meta_leaf(a.w);
        if (meta_level(a.w) == 0 && (r.y <= G || leaf)) gflag[r.x] = 1u;
        if (r.y <= G || leaf) continue;
        const unsigned fc = nd_b[v].w, nc = meta_nchild(a.w);
        if (fc >= nn || nc > nn - fc) continue;         // truncated build (capacity flag is set)
        // cut: the run is marked every G particles; else a pack of whole
        // children is marked at its start
        const bool cut = (unsigned long long)r.y <= 8ull * G;
        unsigned rb = 0, rc = 0;                        // the current run (or pack) of small children
        for (unsigned c = fc; c < fc + nc; c++) {
            uint2 cr = nd_r[c];
            if (cr.y > G) {
                for (unsigned o = 0; o < rc; o += cut ? G : rc) gflag[rb + o] = 1u;
                rc = 0;
                if (meta_leaf(nd_a[c].w)) gflag[cr.x] = 1u;
                continue;
            }
            if (!cut && rc && rc + cr.y > G) {
                gflag[rb] = 1u;
                rc = 0;
            }
            if (rc == 0) rb = cr.x;
            rc += cr.y;
        }
        for (unsigned o = 0; o < rc; o += cut ? G : rc) gflag[rb + o] = 1u;
    }
}

__global__ void __launch_bounds__(kT) k_group_emit(const unsigned *gflag, const unsigned *gidx,
                                                   unsigned n, unsigned *gbegin) {
    for (unsigned p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
        if (gflag[p]) gbegin[gidx[p]] = p;
}

// One warp per group: range, grid box, set, root node, reference point.
__global__ void __launch_bounds__(kT) k_group_info(const unsigned *gbegin, unsigned n,
                                                   const uint4 *sq, uint2 *gr_r, uint4 *gr_a,
                                                   uint4 *gr_b, const double *ssc, const SetInfo *sets,
                                                   long long *gr_thr, const Status *st) {
    const unsigned ng = st->ngroups;
    const unsigned lane = threadIdx.x & 31;
    for (unsigned g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < ng;
         g += (gridDim.x * blockDim.x) >> 5) {
        unsigned b = gbegin[g];
        unsigned e = (g + 1 < ng) ? gbegin[g + 1] : n;
        unsigned mn[3] = {kGrid, kGrid, kGrid}, mx[3] = {0, 0, 0};
        double smax = 0.0;
        for (unsigned p = b + lane; p < e; p += 32) {
            uint4 q = sq[p];
            smax = fmax(smax, ssc[p]);
            mn[0] = min(mn[0], q.x); mn[1] = min(mn[1], q.y); mn[2] = min(mn[2], q.z);
            mx[0] = max(mx[0], q.x); mx[1] = max(mx[1], q.y); mx[2] = max(mx[2], q.z);
        }
        for (int d = 0; d < 3; d++) {
            mn[d] = __reduce_min_sync(0xffffffffu, mn[d]);
            mx[d] = __reduce_max_sync(0xffffffffu, mx[d]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
        if (lane == 0) {
            unsigned set = sq[b].w;
            if (gr_thr) gr_thr[g] = gap_threshold(sets[set], smax);
            gr_r[g] = make_uint2(b, e - b);
            gr_a[g] = make_uint4(mn[0], mn[1], mn[2], set);
            gr_b[g] = make_uint4(mx[0], mx[1], mx[2], set /* root node of the set */);
        }
    }
}

// ---------------------------------------------------------------------------
// Host-side sequence
// ---------------------------------------------------------------------------

static inline int grid_for(unsigned long long n, int threads, int cap) {
    unsigned long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return (int)(b < (unsigned long long)cap ? b : cap);
}

int build_launch(const BuildArgs &A, cudaStream_t st) {
    const int gmax = sm_count() * 8;
    const unsigned n = A.n;
    Status *S = A.status;
    int nk = 0;
    if (A.nsets > 1) {
        k_set_of<<<grid_for(n, kT, gmax), kT, 0, st>>>(A.sets, A.nsets, n, A.set_of);
        nk++;
    }
    const unsigned *set_of = A.nsets > 1 ? A.set_of : nullptr;
    k_box_init<<<1, 256, 0, st>>>(A.bmin, A.bmax, A.nsets);
    k_box<<<grid_for(n, kT, gmax), kT, 0, st>>>(A.pos, A.mass, n, set_of, A.bmin, A.bmax, S);
    k_box_finalize<<<(A.nsets + 127) / 128, 128, 0, st>>>(A.sets, A.nsets, A.bmin, A.bmax);
    k_keys<<<grid_for(n, kT, gmax), kT, 0, st>>>(A.pos, n, set_of, A.sets, A.keys_in, A.vals_in, A.qbuf);
    nk += 4;
    const double *scale = A.scale;
    if (A.massdep && !scale) {           // Eq. 12 factors from the masses
        k_set_mean_mass<<<A.nsets, kT, 0, st>>>(A.mass, A.sets, A.set_mean);
        k_eq12_scale<<<grid_for(n, kT, gmax), kT, 0, st>>>(A.mass, n, set_of, A.set_mean, A.scale_buf);
        scale = A.scale_buf;
        nk += 2;
    }
    int set_bits = 0;
    if (A.nsets > 1) {
        while ((1 << set_bits) < A.nsets) set_bits++;
    }
    nk += radix_sort(A.keys_in, A.vals_in, A.skey, A.perm, A.n_dev, n, 0, 3 * kBits, set_of,
                     set_bits, A.sort_tmp, st);
    k_gather<<<grid_for(n, kT, gmax), kT, 0, st>>>(A.pos, A.mass, n, A.perm, A.qbuf, scale, A.ssc,
                                                   A.sp64, A.spH, A.spL, A.sq, S);
    // topology
    k_lcp<<<grid_for(n, kT, gmax), kT, 0, st>>>(A.skey, A.n_dev, A.lcp);
    nk++;
    k_topo_roots<<<(A.nsets + 127) / 128, 128, 0, st>>>(A.sets, A.nsets, A.nd_a, A.nd_b, A.nd_r, S);
    nk += 2;
    for (int l = 0; l <= kMaxLevel; l++) {
        k_topo_count<<<gmax, kT, 0, st>>>(l, A.skey, A.lcp, A.nd_a, A.nd_r, A.tmp_u32a, A.nd_bnd,
                                          A.topo_bsum, A.n_leaf, A.cap_nodes, S);
        nk++;
        if (l == kMaxLevel) break;
        k_topo_emit<<<gmax, kT, 0, st>>>(l, A.nd_bnd, A.nd_a, A.nd_b, A.nd_r, A.tmp_u32a, A.topo_bsum,
                                         A.nd_int, A.cap_nodes, S);
        nk++;
    }
    k_topo_finish<<<1, 1, 0, st>>>(S, A.cap_nodes);
    nk++;
    long long *thr = A.massdep ? A.nd_thr : nullptr;
    k_leaf_hist<<<gmax, kT, 0, st>>>(A.nd_a, A.nd_r, A.cap_nodes, S);
    k_leaf_scatter<<<gmax, kT, 0, st>>>(A.nd_a, A.nd_r, A.cap_nodes, A.tmp_u32a, S);
    nk += 2;
    k_moments_leaves<<<gmax, kT, 0, st>>>(A.sp64, A.sq, A.nd_a, A.nd_b, A.nd_r, A.nd_c, A.nd_q, A.nd_t,
                                          A.nd_f, A.ssc, A.sets, thr, A.tmp_u32a, A.cap_nodes, S);
    nk++;
    // two blocks per SM: the kernel's 120 registers allow no more resident
    // ones, and a level's internal nodes are few (the larger grid ran in
    // waves of idle blocks)
    const int mgrid = sm_count() * 2;
    for (int l = kMaxLevel - 1; l >= 0; l--, nk++)
        k_moments_level<<<mgrid, kT, 0, st>>>(l, A.sq, A.nd_a, A.nd_b, A.nd_r, A.nd_c, A.nd_q, A.nd_t,
                                             A.nd_f, A.sets, thr, A.nd_int, A.cap_nodes, S);
    // groups
    cudaMemsetAsync(A.gflag, 0, (size_t)n * sizeof(unsigned), st);
    k_group_mark<<<gmax, kT, 0, st>>>(A.nd_a, A.nd_b, A.nd_r, A.gflag, A.n_group, S);
    nk++;
    nk += scan_exclusive<unsigned>(A.gflag, A.tmp_u32b, A.n_dev, nullptr, &S->ngroups, A.scan_tmp, st);
    k_group_emit<<<grid_for(n, kT, gmax), kT, 0, st>>>(A.gflag, A.tmp_u32b, n, A.gbegin);
    k_group_info<<<gmax, kT, 0, st>>>(A.gbegin, n, A.sq, A.gr_r, A.gr_a, A.gr_b, A.ssc, A.sets,
                                      A.massdep ? A.gr_thr : nullptr, S);
    nk += 2;
    return nk;
}

}  // namespace pt
