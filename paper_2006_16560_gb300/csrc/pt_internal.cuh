// pt_internal.cuh -- device data layout and launch helpers shared by the
// kernels of libpt.so.  Nothing here is part of the public ABI (include/pt.h).
//
// HBM layout (all arrays in sorted key order unless noted; structure of
// arrays so that every kernel streams 16-byte aligned records):
//   particles  sp64  double4 (x, y, z, m)            32 B
//              spH   float4  (hi(x), hi(y), hi(z), m) 16 B   x = hi + lo
//              spL   float4  (lo(x), lo(y), lo(z), 0) 16 B   (float-float)
//              sq    uint4   (q_x, q_y, q_z, set id)  16 B
//              skey  u64, perm u32 (sorted slot -> original index)
//   nodes      nd_a  uint4 (qmin xyz, meta = level | leaf<<5 | nchild<<6)
//              nd_b  uint4 (qmax xyz, first child)
//              nd_r  uint2 (begin, count)
//              nd_c  double4 (com xyz, M);  nd_q double4 x 2 (Q xx yy zz xy, xz yz T-trace 0)
//              nd_f  float4 x 3 (hi(com) M | lo(com) -Qxx | -Qyy -Qxy -Qxz -Qyz), 48 B
//   groups     gr_r  uint2 (begin, count); gr_a uint4 (qmin, set); gr_b uint4 (qmax, root)
//              gr_nc, gr_np u32 list lengths; gr_co, gr_po u64 list offsets;
//              gr_nf u32, gr_fo u64: far PP segment (leaves opened for the
//              opening angle only, every pair at least r_out apart)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pt {

constexpr int kBits = 21;            // grid bits per dimension
constexpr int kMaxLevel = 21;        // deepest node level
constexpr int kLevels = 22;          // levels 0..21
constexpr unsigned kGrid = 1u << kBits;
constexpr int kLeafBuckets = 64;     // leaf size classes of the multipole pass (the last: >= 63)

// status flags (Status::flags)
enum : unsigned {
    kErrNodeCap = 1u << 0,    // node arrays too small
    kErrStack = 1u << 1,      // walk stack overflow
    kErrListCap = 1u << 2,    // interaction list arrays too small
    kErrPairCap = 1u << 3,    // neighbour pair buffer too small
    kErrNonFinite = 1u << 4,  // NaN / Inf position or mass
    kErrNegMass = 1u << 5,    // negative mass
    kErrGroupCap = 1u << 6,   // group arrays too small
    kErrBadScale = 1u << 7,   // radius factor not finite and positive
};

// Per-set (cluster) table entry.
struct SetInfo {
    double origin[3];
    double S, scale;          // box side and 2^21 / S
    double r_in, r_out;
    long long r2thr;          // floor((r_out * scale)^2) + 2
    unsigned begin, n;        // range in input order == range in sorted order
    unsigned pad[2];
};

// Device status block, copied to pinned host memory at the end of a call.
struct Status {
    unsigned flags;
    unsigned nnodes;
    unsigned ngroups;
    unsigned max_level;
    unsigned max_stack;              // deepest walk stack seen (entries per warp)
    unsigned pad0;
    unsigned long long cell_total, pp_total;
    unsigned long long cell_inter, pp_inter;
    unsigned long long npairs;
    unsigned long long pp_full, pp_fast;   // mixed PP pairs on the changeover / Newtonian path
    unsigned long long work[4];      // work counters for persistent kernels
    double energy, mom[3];
    unsigned lvl_begin[kLevels + 1];
    unsigned lvl_count[kLevels + 1];
    unsigned lvl_int[kLevels + 1];   // internal nodes per level (build only)
    unsigned leaf_hist[kLeafBuckets];   // leaves by particle count (build only)
    unsigned leaf_fill[kLeafBuckets];
};

// Walk thresholds shared by every group.
struct WalkParams {
    long long ithr[kLevels];   // accept (theta) iff d2 >= ithr[level]
};

__host__ __device__ inline unsigned meta_level(unsigned m) { return m & 31u; }
__host__ __device__ inline unsigned meta_leaf(unsigned m) { return (m >> 5) & 1u; }
__host__ __device__ inline unsigned meta_nchild(unsigned m) { return (m >> 6) & 15u; }
__host__ __device__ inline unsigned make_meta(unsigned level, unsigned leaf, unsigned nchild) {
    return level | (leaf << 5) | (nchild << 6);
}

// Order-preserving map of a double to an unsigned 64-bit integer (for
// atomic min / max of doubles; min and max are order independent, so the
// result is exact and deterministic).
__device__ __forceinline__ unsigned long long dbl_to_ordered(double v) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double ordered_to_dbl(unsigned long long b) {
    b = (b & 0x8000000000000000ull) ? (b & 0x7fffffffffffffffull) : ~b;
    return __longlong_as_double((long long)b);
}
__host__ inline unsigned long long host_ordered(double v) {
    unsigned long long b;
    static_assert(sizeof(double) == 8, "");
    __builtin_memcpy(&b, &v, 8);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() {
    return (1u << (threadIdx.x & 31u)) - 1u;
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if ((int)lane_id() >= o) v += u;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Streaming multiprocessors of the calling thread's current device
// (cudaDevAttrMultiProcessorCount), queried once per device and cached; every
// persistent or grid-stride launch is sized from it (152 on a GB300).
int sm_count();

// ---------------------------------------------------------------------------
// Device-wide exclusive scan over a device-resident element count, with a
// fixed grid (so the launch sequence never depends on data and can be
// captured in a CUDA graph).  Three launches: per-block sums, scan of the
// block sums, per-block scan with carry.
// ---------------------------------------------------------------------------
constexpr int kScanBlocks = 304;     // fixed partition of the scans (two per SM on a GB300)
constexpr int kScanThreads = 512;

struct ScanTmp {
    unsigned long long *block_sums;  // kScanBlocks + 1
};

// in: n_dev[0] elements of u32; out: exclusive prefix (u32 or u64);
// total_dev (optional) receives the sum.
template <typename OutT>
int scan_exclusive(const unsigned *in, OutT *out, const unsigned *n_dev,
                    unsigned long long *total_dev, unsigned *total_u32_dev,
                    ScanTmp tmp, cudaStream_t st);

// Radix sort of (u64 key, u32 value) pairs on bits [bit0, bit1) of the key,
// stable; n from n_dev (<= n_max).  Optionally a final stable pass ordering by
// set id (set_of[value]).  Result in keys_out / vals_out.  Both return the
// number of kernels they launched.
struct SortTmp {
    unsigned long long *k2;  // n_max
    unsigned *v2;            // n_max
    unsigned *counts;        // kSortCountsLen
};
constexpr int kSortBlocks = 304;
constexpr int kSortCountsLen = 256 * kSortBlocks + 256;   // per-block digit counts + digit totals
int radix_sort(const unsigned long long *keys_in, const unsigned *vals_in,
                unsigned long long *keys_out, unsigned *vals_out,
                const unsigned *n_dev, unsigned n_max, int bit0, int bit1,
                const unsigned *set_of, int set_bits, SortTmp tmp, cudaStream_t st);

}  // namespace pt
