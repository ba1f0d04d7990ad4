// pt_scan_sort.cu -- device-wide exclusive scan and stable LSD radix sort.
//
// Both use a fixed grid whose blocks each own one contiguous chunk of the
// input, and read the element count from device memory, so the launch
// sequence of a whole tree build is independent of the data.
//
// Radix sort: 8-bit digits, one (histogram, scan, scatter) triple per pass.
// The scatter ranks equal digits with warp primitives: __match_any_sync
// groups the lanes holding the same digit and the popcount of the lower
// peers gives each lane's stable rank; per-warp digit counts in shared
// memory order the warps of a tile and a running per-digit offset orders
// the tiles of a block, so equal keys keep their input order.
#include "pt_internal.cuh"

namespace pt {

// ------------------------------- scan --------------------------------------

__device__ __forceinline__ void chunk_of(unsigned n, unsigned b, unsigned nb,
                                         unsigned &lo, unsigned &hi) {
    unsigned long long chunk = ((unsigned long long)n + nb - 1) / nb;
    unsigned long long l = chunk * b, h = l + chunk;
    if (l > n) l = n;
    if (h > n) h = n;
    lo = (unsigned)l;
    hi = (unsigned)h;
}

// Block-wide inclusive scan of one value per thread (u64).
__device__ unsigned long long block_incl_scan(unsigned long long v, unsigned long long *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_incl_scan(v);
    if (lane == 31) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        unsigned long long t = (lane < nw) ? sh[lane] : 0ull;
        t = warp_incl_scan(t);
        if (lane < nw) sh[lane] = t;
    }
    __syncthreads();
    if (w > 0) v += sh[w - 1];
    __syncthreads();
    return v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const unsigned *in, const unsigned *n_dev,
                                                              unsigned long long *bsum) {
    __shared__ unsigned long long sh[32];
    unsigned lo, hi;
    chunk_of(*n_dev, blockIdx.x, gridDim.x, lo, hi);
    unsigned long long s = 0;
    for (unsigned i = lo + threadIdx.x; i < hi; i += blockDim.x) s += in[i];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[w];
        bsum[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) k_scan_blocks(unsigned long long *bsum, int nb,
                                                      unsigned long long *total,
                                                      unsigned *total32) {
    __shared__ unsigned long long sh[32];
    unsigned long long v = (threadIdx.x < (unsigned)nb) ? bsum[threadIdx.x] : 0ull;
    unsigned long long inc = block_incl_scan(v, sh);
    if (threadIdx.x < (unsigned)nb) bsum[threadIdx.x] = inc - v;
    if (threadIdx.x == blockDim.x - 1) {
        bsum[nb] = inc;
        if (total) *total = inc;
        if (total32) *total32 = (unsigned)inc;
    }
}

template <typename OutT>
__global__ void __launch_bounds__(kScanThreads) k_scan_final(const unsigned *in, OutT *out,
                                                             const unsigned *n_dev,
                                                             const unsigned long long *bsum) {
    __shared__ unsigned long long sh[32];
    __shared__ unsigned long long carry_sh;
    unsigned lo, hi;
    chunk_of(*n_dev, blockIdx.x, gridDim.x, lo, hi);
    unsigned long long carry = bsum[blockIdx.x];
    for (unsigned base = lo; base < hi; base += blockDim.x) {
        unsigned i = base + threadIdx.x;
        unsigned long long v = (i < hi) ? in[i] : 0ull;
        unsigned long long inc = block_incl_scan(v, sh);
        if (i < hi) out[i] = (OutT)(carry + inc - v);
        if (threadIdx.x == blockDim.x - 1) carry_sh = inc;
        __syncthreads();
        carry += carry_sh;
        __syncthreads();
    }
}

template <typename OutT>
int scan_exclusive(const unsigned *in, OutT *out, const unsigned *n_dev,
                   unsigned long long *total_dev, unsigned *total_u32_dev, ScanTmp tmp,
                   cudaStream_t st) {
    k_scan_reduce<<<kScanBlocks, kScanThreads, 0, st>>>(in, n_dev, tmp.block_sums);
    k_scan_blocks<<<1, 1024, 0, st>>>(tmp.block_sums, kScanBlocks, total_dev, total_u32_dev);
    k_scan_final<OutT><<<kScanBlocks, kScanThreads, 0, st>>>(in, out, n_dev, tmp.block_sums);
    return 3;
}

template int scan_exclusive<unsigned>(const unsigned *, unsigned *, const unsigned *,
                                      unsigned long long *, unsigned *, ScanTmp, cudaStream_t);
template int scan_exclusive<unsigned long long>(const unsigned *, unsigned long long *,
                                                 const unsigned *, unsigned long long *,
                                                unsigned *, ScanTmp, cudaStream_t);

// ------------------------------- radix sort --------------------------------

constexpr int kSortThreads = 256;               // 8 warps; one thread per digit
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortRounds = 4;                  // 32-item rounds per warp per tile
constexpr int kSortTile = kSortThreads * kSortRounds;   // 1024 items
constexpr int kSortScanThreads = 320;                   // >= kSortBlocks, multiple of 32

template <bool SET_PASS>
__device__ __forceinline__ unsigned digit_of(unsigned long long k, unsigned v, int shift,
                                             const unsigned *set_of) {
    if (SET_PASS) return (set_of[v] >> shift) & 255u;
    return (unsigned)(k >> shift) & 255u;
}

template <bool SET_PASS>
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const unsigned long long *keys,
                                                            const unsigned *vals,
                                                            const unsigned *n_dev, int shift,
                                                            const unsigned *set_of,
                                                            unsigned *counts) {
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    unsigned lo, hi;
    chunk_of(*n_dev, blockIdx.x, gridDim.x, lo, hi);
    constexpr int U = 4;                 // loads in flight per thread
    for (unsigned i = lo + threadIdx.x; i < hi; i += U * blockDim.x) {
        unsigned d[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const unsigned j = i + u * blockDim.x;
            d[u] = j < hi ? digit_of<SET_PASS>(SET_PASS ? 0ull : keys[j], SET_PASS ? vals[j] : 0u, shift, set_of)
                          : 0xffffffffu;
        }
#pragma unroll
        for (int u = 0; u < U; u++)
            if (d[u] != 0xffffffffu) atomicAdd(&h[d[u]], 1u);
    }
    __syncthreads();
    counts[threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// One block per digit: exclusive scan of that digit's per-block counts (in
// place) and the digit's total in counts[256 * nb + digit].
__global__ void __launch_bounds__(kSortScanThreads) k_sort_scan(unsigned *counts, int nb) {
    __shared__ unsigned long long sh[32];
    const int d = blockIdx.x;
    const unsigned v = (threadIdx.x < (unsigned)nb) ? counts[d * nb + threadIdx.x] : 0u;
    const unsigned long long inc = block_incl_scan(v, sh);
    if (threadIdx.x < (unsigned)nb) counts[d * nb + threadIdx.x] = (unsigned)(inc - v);
    if (threadIdx.x == blockDim.x - 1) counts[256 * nb + d] = (unsigned)inc;
}

template <bool SET_PASS>
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(
    const unsigned long long *keys, const unsigned *vals, unsigned long long *keys_o,
    unsigned *vals_o, const unsigned *n_dev, int shift, const unsigned *set_of,
    const unsigned *offsets) {
    __shared__ unsigned hist[kSortWarps][256];
    __shared__ unsigned off[kSortWarps][256];
    __shared__ unsigned run[256];
    __shared__ unsigned long long scan_sh[32];
    const unsigned w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned lo, hi;
    chunk_of(*n_dev, blockIdx.x, gridDim.x, lo, hi);
    {   // start of this digit's bucket = sum of the smaller digits' totals
        const unsigned tot = offsets[256 * gridDim.x + threadIdx.x];
        const unsigned long long base = block_incl_scan(tot, scan_sh) - tot;
        run[threadIdx.x] = (unsigned)base + offsets[threadIdx.x * gridDim.x + blockIdx.x];
    }
    for (unsigned base = lo; base < hi; base += kSortTile) {
        for (int k = 0; k < kSortWarps; k++) hist[k][threadIdx.x] = 0;
        __syncthreads();
        unsigned long long kr[kSortRounds];
        unsigned vr[kSortRounds], dr[kSortRounds];
#pragma unroll
        for (int r = 0; r < kSortRounds; r++) {
            unsigned i = base + w * (32 * kSortRounds) + r * 32 + lane;
            if (i < hi) {
                kr[r] = keys[i];
                vr[r] = vals[i];
                dr[r] = digit_of<SET_PASS>(kr[r], vr[r], shift, set_of);
                atomicAdd(&hist[w][dr[r]], 1u);
            } else {
                dr[r] = 0xffffu;          // sentinel: never written
            }
        }
        __syncthreads();
        {   // per digit: offsets of each warp within this tile
            unsigned d = threadIdx.x, acc = run[d];
            for (int k = 0; k < kSortWarps; k++) {
                unsigned c = hist[k][d];
                off[k][d] = acc;
                acc += c;
            }
            run[d] = acc;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kSortRounds; r++) {
            unsigned d = dr[r];
            unsigned peers = __match_any_sync(0xffffffffu, d);
            if (d != 0xffffu) {
                unsigned rank = __popc(peers & lanemask_lt());
                unsigned pos = off[w][d] + rank;
                keys_o[pos] = kr[r];
                vals_o[pos] = vr[r];
            }
            __syncwarp();
            if (d != 0xffffu && (peers & lanemask_lt()) == 0u) off[w][d] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
    }
}

int radix_sort(const unsigned long long *keys_in, const unsigned *vals_in,
               unsigned long long *keys_out, unsigned *vals_out, const unsigned *n_dev,
               unsigned n_max, int bit0, int bit1, const unsigned *set_of, int set_bits,
               SortTmp tmp, cudaStream_t st) {
    (void)n_max;
    int npass = (bit1 - bit0 + 7) / 8 + (set_of ? (set_bits + 7) / 8 : 0);
    // choose the first destination so that the last pass lands in *_out
    bool to_out = (npass % 2) == 1;
    const unsigned long long *ks = keys_in;
    const unsigned *vs = vals_in;
    int pass = 0;
    auto run_pass = [&](int shift, bool set_pass) {
        unsigned long long *kd = to_out ? keys_out : tmp.k2;
        unsigned *vd = to_out ? vals_out : tmp.v2;
        if (set_pass) {
            k_sort_hist<true><<<kSortBlocks, kSortThreads, 0, st>>>(ks, vs, n_dev, shift, set_of, tmp.counts);
            k_sort_scan<<<256, kSortScanThreads, 0, st>>>(tmp.counts, kSortBlocks);
            k_sort_scatter<true><<<kSortBlocks, kSortThreads, 0, st>>>(ks, vs, kd, vd, n_dev, shift, set_of, tmp.counts);
        } else {
            k_sort_hist<false><<<kSortBlocks, kSortThreads, 0, st>>>(ks, vs, n_dev, shift, nullptr, tmp.counts);
            k_sort_scan<<<256, kSortScanThreads, 0, st>>>(tmp.counts, kSortBlocks);
            k_sort_scatter<false><<<kSortBlocks, kSortThreads, 0, st>>>(ks, vs, kd, vd, n_dev, shift, nullptr, tmp.counts);
        }
        ks = kd;
        vs = vd;
        to_out = !to_out;
        pass++;
    };
    for (int b = bit0; b < bit1; b += 8) run_pass(b, false);
    if (set_of)
        for (int b = 0; b < set_bits; b += 8) run_pass(b, true);
    if (npass == 0) {
        cudaMemcpyAsync(keys_out, keys_in, (size_t)n_max * 8, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(vals_out, vals_in, (size_t)n_max * 4, cudaMemcpyDeviceToDevice, st);
    }
    return 3 * pass;
}

}  // namespace pt
