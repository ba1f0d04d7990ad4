// pt_noalloc.cu -- pt_sort_keys_noalloc: the library's stable radix sort of
// 64-bit keys for callers that cannot allocate device memory.
//
// Who needs it: code that must not call cudaMalloc -- a process whose device
// memory is owned entirely by another allocator (a framework's caching
// allocator or a fixed arena), or a real-time loop that may not allocate.
// The regular entry points size their workspace with cudaMalloc on first
// use; this one uses a fixed scratch array that lives in the library image.
//
// The scratch is a file-scope __device__ array of kNoallocBytes (about
// 4.3 MiB).  Every GPU on which the library is loaded holds it until the
// process exits.  In host code the array's name is only a host-side
// stand-in, so its device address is looked up with cudaGetSymbolAddress
// once per device (on that device's first call, with that device current)
// and cached for the life of the process; a cudaDeviceReset of the device
// invalidates it, so the entry point must not be called on that device
// afterwards.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/pt.h"
#include "pt_internal.cuh"

namespace {

constexpr long long kNoallocMaxN = 1ll << 18;                 // 262,144 keys
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kOffVals = 0;                                               // u32 x max n
constexpr size_t kOffKeys2 = align_up(kOffVals + 4 * (size_t)kNoallocMaxN);  // u64 x max n
constexpr size_t kOffVals2 = align_up(kOffKeys2 + 8 * (size_t)kNoallocMaxN); // u32 x max n
constexpr size_t kOffCounts = align_up(kOffVals2 + 4 * (size_t)kNoallocMaxN);
constexpr size_t kOffN = align_up(kOffCounts + 4 * (size_t)pt::kSortCountsLen);
constexpr size_t kNoallocBytes = align_up(kOffN + 16);

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {};

__global__ void k_noalloc_init(unsigned *vals, unsigned *n_dev, unsigned n) {
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        vals[i] = i;
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_dev = n;
}

bool on_device(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" int pt_sort_keys_noalloc(int64_t n, const uint64_t *keys, uint64_t *keys_sorted,
                                    uint32_t *perm, void *stream) {
    if (n < 1 || n > kNoallocMaxN) return PT_ERR_ARG;
    if (!keys || !keys_sorted || !perm) return PT_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        (void)cudaGetLastError();
        return PT_ERR_CUDA;
    }
    if (!on_device(keys, dev) || !on_device(keys_sorted, dev) || !on_device(perm, dev))
        return PT_ERR_ARG;
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                (void)cudaGetLastError();
                return PT_ERR_CUDA;
            }
            g_scratch_addr[dev] = static_cast<unsigned char *>(p);
        }
        base = g_scratch_addr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned *vals = reinterpret_cast<unsigned *>(base + kOffVals);
    unsigned *n_dev = reinterpret_cast<unsigned *>(base + kOffN);
    pt::SortTmp tmp{reinterpret_cast<unsigned long long *>(base + kOffKeys2),
                    reinterpret_cast<unsigned *>(base + kOffVals2),
                    reinterpret_cast<unsigned *>(base + kOffCounts)};
    // everything the sort reads from the scratch is rewritten here: the
    // identity values, the count; histograms are rewritten by every pass
    k_noalloc_init<<<256, 256, 0, st>>>(vals, n_dev, (unsigned)n);
    pt::radix_sort(reinterpret_cast<const unsigned long long *>(keys), vals,
                   reinterpret_cast<unsigned long long *>(keys_sorted), perm, n_dev, (unsigned)n,
                   0, 64, nullptr, 0, tmp, st);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}
