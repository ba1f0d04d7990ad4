// pt_batch.cu -- gather / scatter kernels of pt_batch_longrange_force.
//
// A batch is a forest: the sets are concatenated, every tree kernel runs once
// over all of them (each set is one root), and these kernels move each set's
// inputs and outputs between the caller's per-set buffers and the
// concatenated arrays through a device-resident pointer table.
#include "pt_kernels.cuh"

namespace pt {

__device__ __forceinline__ int set_of_index(const SetInfo *sets, int nsets, unsigned i) {
    int lo = 0, hi = nsets - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sets[mid].begin <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_batch_gather(const BatchTab *tab, const SetInfo *sets, int nsets, unsigned n,
                               double *pos, double *mass, double *scale) {
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = set_of_index(sets, nsets, i);
        const unsigned k = i - sets[c].begin;
        const double *p = tab[c].pos;
        pos[3ull * i] = p[3ull * k];
        pos[3ull * i + 1] = p[3ull * k + 1];
        pos[3ull * i + 2] = p[3ull * k + 2];
        mass[i] = tab[c].mass[k];
        if (scale) scale[i] = tab[c].scale ? tab[c].scale[k] : 1.0;
    }
}

__global__ void k_batch_scatter(const BatchTab *tab, const SetInfo *sets, int nsets, unsigned n,
                                const double *acc, const double *pot) {
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = set_of_index(sets, nsets, i);
        const unsigned k = i - sets[c].begin;
        double *a = tab[c].acc;
        a[3ull * k] = acc[3ull * i];
        a[3ull * k + 1] = acc[3ull * i + 1];
        a[3ull * k + 2] = acc[3ull * i + 2];
        tab[c].pot[k] = pot[i];
    }
}

// Per-set neighbour totals from the global CSR (rows in concatenated order).
__global__ void k_batch_nb_totals(const SetInfo *sets, int nsets, const long long *off,
                                  long long *totals) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nsets; c += gridDim.x * blockDim.x)
        totals[c] = off[sets[c].begin + sets[c].n] - off[sets[c].begin];
}

// Split the global CSR into each set's CSR with set-local indices; sets whose
// capacity is too small (or that asked for no lists) are left untouched.
__global__ void k_batch_nb_split(const BatchTab *tab, const SetInfo *sets, int nsets, unsigned n,
                                 const long long *off, const int *idx, const long long *totals) {
    const unsigned long long ne = (unsigned long long)off[n];
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = set_of_index(sets, nsets, i);
        if (!tab[c].nb_off || (unsigned long long)totals[c] > tab[c].nb_cap) continue;
        const unsigned b = sets[c].begin, k = i - b;
        tab[c].nb_off[k] = off[i] - off[b];
        if (k + 1 == sets[c].n) tab[c].nb_off[k + 1] = off[i + 1] - off[b];
    }
    for (unsigned long long e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
        unsigned lo = 0, hi = n - 1;                  // row of entry e: last row with off <= e
        while (lo < hi) {
            const unsigned mid = (lo + hi + 1) >> 1;
            if ((unsigned long long)off[mid] <= e) lo = mid; else hi = mid - 1;
        }
        const int c = set_of_index(sets, nsets, lo);
        if (!tab[c].nb_off || (unsigned long long)totals[c] > tab[c].nb_cap) continue;
        const unsigned b = sets[c].begin;
        tab[c].nb_idx[e - (unsigned long long)off[b]] = idx[e] - (int)b;
    }
}

int batch_gather_launch(const BatchTab *tab, const SetInfo *sets, int nsets, unsigned n,
                        double *pos, double *mass, double *scale, cudaStream_t st) {
    k_batch_gather<<<sm_count() * 8, 256, 0, st>>>(tab, sets, nsets, n, pos, mass, scale);
    return 1;
}

int batch_scatter_launch(const BatchTab *tab, const SetInfo *sets, int nsets, unsigned n,
                         const double *acc, const double *pot, cudaStream_t st) {
    k_batch_scatter<<<sm_count() * 8, 256, 0, st>>>(tab, sets, nsets, n, acc, pot);
    return 1;
}

int batch_nb_launch(const BatchTab *tab, const SetInfo *sets, int nsets, unsigned n,
                    const long long *off, const int *idx, long long *totals, bool split,
                    cudaStream_t st) {
    k_batch_nb_totals<<<(nsets + 255) / 256, 256, 0, st>>>(sets, nsets, off, totals);
    if (!split) return 1;
    k_batch_nb_split<<<sm_count() * 8, 256, 0, st>>>(tab, sets, nsets, n, off, idx, totals);
    return 2;
}

}  // namespace pt
