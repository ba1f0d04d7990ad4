// pt_tidal.cu -- tidal-tensor measure points (Sec. 6.4.1, Eqs. 25-28, Table 1).
//
// The long-range field near a binary is represented by its acceleration at
// the centre of mass plus a Taylor expansion in r' = r - r_cm: to first order
// (second-order method, tensor A_ij, 6 elements) or second order (third-order
// method, A_ij and the fully symmetric A_ijk, 16 elements; the 1/2 of Eq. 25
// is absorbed into A_ijk as in Table 1).  The accelerations are measured at
// zero-mass points around r_cm -- 4 tetrahedron corners or 8 cube-like
// corners at distance scale d_c -- evaluated by the ordinary long-range force
// pipeline, and the elements follow from the linear system M T = A' (Eq. 28)
// by least squares.  The least-squares operator is derived here from the point
// coordinates (normal equations, solved once on the host in float64) and
// applied per binary by a kernel.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/pt.h"
#include "pt_kernels.cuh"

namespace {

constexpr int kMaxPts = 8, kMaxEl = 16;
const char *const kElem[kMaxEl] = {"xx", "xy", "xz", "yy", "yz", "zz", "xxx", "xxy",
                                   "xxz", "xyy", "xyz", "xzz", "yyy", "yyz", "yzz", "zzz"};

int npts_of(int order) { return order == 2 ? 4 : 8; }
int nel_of(int order) { return order == 2 ? 6 : 16; }

// Unit measure points (Table 1, coordinates / d_c).
void unit_points(int order, double (*p)[3]) {
    const double h = std::sqrt(2.0) / 2.0;
    if (order == 2) {
        const double q[4][3] = {{1, 0, -h}, {-1, 0, -h}, {0, 1, h}, {0, -1, h}};
        std::memcpy(p, q, sizeof q);
    } else {
        const double q[8][3] = {{1, 0, -1}, {0, 1, -1}, {-1, 0, -1}, {0, -1, -1},
                                {1, 0, 1},  {0, 1, 1},  {-1, 0, 1}, {0, -1, 1}};
        std::memcpy(p, q, sizeof q);
    }
}

// d A'_i / d T_e at offset r: the coefficient of element e in component i.
double coef(int i, const char *e, const double *r) {
    const int n = (int)std::strlen(e);
    int idx[3];
    for (int k = 0; k < n; k++) idx[k] = e[k] - 'x';
    if (n == 2) {
        double c = 0;
        if (i == idx[0]) c += r[idx[1]];
        if (i == idx[1] && idx[0] != idx[1]) c += r[idx[0]];
        return c;
    }
    double c = 0;
    for (int j = 0; j < 3; j++)
        for (int k = 0; k < 3; k++) {
            int a[3] = {i, j, k}, b[3] = {idx[0], idx[1], idx[2]};
            // same multiset?
            for (int u = 0; u < 3; u++)
                for (int v = u + 1; v < 3; v++) {
                    if (a[v] < a[u]) { int t = a[u]; a[u] = a[v]; a[v] = t; }
                    if (b[v] < b[u]) { int t = b[u]; b[u] = b[v]; b[v] = t; }
                }
            if (a[0] == b[0] && a[1] == b[1] && a[2] == b[2]) c += r[j] * r[k];
        }
    return c;
}

// Least-squares operator L (nel x 3 npts) with T = L A' for d_c = 1:
// L = (M^T M)^-1 M^T by Gauss-Jordan elimination of the normal matrix.
void least_squares_operator(int order, double *L) {
    const int np = npts_of(order), ne = nel_of(order), nr = 3 * np;
    double pts[kMaxPts][3];
    unit_points(order, pts);
    std::vector<double> M(nr * ne);
    for (int p = 0; p < np; p++)
        for (int i = 0; i < 3; i++)
            for (int e = 0; e < ne; e++) M[(3 * p + i) * ne + e] = coef(i, kElem[e], pts[p]);
    // augmented [M^T M | M^T]
    const int w = ne + nr;
    std::vector<double> A(ne * w, 0.0);
    for (int a = 0; a < ne; a++) {
        for (int b = 0; b < ne; b++)
            for (int r = 0; r < nr; r++) A[a * w + b] += M[r * ne + a] * M[r * ne + b];
        for (int r = 0; r < nr; r++) A[a * w + ne + r] = M[r * ne + a];
    }
    for (int c = 0; c < ne; c++) {
        int piv = c;
        for (int r = c + 1; r < ne; r++)
            if (std::fabs(A[r * w + c]) > std::fabs(A[piv * w + c])) piv = r;
        if (piv != c)
            for (int k = 0; k < w; k++) std::swap(A[c * w + k], A[piv * w + k]);
        const double d = A[c * w + c];
        for (int k = 0; k < w; k++) A[c * w + k] /= d;
        for (int r = 0; r < ne; r++) {
            if (r == c) continue;
            const double f = A[r * w + c];
            if (f != 0.0)
                for (int k = 0; k < w; k++) A[r * w + k] -= f * A[c * w + k];
        }
    }
    for (int e = 0; e < ne; e++)
        for (int r = 0; r < nr; r++) L[e * nr + r] = A[e * w + ne + r];
}

__constant__ double c_L2[6 * 12];     // second-order operator, d_c = 1
__constant__ double c_L3[16 * 24];    // third-order operator, d_c = 1
__constant__ double c_P2[4 * 3];
__constant__ double c_P3[8 * 3];

std::mutex g_mu;
bool g_ready[64] = {};

int upload_tables() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PT_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_ready[dev]) return PT_OK;
    double L2[6 * 12], L3[16 * 24], P2[4][3], P3[8][3];
    least_squares_operator(2, L2);
    least_squares_operator(3, L3);
    unit_points(2, P2);
    unit_points(3, P3);
    if (cudaMemcpyToSymbol(c_L2, L2, sizeof L2) != cudaSuccess ||
        cudaMemcpyToSymbol(c_L3, L3, sizeof L3) != cudaSuccess ||
        cudaMemcpyToSymbol(c_P2, P2, sizeof P2) != cudaSuccess ||
        cudaMemcpyToSymbol(c_P3, P3, sizeof P3) != cudaSuccess)
        return PT_ERR_CUDA;
    g_ready[dev] = true;
    return PT_OK;
}

__global__ void k_tidal_points(int order, long long n, const double *cm, const double *dc, double *pts) {
    const int np = order == 2 ? 4 : 8;
    const double *P = order == 2 ? c_P2 : c_P3;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * np;
         t += (long long)gridDim.x * blockDim.x) {
        const long long b = t / np;
        const int p = (int)(t % np);
        for (int d = 0; d < 3; d++) pts[3 * t + d] = __dadd_rn(cm[3 * b + d], __dmul_rn(dc[b], P[3 * p + d]));
    }
}

// T_e = sum_r L[e][r] A'_r / d_c^(rank - 1), A' = A(point) - A(cm).
__global__ void k_tidal_fit(int order, long long n, const double *acc, const double *dc, double *T) {
    const int np = order == 2 ? 4 : 8, ne = order == 2 ? 6 : 16, nr = 3 * np;
    const double *L = order == 2 ? c_L2 : c_L3;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * ne;
         t += (long long)gridDim.x * blockDim.x) {
        const long long b = t / ne;
        const int e = (int)(t % ne);
        const double *a = acc + b * (long long)(1 + np) * 3;
        double s = 0.0;
        for (int r = 0; r < nr; r++) s += L[e * nr + r] * (a[3 + r] - a[r % 3]);
        const double inv = 1.0 / dc[b];
        T[t] = (e < 6) ? s * inv : s * inv * inv;
    }
}

// A(r) = A(r_cm) + A_ij r'_j (+ A_ijk r'_j r'_k) at query offsets r'.
__global__ void k_tidal_eval(int order, long long nq, long long nb, const long long *owner,
                             const double *T, const double *acc_cm, const double *rel, double *out) {
    const int ne = order == 2 ? 6 : 16;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nq;
         q += (long long)gridDim.x * blockDim.x) {
        const long long b = owner[q];
        if (b < 0 || b >= nb) {   // owner out of range: NaN result, no access
            out[3 * q] = out[3 * q + 1] = out[3 * q + 2] = __longlong_as_double(0x7ff8000000000000ll);
            continue;
        }
        const double *t = T + b * ne;
        const double x = rel[3 * q], y = rel[3 * q + 1], z = rel[3 * q + 2];
        // rank 2: xx xy xz yy yz zz
        double ax = t[0] * x + t[1] * y + t[2] * z;
        double ay = t[1] * x + t[3] * y + t[4] * z;
        double az = t[2] * x + t[4] * y + t[5] * z;
        if (order == 3) {
            // rank 3: xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz (Table 1, second block)
            ax += t[6] * x * x + 2 * t[7] * x * y + 2 * t[8] * x * z + t[9] * y * y + 2 * t[10] * y * z + t[11] * z * z;
            ay += t[7] * x * x + 2 * t[9] * x * y + 2 * t[10] * x * z + t[12] * y * y + 2 * t[13] * y * z + t[14] * z * z;
            az += t[8] * x * x + 2 * t[10] * x * y + 2 * t[11] * x * z + t[13] * y * y + 2 * t[14] * y * z + t[15] * z * z;
        }
        out[3 * q] = acc_cm[3 * b] + ax;
        out[3 * q + 1] = acc_cm[3 * b + 1] + ay;
        out[3 * q + 2] = acc_cm[3 * b + 2] + az;
    }
}

bool dev_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device views of caller buffers: host inputs are copied in, host outputs are
// staged and copied back by finish(); temporaries live until destruction.
struct Staged {
    cudaStream_t st;
    int rc = PT_OK;
    std::vector<void *> owned;
    std::vector<std::pair<void *, void *>> back;   // (host, device)
    std::vector<size_t> back_bytes;
    explicit Staged(cudaStream_t s) : st(s) {}
    void *alloc(size_t bytes) {
        void *d = nullptr;
        if (cudaMalloc(&d, bytes) != cudaSuccess) {
            (void)cudaGetLastError();
            rc = PT_ERR_OOM;
            return nullptr;
        }
        owned.push_back(d);
        return d;
    }
    const void *in(const void *p, size_t bytes) {
        if (rc != PT_OK || dev_ptr(p)) return p;
        void *d = alloc(bytes);
        if (d && cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) rc = PT_ERR_CUDA;
        return d;
    }
    void *out(void *p, size_t bytes) {
        if (rc != PT_OK || dev_ptr(p)) return p;
        void *d = alloc(bytes);
        back.push_back({p, d});
        back_bytes.push_back(bytes);
        return d;
    }
    int finish() {
        if (cudaGetLastError() != cudaSuccess) return PT_ERR_CUDA;
        for (size_t k = 0; k < back.size(); k++)
            if (cudaMemcpyAsync(back[k].first, back[k].second, back_bytes[k], cudaMemcpyDeviceToHost, st) !=
                cudaSuccess)
                return PT_ERR_CUDA;
        return cudaStreamSynchronize(st) == cudaSuccess ? PT_OK : PT_ERR_CUDA;
    }
    ~Staged() {
        if (!owned.empty()) cudaStreamSynchronize(st);
        for (void *d : owned) cudaFree(d);
    }
};

int report(pt_ctx *ctx, int rc, const char *what) {
    if (rc == PT_OK) return rc;
    char msg[160];
    snprintf(msg, sizeof msg, "%s: %s", what,
             rc == PT_ERR_ARG ? "invalid argument" : rc == PT_ERR_OOM ? "out of device memory" : "CUDA error");
    return pt::ctx_fail(ctx, rc, msg);
}

constexpr int kBlock = 256;
int tidal_grid() { return pt::sm_count() * 4; }

}  // namespace

extern "C" {

int pt_tidal_points(pt_ctx *ctx, int order, int64_t n, const double *r_cm, const double *d_c,
                    double *points) {
    if (!ctx) return PT_ERR_ARG;
    if ((order != 2 && order != 3) || n < 0 || (n > 0 && (!r_cm || !d_c || !points)))
        return report(ctx, PT_ERR_ARG, "pt_tidal_points");
    if (n == 0) return PT_OK;
    Staged S(pt::ctx_enter(ctx));
    int rc = upload_tables();
    if (rc != PT_OK) return report(ctx, rc, "pt_tidal_points");
    const int np = npts_of(order);
    const double *cm = (const double *)S.in(r_cm, n * 24);
    const double *dc = (const double *)S.in(d_c, n * 8);
    double *pts = (double *)S.out(points, n * np * 24);
    if (S.rc != PT_OK) return report(ctx, S.rc, "pt_tidal_points");
    k_tidal_points<<<tidal_grid(), kBlock, 0, S.st>>>(order, n, cm, dc, pts);
    return report(ctx, S.finish(), "pt_tidal_points");
}

int pt_tidal_tensor(pt_ctx *ctx, int order, int64_t n, const double *acc, const double *d_c, double *T) {
    if (!ctx) return PT_ERR_ARG;
    if ((order != 2 && order != 3) || n < 0 || (n > 0 && (!acc || !d_c || !T)))
        return report(ctx, PT_ERR_ARG, "pt_tidal_tensor");
    if (n == 0) return PT_OK;
    Staged S(pt::ctx_enter(ctx));
    int rc = upload_tables();
    if (rc != PT_OK) return report(ctx, rc, "pt_tidal_tensor");
    const int np = npts_of(order), ne = nel_of(order);
    const double *a = (const double *)S.in(acc, n * (1 + np) * 24);
    const double *dc = (const double *)S.in(d_c, n * 8);
    double *t = (double *)S.out(T, n * ne * 8);
    if (S.rc != PT_OK) return report(ctx, S.rc, "pt_tidal_tensor");
    k_tidal_fit<<<tidal_grid(), kBlock, 0, S.st>>>(order, n, a, dc, t);
    return report(ctx, S.finish(), "pt_tidal_tensor");
}

int pt_tidal_eval(pt_ctx *ctx, int order, int64_t n_query, const int64_t *owner, const double *T,
                  int64_t n_binaries, const double *acc_cm, const double *rel, double *acc_out) {
    if (!ctx) return PT_ERR_ARG;
    if ((order != 2 && order != 3) || n_query < 0 || n_binaries < 0 ||
        (n_query > 0 && (n_binaries < 1 || !owner || !T || !acc_cm || !rel || !acc_out)))
        return report(ctx, PT_ERR_ARG, "pt_tidal_eval");
    if (n_query == 0) return PT_OK;
    Staged S(pt::ctx_enter(ctx));
    const int ne = nel_of(order);
    const long long *ow = (const long long *)S.in(owner, n_query * 8);
    const double *t = (const double *)S.in(T, n_binaries * ne * 8);
    const double *ac = (const double *)S.in(acc_cm, n_binaries * 24);
    const double *r = (const double *)S.in(rel, n_query * 24);
    double *o = (double *)S.out(acc_out, n_query * 24);
    if (S.rc != PT_OK) return report(ctx, S.rc, "pt_tidal_eval");
    k_tidal_eval<<<tidal_grid(), kBlock, 0, S.st>>>(order, n_query, n_binaries, ow, t, ac, r, o);
    return report(ctx, S.finish(), "pt_tidal_eval");
}

}  // extern "C"
