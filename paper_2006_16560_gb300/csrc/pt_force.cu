// pt_force.cu -- the P3T long-range force kernels, fused neighbour
// extraction, the energy / momentum sums and the neighbour CSR.
//
// One CTA (4 warps) evaluates one walk group at a time, taking groups from
// an atomic work counter.  Every warp holds all of the group's targets (one
// or two per lane) and streams its own quarter of the group's lists: it
// gathers 64 list entries into shared memory, then every lane reads them by
// broadcast and accumulates.  The four warps' partial sums are reduced in
// float64 at the end of the group.
//
// Pair force (Sec. 5.1, Eq. 11; Sec. 6.1, Eqs. 15-17), for x_ij > 0:
//   a_i += m_j (x_j - x_i) (1 - K(x)) / r^3,  P_i += m_j (1 - W(x)) / r
// written branch-free with xs = clamp(x, 0, 1):
//   1 - W = min(2 r/(r_out + r_in) - Lambda xs^5 (14 - 28 xs + 20 xs^2 - 5 xs^3), 1)
// which is 2r/(r_out+r_in) for r <= r_in (so (1 - W)/r is the finite
// constant 2/(r_out+r_in) there), the Eq. 15 interior value for 0 < x < 1
// and 1 beyond r_out.  K(0) = 1 exactly, so no force acts inside r_in.  The
// target's own entry in the PP list adds exactly m_i 2/(r_out+r_in) to P_i,
// which is removed in float64 at the end.  Cells (Sec. 4; Sec. 6.4.2,
// Eqs. 30-31) act through monopole and quadrupole about their centre of
// mass.  phi_i = -G P_i.
//
// Mixed precision: positions are kept as float-float (hi + lo); a PP pair
// forms dx = (hi_j - hi_i) + (lo_j - lo_i), accurate to ~2^-23 |dx| whatever
// the offset from the origin; cells use float offsets from the group's
// first particle.  Per tile the float sums are folded into float-float
// accumulators (Knuth TwoSum).  A neighbour candidate (float r^2 within
// 2^-10 of r_out^2) is confirmed with the exact float64 test.
#include "pt_kernels.cuh"

namespace pt {

constexpr int kFWarps = 4;
constexpr int kFThreads = 32 * kFWarps;
constexpr int kJ = 64;        // list entries per warp tile
constexpr int kIB = 64;       // targets per pass (two per lane)

__device__ __forceinline__ void ff_add(float &hi, float &lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
}

__device__ __forceinline__ double exact_r2(double4 a, double4 b) {
    const double dx = __dsub_rn(b.x, a.x), dy = __dsub_rn(b.y, a.y), dz = __dsub_rn(b.z, a.z);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

__device__ __forceinline__ void emit_pair(const ForceArgs &A, unsigned pi, unsigned pj) {
    unsigned long long k = atomicAdd(&A.st->npairs, 1ull);
    if (k < A.pair_cap) A.pairs[k] = make_uint2(pi, pj);
}

// Per-set constants of the changeover, float64 and float32.
struct Chg {
    double ri, ro, c2, lam, invw, c0, tiny, rout2;
};
__device__ __forceinline__ Chg make_chg(const SetInfo &S) {
    Chg c;
    c.ri = S.r_in;
    c.ro = S.r_out;
    c.c2 = 2.0 / (S.r_out + S.r_in);
    c.lam = (S.r_out - S.r_in) / (S.r_out + S.r_in);
    c.invw = 1.0 / (S.r_out - S.r_in);
    c.c0 = -S.r_in * c.invw;
    const double t = S.r_in > 0.0 ? S.r_in * (1.0 / 1024.0) : S.r_out * (1.0 / 1048576.0);
    c.tiny = t * t;
    c.rout2 = __dmul_rn(S.r_out, S.r_out);
    return c;
}

// ===========================================================================
// Mixed precision (float32 pair arithmetic)
// ===========================================================================

struct ChgF {
    float invw, c0, c2, lam, c35l, tiny, rout2m;
};

template <int NI, int ORDER>
__device__ __forceinline__ void cells_tile_f(const float4 *sA, const float4 *sB, const float2 *sC,
                                             int cnt, const float (&ox)[2], const float (&oy)[2],
                                             const float (&oz)[2], float (&pa)[2][4]) {
#pragma unroll 2
    for (int j = 0; j < cnt; j++) {
        const float4 c = sA[j];
        float4 q;
        float2 q2;
        if (ORDER == 2) {
            q = sB[j];
            q2 = sC[j];
        }
#pragma unroll
        for (int s = 0; s < NI; s++) {
            const float dx = c.x - ox[s], dy = c.y - oy[s], dz = c.z - oz[s];
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const float rinv = rsqrtf(r2);
            const float rinv2 = rinv * rinv;
            const float mr = c.w * rinv;
            const float mr3 = mr * rinv2;
            if (ORDER == 2) {
                // q = (Qxx, Qyy, Qzz, Qxy), q2 = (Qxz, Qyz)
                const float qx = fmaf(q2.x, dz, fmaf(q.w, dy, q.x * dx));
                const float qy = fmaf(q2.y, dz, fmaf(q.y, dy, q.w * dx));
                const float qz = fmaf(q.z, dz, fmaf(q2.y, dy, q2.x * dx));
                const float dqd = fmaf(dz, qz, fmaf(dy, qy, dx * qx));
                const float rinv5 = rinv2 * rinv2 * rinv;
                const float t = dqd * rinv5;
                const float f = fmaf(2.5f * t, rinv2, mr3);
                pa[s][0] = fmaf(-qx, rinv5, fmaf(f, dx, pa[s][0]));
                pa[s][1] = fmaf(-qy, rinv5, fmaf(f, dy, pa[s][1]));
                pa[s][2] = fmaf(-qz, rinv5, fmaf(f, dz, pa[s][2]));
                pa[s][3] = fmaf(0.5f, t, pa[s][3] + mr);
            } else {
                pa[s][0] = fmaf(mr3, dx, pa[s][0]);
                pa[s][1] = fmaf(mr3, dy, pa[s][1]);
                pa[s][2] = fmaf(mr3, dz, pa[s][2]);
                pa[s][3] += mr;
            }
        }
    }
}

template <int NI, bool NB>
__device__ __forceinline__ void pp_tile_f(const ForceArgs &A, const float4 *sH, const float4 *sL,
                                          int cnt, const ChgF &C, const float (&hx)[2],
                                          const float (&hy)[2], const float (&hz)[2],
                                          const float (&lx)[2], const float (&ly)[2],
                                          const float (&lz)[2], const unsigned (&pid)[2],
                                          const bool (&valid)[2], double rout2,
                                          float (&pa)[2][4]) {
#pragma unroll 2
    for (int j = 0; j < cnt; j++) {
        const float4 H = sH[j];
        const float4 L = sL[j];
#pragma unroll
        for (int s = 0; s < NI; s++) {
            const float dx = (H.x - hx[s]) + (L.x - lx[s]);
            const float dy = (H.y - hy[s]) + (L.y - ly[s]);
            const float dz = (H.z - hz[s]) + (L.z - lz[s]);
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (NB && r2 < C.rout2m) {
                const unsigned pj = __float_as_uint(L.w);
                if (valid[s] && pj != pid[s] && exact_r2(A.sp64[pid[s]], A.sp64[pj]) < rout2)
                    emit_pair(A, pid[s], pj);
            }
            const float r2c = fmaxf(r2, C.tiny);
            const float rinv = rsqrtf(r2c);
            const float r = r2c * rinv;
            const float xs = __saturatef(fmaf(r, C.invw, C.c0));
            // K(xs) = (xs - 1)^4 (1 + 4 xs + 10 xs^2 + 20 xs^3 + 35 Lambda xs^4)
            const float t = xs - 1.0f;
            const float t2 = t * t;
            const float kq = fmaf(fmaf(fmaf(fmaf(C.c35l, xs, 20.0f), xs, 10.0f), xs, 4.0f), xs, 1.0f);
            const float omk = fmaf(-t2 * t2, kq, 1.0f);          // 1 - K
            // 1 - W = min(2r/(r_out+r_in) - Lambda xs^5 (14 - 28 xs + 20 xs^2 - 5 xs^3), 1)
            const float x2 = xs * xs;
            const float x5 = x2 * x2 * xs;
            const float wp = fmaf(fmaf(fmaf(-5.0f, xs, 20.0f), xs, -28.0f), xs, 14.0f);
            const float omw = fminf(fmaf(-C.lam * x5, wp, r * C.c2), 1.0f);
            const float mr = H.w * rinv;
            const float fk = (omk * mr) * (rinv * rinv);
            pa[s][0] = fmaf(fk, dx, pa[s][0]);
            pa[s][1] = fmaf(fk, dy, pa[s][1]);
            pa[s][2] = fmaf(fk, dz, pa[s][2]);
            pa[s][3] = fmaf(omw, mr, pa[s][3]);
        }
    }
}

template <int NI>
__device__ __forceinline__ void fold(float (&pa)[2][4], float (&fh)[2][4], float (&fl)[2][4]) {
#pragma unroll
    for (int s = 0; s < NI; s++)
#pragma unroll
        for (int c = 0; c < 4; c++) {
            ff_add(fh[s][c], fl[s][c], pa[s][c]);
            pa[s][c] = 0.0f;
        }
}

template <int NI, int ORDER, bool NB>
__device__ void group_pass_f(const ForceArgs &A, unsigned g, const uint2 gr, unsigned i0,
                             const ChgF &C, double rout2, float4 (*sA)[kJ], float4 (*sB)[kJ],
                             float2 (*sC)[kJ], double (*red)[kIB][4]) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float4 Hg = A.spH[gr.x], Lg = A.spL[gr.x];
    float hx[2], hy[2], hz[2], lx[2], ly[2], lz[2], ox[2], oy[2], oz[2];
    unsigned pid[2];
    bool valid[2];
#pragma unroll
    for (int s = 0; s < 2; s++) {
        const unsigned idx = i0 + lane + 32 * s;
        valid[s] = idx < gr.y;
        pid[s] = gr.x + (valid[s] ? idx : 0u);
        const float4 H = A.spH[pid[s]], L = A.spL[pid[s]];
        hx[s] = H.x; hy[s] = H.y; hz[s] = H.z;
        lx[s] = L.x; ly[s] = L.y; lz[s] = L.z;
        ox[s] = (H.x - Hg.x) + (L.x - Lg.x);
        oy[s] = (H.y - Hg.y) + (L.y - Lg.y);
        oz[s] = (H.z - Hg.z) + (L.z - Lg.z);
    }
    float pa[2][4], fh[2][4], fl[2][4];
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int c = 0; c < 4; c++) pa[s][c] = fh[s][c] = fl[s][c] = 0.0f;
    // ---- cells
    const unsigned nc = A.gr_nc[g];
    const unsigned long long co = A.gr_co[g];
    for (unsigned t = w * kJ; t < nc; t += kFWarps * kJ) {
        const int cnt = (int)min((unsigned)kJ, nc - t);
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int e = lane + 32 * h;
            if (e < cnt) {
                const unsigned v = A.cells[co + t + e];
                const float4 f0 = A.nd_f[4 * v], f1 = A.nd_f[4 * v + 1];
                sA[w][e] = make_float4((f0.x - Hg.x) + (f1.x - Lg.x), (f0.y - Hg.y) + (f1.y - Lg.y),
                                       (f0.z - Hg.z) + (f1.z - Lg.z), f0.w);
                if (ORDER == 2) {
                    const float4 f2 = A.nd_f[4 * v + 2], f3 = A.nd_f[4 * v + 3];
                    sB[w][e] = make_float4(f1.w, f2.x, f2.y, f2.z);
                    sC[w][e] = make_float2(f2.w, f3.x);
                }
            }
        }
        __syncwarp();
        cells_tile_f<NI, ORDER>(sA[w], sB[w], sC[w], cnt, ox, oy, oz, pa);
        __syncwarp();
        fold<NI>(pa, fh, fl);
    }
    // ---- particle-particle
    const unsigned np = A.gr_np[g];
    const unsigned long long po = A.gr_po[g];
    for (unsigned t = w * kJ; t < np; t += kFWarps * kJ) {
        const int cnt = (int)min((unsigned)kJ, np - t);
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int e = lane + 32 * h;
            if (e < cnt) {
                const unsigned p = A.pp[po + t + e];
                sA[w][e] = A.spH[p];
                float4 L = A.spL[p];
                L.w = __uint_as_float(p);
                sB[w][e] = L;
            }
        }
        __syncwarp();
        if (NB && A.want_nb)
            pp_tile_f<NI, true>(A, sA[w], sB[w], cnt, C, hx, hy, hz, lx, ly, lz, pid, valid, rout2, pa);
        else
            pp_tile_f<NI, false>(A, sA[w], sB[w], cnt, C, hx, hy, hz, lx, ly, lz, pid, valid, rout2, pa);
        __syncwarp();
        fold<NI>(pa, fh, fl);
    }
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int c = 0; c < 4; c++)
            red[w][lane + 32 * s][c] = (s < NI) ? (double)fh[s][c] + (double)fl[s][c] : 0.0;
}

// Final per-target sums (threads 0..kIB-1): fixed-order float64 reduction over
// the warps, removal of the self entry, output in caller order.
__device__ __forceinline__ void write_targets(const ForceArgs &A, const uint2 gr, unsigned i0,
                                              double c2, double (*red)[kIB][4], double (&ep)[4]) {
    const unsigned t = threadIdx.x;
    if (t < kIB && i0 + t < gr.y) {
        double s[4] = {0, 0, 0, 0};
        for (int w = 0; w < kFWarps; w++)
            for (int c = 0; c < 4; c++) s[c] += red[w][t][c];
        const unsigned p = gr.x + i0 + t;
        const double m = A.sp64[p].w;
        const double P = s[3] - m * c2;              // remove the self entry
        const unsigned i = A.perm[p];
        const double ax = A.G * s[0], ay = A.G * s[1], az = A.G * s[2], phi = -A.G * P;
        A.acc[3ull * i] = ax;
        A.acc[3ull * i + 1] = ay;
        A.acc[3ull * i + 2] = az;
        A.pot[i] = phi;
        ep[0] += 0.5 * m * phi;
        ep[1] += m * ax;
        ep[2] += m * ay;
        ep[3] += m * az;
    }
}

__device__ __forceinline__ void group_partials(const ForceArgs &A, unsigned g, double (&ep)[4],
                                               double (*ered)[4]) {
    // threads 0..63 (warps 0 and 1) hold the partials
    const int w = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 4; c++) ep[c] = warp_sum(ep[c]);
    if ((threadIdx.x & 31) == 0)
        for (int c = 0; c < 4; c++) ered[w][c] = ep[c];
    __syncthreads();
    if (threadIdx.x == 0) {
        double e[4];
        for (int c = 0; c < 4; c++) e[c] = ered[0][c] + ered[1][c];
        A.gpart[g] = make_double4(e[0], e[1], e[2], e[3]);
    }
}

template <int ORDER, bool NB>
__global__ void __launch_bounds__(kFThreads) k_force_mixed(ForceArgs A) {
    __shared__ float4 sA[kFWarps][kJ];
    __shared__ float4 sB[kFWarps][kJ];
    __shared__ float2 sC[kFWarps][kJ];
    __shared__ double red[kFWarps][kIB][4];
    __shared__ double ered[kFWarps][4];
    __shared__ unsigned gsh;
    const unsigned ng = A.st->ngroups;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) gsh = (unsigned)atomicAdd(&A.st->work[2], 1ull);
        __syncthreads();
        const unsigned g = gsh;
        if (g >= ng) break;
        const uint2 gr = A.gr_r[g];
        const Chg C64 = make_chg(A.sets[A.gr_a[g].w]);
        ChgF C;
        C.invw = (float)C64.invw;
        C.c0 = (float)C64.c0;
        C.c2 = (float)C64.c2;
        C.lam = (float)C64.lam;
        C.c35l = (float)(35.0 * C64.lam);
        C.tiny = fmaxf((float)C64.tiny, 1e-36f);
        C.rout2m = (float)(C64.rout2 * (1.0 + 1.0 / 1024.0));
        double ep[4] = {0, 0, 0, 0};
        for (unsigned i0 = 0; i0 < gr.y; i0 += kIB) {
            if (gr.y - i0 > 32)
                group_pass_f<2, ORDER, NB>(A, g, gr, i0, C, C64.rout2, sA, sB, sC, red);
            else
                group_pass_f<1, ORDER, NB>(A, g, gr, i0, C, C64.rout2, sA, sB, sC, red);
            __syncthreads();
            write_targets(A, gr, i0, C64.c2, red, ep);
            __syncthreads();
        }
        group_partials(A, g, ep, ered);
    }
}

// ===========================================================================
// Float64
// ===========================================================================

template <int NI, int ORDER>
__device__ __forceinline__ void cells_tile_d(const double4 *sA, const double4 *sB, const double2 *sC,
                                             int cnt, const double (&xx)[2], const double (&xy)[2],
                                             const double (&xz)[2], double (&pa)[2][4]) {
    for (int j = 0; j < cnt; j++) {
        const double4 c = sA[j];
        double4 q;
        double2 q2;
        if (ORDER == 2) {
            q = sB[j];
            q2 = sC[j];
        }
#pragma unroll
        for (int s = 0; s < NI; s++) {
            const double dx = c.x - xx[s], dy = c.y - xy[s], dz = c.z - xz[s];
            const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
            const double rinv = rsqrt(r2);
            const double rinv2 = rinv * rinv;
            const double mr = c.w * rinv;
            const double mr3 = mr * rinv2;
            if (ORDER == 2) {
                const double qx = fma(q2.x, dz, fma(q.w, dy, q.x * dx));
                const double qy = fma(q2.y, dz, fma(q.y, dy, q.w * dx));
                const double qz = fma(q.z, dz, fma(q2.y, dy, q2.x * dx));
                const double dqd = fma(dz, qz, fma(dy, qy, dx * qx));
                const double rinv5 = rinv2 * rinv2 * rinv;
                const double t = dqd * rinv5;
                const double f = fma(2.5 * t, rinv2, mr3);
                pa[s][0] = fma(-qx, rinv5, fma(f, dx, pa[s][0]));
                pa[s][1] = fma(-qy, rinv5, fma(f, dy, pa[s][1]));
                pa[s][2] = fma(-qz, rinv5, fma(f, dz, pa[s][2]));
                pa[s][3] = fma(0.5, t, pa[s][3] + mr);
            } else {
                pa[s][0] = fma(mr3, dx, pa[s][0]);
                pa[s][1] = fma(mr3, dy, pa[s][1]);
                pa[s][2] = fma(mr3, dz, pa[s][2]);
                pa[s][3] += mr;
            }
        }
    }
}

template <int NI, bool NB>
__device__ __forceinline__ void pp_tile_d(const ForceArgs &A, const double4 *sP, const unsigned *sI,
                                          int cnt, const Chg &C, const double (&xx)[2],
                                          const double (&xy)[2], const double (&xz)[2],
                                          const unsigned (&pid)[2], const bool (&valid)[2],
                                          double (&pa)[2][4]) {
    for (int j = 0; j < cnt; j++) {
        const double4 P = sP[j];
#pragma unroll
        for (int s = 0; s < NI; s++) {
            const double dx = __dsub_rn(P.x, xx[s]), dy = __dsub_rn(P.y, xy[s]), dz = __dsub_rn(P.z, xz[s]);
            const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            if (NB && r2 < C.rout2) {
                const unsigned pj = sI[j];
                if (valid[s] && pj != pid[s]) emit_pair(A, pid[s], pj);
            }
            const double r2c = fmax(r2, C.tiny);
            const double rinv = rsqrt(r2c);
            const double r = r2c * rinv;
            const double xs = fmin(fmax(fma(r, C.invw, C.c0), 0.0), 1.0);
            const double t = xs - 1.0;
            const double t2 = t * t;
            const double kq = fma(fma(fma(fma(35.0 * C.lam, xs, 20.0), xs, 10.0), xs, 4.0), xs, 1.0);
            const double omk = fma(-t2 * t2, kq, 1.0);
            const double x2 = xs * xs;
            const double x5 = x2 * x2 * xs;
            const double wp = fma(fma(fma(-5.0, xs, 20.0), xs, -28.0), xs, 14.0);
            const double omw = fmin(fma(-C.lam * x5, wp, r * C.c2), 1.0);
            const double mr = P.w * rinv;
            const double fk = (omk * mr) * (rinv * rinv);
            pa[s][0] = fma(fk, dx, pa[s][0]);
            pa[s][1] = fma(fk, dy, pa[s][1]);
            pa[s][2] = fma(fk, dz, pa[s][2]);
            pa[s][3] = fma(omw, mr, pa[s][3]);
        }
    }
}

template <int NI, int ORDER, bool NB>
__device__ void group_pass_d(const ForceArgs &A, unsigned g, const uint2 gr, unsigned i0,
                             const Chg &C, double4 (*sA)[kJ], double4 (*sB)[kJ],
                             double2 (*sC)[kJ], unsigned (*sI)[kJ], double (*red)[kIB][4]) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double xx[2], xy[2], xz[2];
    unsigned pid[2];
    bool valid[2];
#pragma unroll
    for (int s = 0; s < 2; s++) {
        const unsigned idx = i0 + lane + 32 * s;
        valid[s] = idx < gr.y;
        pid[s] = gr.x + (valid[s] ? idx : 0u);
        const double4 P = A.sp64[pid[s]];
        xx[s] = P.x; xy[s] = P.y; xz[s] = P.z;
    }
    double pa[2][4];
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int c = 0; c < 4; c++) pa[s][c] = 0.0;
    const unsigned nc = A.gr_nc[g];
    const unsigned long long co = A.gr_co[g];
    for (unsigned t = w * kJ; t < nc; t += kFWarps * kJ) {
        const int cnt = (int)min((unsigned)kJ, nc - t);
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int e = lane + 32 * h;
            if (e < cnt) {
                const unsigned v = A.cells[co + t + e];
                sA[w][e] = A.nd_c[v];
                if (ORDER == 2) {
                    const double4 q0 = A.nd_q[2 * v], q1 = A.nd_q[2 * v + 1];
                    sB[w][e] = q0;
                    sC[w][e] = make_double2(q1.x, q1.y);
                }
            }
        }
        __syncwarp();
        cells_tile_d<NI, ORDER>(sA[w], sB[w], sC[w], cnt, xx, xy, xz, pa);
        __syncwarp();
    }
    const unsigned np = A.gr_np[g];
    const unsigned long long po = A.gr_po[g];
    for (unsigned t = w * kJ; t < np; t += kFWarps * kJ) {
        const int cnt = (int)min((unsigned)kJ, np - t);
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int e = lane + 32 * h;
            if (e < cnt) {
                const unsigned p = A.pp[po + t + e];
                sA[w][e] = A.sp64[p];
                sI[w][e] = p;
            }
        }
        __syncwarp();
        if (NB && A.want_nb)
            pp_tile_d<NI, true>(A, sA[w], sI[w], cnt, C, xx, xy, xz, pid, valid, pa);
        else
            pp_tile_d<NI, false>(A, sA[w], sI[w], cnt, C, xx, xy, xz, pid, valid, pa);
        __syncwarp();
    }
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int c = 0; c < 4; c++) red[w][lane + 32 * s][c] = (s < NI) ? pa[s][c] : 0.0;
}

template <int ORDER, bool NB>
__global__ void __launch_bounds__(kFThreads) k_force_fp64(ForceArgs A) {
    __shared__ double4 sA[kFWarps][kJ];
    __shared__ double4 sB[kFWarps][kJ];
    __shared__ double2 sC[kFWarps][kJ];
    __shared__ unsigned sI[kFWarps][kJ];
    __shared__ double red[kFWarps][kIB][4];
    __shared__ double ered[kFWarps][4];
    __shared__ unsigned gsh;
    const unsigned ng = A.st->ngroups;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) gsh = (unsigned)atomicAdd(&A.st->work[2], 1ull);
        __syncthreads();
        const unsigned g = gsh;
        if (g >= ng) break;
        const uint2 gr = A.gr_r[g];
        const Chg C = make_chg(A.sets[A.gr_a[g].w]);
        double ep[4] = {0, 0, 0, 0};
        for (unsigned i0 = 0; i0 < gr.y; i0 += kIB) {
            if (gr.y - i0 > 32)
                group_pass_d<2, ORDER, NB>(A, g, gr, i0, C, sA, sB, sC, sI, red);
            else
                group_pass_d<1, ORDER, NB>(A, g, gr, i0, C, sA, sB, sC, sI, red);
            __syncthreads();
            write_targets(A, gr, i0, C.c2, red, ep);
            __syncthreads();
        }
        group_partials(A, g, ep, ered);
    }
}

// ===========================================================================
// Totals over groups (fixed-order reduction, one block)
// ===========================================================================

__global__ void __launch_bounds__(1024) k_force_reduce(const double4 *gpart, const uint2 *gr_r,
                                                       const unsigned *gr_nc, const unsigned *gr_np,
                                                       Status *st) {
    __shared__ double se[1024][4];
    __shared__ unsigned long long si[1024][2];
    const unsigned ng = st->ngroups;
    double e[4] = {0, 0, 0, 0};
    unsigned long long ci = 0, pi = 0;
    for (unsigned g = threadIdx.x; g < ng; g += blockDim.x) {
        const double4 p = gpart[g];
        e[0] += p.x; e[1] += p.y; e[2] += p.z; e[3] += p.w;
        const unsigned long long n = gr_r[g].y;
        ci += n * gr_nc[g];
        pi += n * gr_np[g];
    }
    for (int c = 0; c < 4; c++) se[threadIdx.x][c] = e[c];
    si[threadIdx.x][0] = ci;
    si[threadIdx.x][1] = pi;
    __syncthreads();
    for (int s = 512; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            for (int c = 0; c < 4; c++) se[threadIdx.x][c] += se[threadIdx.x + s][c];
            si[threadIdx.x][0] += si[threadIdx.x + s][0];
            si[threadIdx.x][1] += si[threadIdx.x + s][1];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        st->energy = se[0][0];
        st->mom[0] = se[0][1];
        st->mom[1] = se[0][2];
        st->mom[2] = se[0][3];
        st->cell_inter = si[0][0];
        st->pp_inter = si[0][1];
    }
}

int force_launch(const ForceArgs &A, int precision, cudaStream_t st) {
    const int blocks = 152 * 8;
    if (precision == 1) {
        if (A.order == 2) k_force_mixed<2, true><<<blocks, kFThreads, 0, st>>>(A);
        else k_force_mixed<0, true><<<blocks, kFThreads, 0, st>>>(A);
    } else {
        if (A.order == 2) k_force_fp64<2, true><<<blocks, kFThreads, 0, st>>>(A);
        else k_force_fp64<0, true><<<blocks, kFThreads, 0, st>>>(A);
    }
    return 1;
}

int force_reduce_launch(const ForceArgs &A, cudaStream_t st) {
    k_force_reduce<<<1, 1024, 0, st>>>(A.gpart, A.gr_r, A.gr_nc, A.gr_np, A.st);
    return 1;
}

// ===========================================================================
// Neighbour CSR: pairs (sorted i, sorted j) -> keys (orig i * n + orig j) ->
// radix sort -> row offsets by binary search -> column indices.
// ===========================================================================

__global__ void k_nb_keys(NbArgs A) {
    unsigned long long np = A.st->npairs;
    if (np > A.pair_cap) np = A.pair_cap;
    if (blockIdx.x == 0 && threadIdx.x == 0) *A.npairs_dev = (unsigned)np;
    for (unsigned long long k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
        const uint2 p = A.pairs[k];
        A.keys[k] = (unsigned long long)A.perm[p.x] * A.n + A.perm[p.y];
        A.vals[k] = (unsigned)k;
    }
}

__global__ void k_nb_csr(NbArgs A) {
    const unsigned np = *A.npairs_dev;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i <= A.n; i += gridDim.x * blockDim.x) {
        const unsigned long long key = (unsigned long long)i * A.n;
        unsigned lo = 0, hi = np;
        while (lo < hi) {
            unsigned mid = lo + ((hi - lo) >> 1);
            if (A.keys_sorted[mid] < key) lo = mid + 1; else hi = mid;
        }
        A.nb_off[i] = (long long)lo;
    }
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x)
        A.nb_idx[k] = (int)(A.keys_sorted[k] % A.n);
}

int nb_launch(const NbArgs &A, cudaStream_t st) {
    k_nb_keys<<<152 * 4, 256, 0, st>>>(A);
    int nk = radix_sort(A.keys, A.vals, A.keys_sorted, A.vals_sorted, A.npairs_dev,
                        (unsigned)A.pair_cap, 0, A.key_bits, nullptr, 0, A.sort_tmp, st);
    k_nb_csr<<<152 * 4, 256, 0, st>>>(A);
    return nk + 2;
}

}  // namespace pt
