// pt_force.cu -- the P3T long-range force kernels, fused neighbour
// extraction, the energy / momentum sums and the neighbour CSR.
//
// One CTA (4 warps) evaluates one walk group at a time, taking groups from
// an atomic work counter in the order k_group_order writes (largest pass
// configuration first).  Every warp holds all of the group's targets (two or
// three per lane) and streams its own quarter of the group's lists: it
// gathers a tile of list entries into shared memory (128 in the mixed
// kernel, 64 in the float64 one), then every lane reads them by broadcast and
// accumulates.  The four warps' partial sums are reduced in float64 at the
// end of the group, in a fixed order.  Four warps per group rather than one
// keep small sets (a few thousand particles, a few hundred groups) spread
// over the whole GPU.  A group has one cell list and two PP segments: near
// (leaves within r_out of the group's box: changeover and neighbour tests)
// and far (every pair at least r_out apart: plain Newtonian pairs).
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
// accumulators (Knuth TwoSum).  A neighbour candidate (float r^2 below a
// per-group bound that no pair within r_out can exceed, see vote_rout2) is
// confirmed with the exact float64 test.
#include <algorithm>

#include "pt_kernels.cuh"

namespace pt {

constexpr int kFWarps = 4;
constexpr int kFThreads = 32 * kFWarps;
#ifndef PT_FORCE_TILE
#define PT_FORCE_TILE 128
#endif
constexpr int kJ = PT_FORCE_TILE;   // list entries per warp tile of the mixed kernel
constexpr int kJD = 64;             // list entries per warp tile of the float64 kernel
#ifndef PT_FORCE_UNROLL_PAIRS
#define PT_FORCE_UNROLL_PAIRS 1
#endif
constexpr int kUnrollPairs = PT_FORCE_UNROLL_PAIRS;   // unroll of the packed cell-pair loop
#ifndef PT_FORCE_UNROLL_PP
#define PT_FORCE_UNROLL_PP 1
#endif
constexpr int kUnrollPP = PT_FORCE_UNROLL_PP;   // unroll of the near-segment PP-pair loop
#ifndef PT_FORCE_UNROLL_FAR
#define PT_FORCE_UNROLL_FAR 4
#endif
constexpr int kUnrollFar = PT_FORCE_UNROLL_FAR;   // unroll of the far-segment PP-pair loop
constexpr int kIB = 64;       // targets per pass of the float64 kernel (two per lane)
constexpr int kSlotMax = 96;  // largest pass of the mixed kernel
#ifndef PT_FORCE_MIN_BLOCKS
#define PT_FORCE_MIN_BLOCKS 4     // resident CTAs per SM the register budget is sized for
#endif

__device__ __forceinline__ void ff_add(float &hi, float &lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
}

// Packed float32 pairs: one f32x2 instruction does the same operation on two
// values (two cells of a tile at once), halving the issue slots the float32
// arithmetic takes; the FP32 pipe's throughput is the same as for scalars.
typedef unsigned long long f2x;
__device__ __forceinline__ f2x pk2(float a, float b) {
    f2x r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 up2(f2x v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ f2x add2(f2x a, f2x b) {
    f2x r;
    asm("add.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2x sub2(f2x a, f2x b) {
    f2x r;
    asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2x mul2(f2x a, f2x b) {
    f2x r;
    asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c) {
    f2x r;
    asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
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
    float invw, c0, c2, k0, w0, w1, w2, w3, tiny, rout2m;
};

// Near-vote bound of a group: a float32 r^2 at or above it proves that the
// pair is at least r_out (r_out,ij = s_ij r_out for mass-dependent radii)
// apart, so K = W = 0 and the pair cannot be a neighbour.  With u = 2^-24:
// an offset o from the group's first particle, formed as
// (hi_j - hi_g) + (lo_j - lo_g), is within 2u|o| + 2u^2 (|x_j| + |x_g|) of
// the true offset; dx = o_j - o_i adds u|dx|.  Every member is within E of
// the first particle (E = diagonal of the group's grid box, two cells added
// for the rounding of the keys), and a partner j within r_out of member i is
// within E + r_out of it, so |r_float - r| <= 4uE + 3ur + O(u^2 X).  r^2 in
// float32 adds 3u relative, 1/s_ij and its square 4u more.  The bound takes
// twice the E term and the relative terms many times over:
//   r_v = r_out (1 + 2^-18) + 2^-21 E + 2^-40 X,  bound = r_v^2 (1 + 2^-20),
// X = sum over the axes of |origin| + S (the largest coordinate sizes).  A
// compact group (E ~ 10 r_out) gets a margin of ~2^-17 on r_out; a wide halo
// group a proportionally larger one.
__device__ __forceinline__ float vote_rout2(const uint4 ga, const uint4 gb, const SetInfo &S) {
    const double cell = S.S * (1.0 / (double)kGrid);
    const double ex = ((double)gb.x - (double)ga.x + 2.0) * cell;
    const double ey = ((double)gb.y - (double)ga.y + 2.0) * cell;
    const double ez = ((double)gb.z - (double)ga.z + 2.0) * cell;
    const double E = sqrt(ex * ex + ey * ey + ez * ez);
    const double X = fabs(S.origin[0]) + fabs(S.origin[1]) + fabs(S.origin[2]) + 3.0 * S.S;
    const double rv = S.r_out * (1.0 + 0x1p-18) + 0x1p-21 * E + 0x1p-40 * X;
    return (float)(rv * rv * (1.0 + 0x1p-20));
}

// Lane layout of one warp for a pass over up to NI * L targets: the warp's
// lanes form J = 32 / L sub-streams of L lanes; lane (s, l) holds targets
// l, l + L, .., l + (NI-1) L and takes list entries s, s + J, .. of every
// tile, so all lanes of a sub-stream read the same entry (shared-memory
// broadcast).  The configuration is picked per pass as the smallest slot
// count NI * L that covers the remaining targets, which keeps most lanes busy
// for the uneven group sizes a tree produces.
// Cell tile in pair layout: pair P holds two cells (a, b) as five float4
// rows (xa, xb, ya, yb), (za, zb, ma, mb), (Qxx, Qyy), (Qzz, Qxy), (Qxz, Qyz),
// each 64-bit half a packed (a, b) operand.  Sub-stream s takes pairs
// s, s + J, ..; npairs is a multiple of J (the tile is padded with massless
// cells far away).
template <int NI, int J, int ORDER>
__device__ __forceinline__ void cells_tile_f2(const ulonglong2 (*sP)[kJ / 2], int s, int npairs,
                                              const f2x (&OX)[NI], const f2x (&OY)[NI],
                                              const f2x (&OZ)[NI], f2x (&PA)[NI][4]) {
    const f2x m25 = pk2(-2.5f, -2.5f), mhalf = pk2(-0.5f, -0.5f);
#pragma unroll kUnrollPairs
    for (int P = s; P < npairs; P += J) {
        const ulonglong2 xy = sP[0][P], zm = sP[1][P];
        ulonglong2 qa, qb, qc;
        if (ORDER == 2) {
            qa = sP[2][P];
            qb = sP[3][P];
            qc = sP[4][P];
        }
#pragma unroll
        for (int k = 0; k < NI; k++) {
            const f2x dx = sub2(xy.x, OX[k]), dy = sub2(xy.y, OY[k]), dz = sub2(zm.x, OZ[k]);
            const float2 r2 = up2(fma2(dz, dz, fma2(dy, dy, mul2(dx, dx))));
            const f2x rinv = pk2(rsqrtf(r2.x), rsqrtf(r2.y));
            const f2x rinv2 = mul2(rinv, rinv);
            const f2x mr = mul2(zm.y, rinv);
            if (ORDER == 2) {
                // the tile holds -Q: qa = -(Qxx, Qyy), qb = -(Qzz, Qxy), qc = -(Qxz, Qyz)
                const f2x qx = fma2(qc.x, dz, fma2(qb.y, dy, mul2(qa.x, dx)));   // (-Q d)_x
                const f2x qy = fma2(qc.y, dz, fma2(qa.y, dy, mul2(qb.y, dx)));
                const f2x qz = fma2(qb.x, dz, fma2(qc.y, dy, mul2(qc.x, dx)));
                const f2x rinv5 = mul2(mul2(rinv2, rinv2), rinv);
                const f2x nt = mul2(fma2(dz, qz, fma2(dy, qy, mul2(dx, qx))), rinv5);   // -t, t = d.Q.d / r^5
                // f = (mr + 2.5 t) / r^2;  a += f d - Q d / r^5;  P += mr + t / 2
                const f2x f = mul2(fma2(nt, m25, mr), rinv2);
                PA[k][0] = fma2(qx, rinv5, fma2(f, dx, PA[k][0]));
                PA[k][1] = fma2(qy, rinv5, fma2(f, dy, PA[k][1]));
                PA[k][2] = fma2(qz, rinv5, fma2(f, dz, PA[k][2]));
                PA[k][3] = fma2(nt, mhalf, add2(PA[k][3], mr));
            } else {
                const f2x mr3 = mul2(mr, rinv2);
                PA[k][0] = fma2(mr3, dx, PA[k][0]);
                PA[k][1] = fma2(mr3, dy, PA[k][1]);
                PA[k][2] = fma2(mr3, dz, PA[k][2]);
                PA[k][3] = add2(PA[k][3], mr);
            }
        }
    }
}

// Changeover pair (one list entry H, L against target k): the full 1 - K,
// 1 - W path, and the float64 confirmation of a neighbour candidate.
template <int NI, bool NB, bool MD>
__device__ __forceinline__ void pp_changeover_f(const ForceArgs &A, const float4 &H, const float4 &L,
                                                unsigned pj, bool real, const ChgF &C, int k,
                                                float hx, float hy, float hz, float lx, float ly, float lz,
                                                float invs_t, unsigned pid, bool valid, double rout2,
                                                double rout, float (&pa)[NI][4]) {
    const float dx = (H.x - hx) + (L.x - lx);
    const float dy = (H.y - hy) + (L.y - ly);
    const float dz = (H.z - hz) + (L.z - lz);
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    float invs = 1.0f, q2 = r2;
    if (MD) {       // pair radii s_ij (r_in, r_out); 1/s_ij is the smaller inverse (L.w = 1/s_j)
        invs = fminf(invs_t, L.w);
        q2 = r2 * (invs * invs);
    }
    if (NB && q2 < C.rout2m && valid && real) {
        double ro2 = rout2;
        if (MD) {
            const double ro = __dmul_rn(rout, fmax(A.ssc[pid], A.ssc[pj]));
            ro2 = __dmul_rn(ro, ro);
        }
        if (pj != pid && exact_r2(A.sp64[pid], A.sp64[pj]) < ro2) emit_pair(A, pid, pj);
    }
    const float r2c = fmaxf(r2, C.tiny);
    const float rinv = rsqrtf(r2c);
    const float r = MD ? (r2c * rinv) * invs : r2c * rinv;    // r / s_ij
    const float xs = __saturatef(fmaf(r, C.invw, C.c0));
    // 1 - K(xs), K = (xs - 1)^4 (1 + 4 xs + 10 xs^2 + 20 xs^3 + 35 Lambda xs^4).
    // With k0 = 35 (1 - Lambda) = 70 r_in / (r_out + r_in):
    //   K's quartic  = 1 + 4 xs + 10 xs^2 + 20 xs^3 + 35 xs^4 - k0 xs^4,
    //   1 - K        = xs^4 (k0 + xs (A(xs) - k0 B(xs))),
    //   A = 56 - 140 xs + 120 xs^2 - 35 xs^3,  B = 4 - 6 xs + 4 xs^2 - xs^3.
    // Subtracting K from 1 loses all relative accuracy as xs -> 0 (K -> 1),
    // where a close companion's pull m (1 - K) / r^2 can still dominate the
    // sum; the second form keeps it there but cancels near xs = 1, so each is
    // used on its own half.  Only k0 is a per-set constant: the rest are
    // immediates, which keeps the register budget unchanged.
    const float x2 = xs * xs;
    const float x4 = x2 * x2;
    const float t = xs - 1.0f;
    const float t2 = t * t;
    const float kq = fmaf(-C.k0, x4, fmaf(fmaf(fmaf(fmaf(35.0f, xs, 20.0f), xs, 10.0f), xs, 4.0f), xs, 1.0f));
    const float hi = fmaf(-t2 * t2, kq, 1.0f);
    const float pa3 = fmaf(fmaf(fmaf(-35.0f, xs, 120.0f), xs, -140.0f), xs, 56.0f);
    const float pb3 = fmaf(fmaf(fmaf(-1.0f, xs, 4.0f), xs, -6.0f), xs, 4.0f);
    const float lo = x4 * fmaf(xs, fmaf(-C.k0, pb3, pa3), C.k0);
    const float omk = xs < 0.5f ? lo : hi;
    // 1 - W = min(2r/(r_out+r_in) - Lambda xs^5 (14 - 28 xs + 20 xs^2 - 5 xs^3), 1),
    // with Lambda folded into the cubic's coefficients
    const float x5 = x4 * xs;
    const float wp = fmaf(fmaf(fmaf(C.w3, xs, C.w2), xs, C.w1), xs, C.w0);
    const float omw = fminf(fmaf(-x5, wp, r * C.c2), 1.0f);
    const float mr = H.w * rinv;
    const float fk = (omk * mr) * (rinv * rinv);
    pa[k][0] = fmaf(fk, dx, pa[k][0]);
    pa[k][1] = fmaf(fk, dy, pa[k][1]);
    pa[k][2] = fmaf(fk, dz, pa[k][2]);
    pa[k][3] = fmaf(omw, mr, pa[k][3]);
}

// PP tile in pair layout: pair P holds list entries (a, b) as float4 rows
// (ox, oy), (oz, m) of packed (a, b) halves -- float offsets from the
// group's first particle, formed from the float-float positions -- plus
// (1/s, -) for mass-dependent radii, and their particle ids in sI[2P],
// sI[2P + 1].  Every lane runs the same number of iterations (the tile is
// padded to a multiple of 2J with massless entries far away), so the warp can
// vote per iteration: when neither entry of any lane lies within r_out
// (float r^2 at or above the group's vote_rout2 bound), K = W = 0 exactly and both plain
// Newtonian pairs are evaluated with packed f32x2 arithmetic on the offsets;
// otherwise every lane takes the full changeover path for both entries on
// float-float differences, with neighbour candidates confirmed in float64.
template <int NI, int J, bool NB, bool MD>
__device__ __forceinline__ void pp_tile_f2(const ForceArgs &A, const ulonglong2 (*sQ)[kJ / 2],
                                           const unsigned *sI, int s, int npairs, int cnt, const ChgF &C,
                                           const f2x (&OX)[NI], const f2x (&OY)[NI], const f2x (&OZ)[NI],
                                           const float (&invs_t)[NI], const unsigned (&pid)[NI],
                                           const bool (&valid)[NI], int nvalid, double rout2, double rout,
                                           f2x (&PA)[NI][4], float (&pa)[NI][4], unsigned &n_full,
                                           unsigned &n_fast) {
#pragma unroll kUnrollPP
    for (int P = s; P < npairs; P += J) {
        const ulonglong2 q0 = sQ[0][P], q1 = sQ[1][P];
        // list positions of the two entries (for the padding test)
        const int ea = (P / J) * 2 * J + (P % J), eb = ea + J;
        f2x dx[NI], dy[NI], dz[NI];
        float2 r2[NI];
        bool near = false;
#pragma unroll
        for (int k = 0; k < NI; k++) {
            dx[k] = sub2(q0.x, OX[k]);
            dy[k] = sub2(q0.y, OY[k]);
            dz[k] = sub2(q1.x, OZ[k]);
            r2[k] = up2(fma2(dz[k], dz[k], fma2(dy[k], dy[k], mul2(dx[k], dx[k]))));
            float qa = r2[k].x, qb = r2[k].y;
            if (MD) {
                const float2 w = up2(sQ[2][P].x);
                const float ia = fminf(invs_t[k], w.x), ib = fminf(invs_t[k], w.y);
                qa *= ia * ia;
                qb *= ib * ib;
            }
            near |= (qa < C.rout2m) | (qb < C.rout2m);
        }
        const unsigned real = (ea < cnt ? (unsigned)nvalid : 0u) + (eb < cnt ? (unsigned)nvalid : 0u);
        if (__any_sync(0xffffffffu, near)) {
            n_full += real;
            const unsigned pa_id = sI[2 * P], pb_id = sI[2 * P + 1];
            const float4 far = make_float4(1e15f, 1e15f, 1e15f, 0.0f), far_l = make_float4(0.0f, 0.0f, 0.0f, 1.0f);
            const float4 Ha = ea < cnt ? A.spH[pa_id] : far, La = ea < cnt ? A.spL[pa_id] : far_l;
            const float4 Hb = eb < cnt ? A.spH[pb_id] : far, Lb = eb < cnt ? A.spL[pb_id] : far_l;
#pragma unroll
            for (int k = 0; k < NI; k++) {
                const float4 Hi = A.spH[pid[k]], Li = A.spL[pid[k]];
                pp_changeover_f<NI, NB, MD>(A, Ha, La, pa_id, ea < cnt, C, k, Hi.x, Hi.y, Hi.z, Li.x, Li.y,
                                            Li.z, invs_t[k], pid[k], valid[k], rout2, rout, pa);
                pp_changeover_f<NI, NB, MD>(A, Hb, Lb, pb_id, eb < cnt, C, k, Hi.x, Hi.y, Hi.z, Li.x, Li.y,
                                            Li.z, invs_t[k], pid[k], valid[k], rout2, rout, pa);
            }
        } else {
            n_fast += real;
#pragma unroll
            for (int k = 0; k < NI; k++) {
                const f2x rinv = pk2(rsqrtf(r2[k].x), rsqrtf(r2[k].y));
                const f2x mr = mul2(q1.y, rinv);
                const f2x mr3 = mul2(mr, mul2(rinv, rinv));
                PA[k][0] = fma2(mr3, dx[k], PA[k][0]);
                PA[k][1] = fma2(mr3, dy[k], PA[k][1]);
                PA[k][2] = fma2(mr3, dz[k], PA[k][2]);
                PA[k][3] = add2(PA[k][3], mr);
            }
        }
    }
}

// Far PP entries (the walk guarantees every pair at least r_out apart, so
// K = W = 0): plain Newtonian pairs, two list entries per f32x2 operation,
// with no per-iteration test; unrolled four times (the loop is short enough
// to keep four iterations in flight: 12.20 -> 11.86 ms for the kernel at
// N = 2^20; two, eight: slower).
template <int NI, int J>
__device__ __forceinline__ void pp_tile_far(const ulonglong2 (*sQ)[kJ / 2], int s, int npairs,
                                            const f2x (&OX)[NI], const f2x (&OY)[NI],
                                            const f2x (&OZ)[NI], f2x (&PA)[NI][4]) {
#pragma unroll kUnrollFar
    for (int P = s; P < npairs; P += J) {
        const ulonglong2 q0 = sQ[0][P], q1 = sQ[1][P];
#pragma unroll
        for (int k = 0; k < NI; k++) {
            const f2x dx = sub2(q0.x, OX[k]), dy = sub2(q0.y, OY[k]), dz = sub2(q1.x, OZ[k]);
            const float2 r2 = up2(fma2(dz, dz, fma2(dy, dy, mul2(dx, dx))));
            const f2x rinv = pk2(rsqrtf(r2.x), rsqrtf(r2.y));
            const f2x mr = mul2(q1.y, rinv);
            const f2x mr3 = mul2(mr, mul2(rinv, rinv));
            PA[k][0] = fma2(mr3, dx, PA[k][0]);
            PA[k][1] = fma2(mr3, dy, PA[k][1]);
            PA[k][2] = fma2(mr3, dz, PA[k][2]);
            PA[k][3] = add2(PA[k][3], mr);
        }
    }
}

// Per-lane float-float accumulators live in shared memory (touched once per
// tile), which keeps their 8 NI registers free for the inner loops.

// Float-float sum of two float-float values (Knuth TwoSum of the high parts,
// low parts added): about 2^-44 relative, all on the FP32 pipe.
__device__ __forceinline__ float2 ff_sum(float2 a, float2 b) {
    const float s = __fadd_rn(a.x, b.x);
    const float bp = __fsub_rn(s, a.x);
    const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bp)), __fsub_rn(b.x, bp));
    const float lo = __fadd_rn(__fadd_rn(a.y, b.y), e);
    const float hi = __fadd_rn(s, lo);
    return make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, s)));
}

template <int NI, int J, int ORDER, bool NB, bool MD>
__device__ void group_pass_f(const ForceArgs &A, unsigned g, const uint2 gr, unsigned i0,
                             const ChgF &C, double rout2, double rout, ulonglong2 (*sP)[5][kJ / 2],
                             unsigned (*sI)[kJ], float2 (*sF)[3][4][32], float2 (*red)[kSlotMax][4]) {
    constexpr int L = 32 / J;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = lane / L, l = lane % L;
    const float4 Hg = A.spH[gr.x], Lg = A.spL[gr.x];
    unsigned pid[NI];
    bool valid[NI];
#pragma unroll
    for (int k = 0; k < NI; k++) {
        const unsigned idx = i0 + l + L * k;
        valid[k] = idx < gr.y;
        pid[k] = gr.x + (valid[k] ? idx : 0u);
    }
    float pa[NI][4];
    float2 (*acc)[4][32] = sF[w];
#pragma unroll
    for (int k = 0; k < NI; k++)
#pragma unroll
        for (int c = 0; c < 4; c++) {
            pa[k][c] = 0.0f;
            acc[k][c][lane] = make_float2(0.0f, 0.0f);
        }
    // ---- cells: float offsets from the group's first particle; the tile is
    // stored in pair layout and evaluated two cells per f32x2 operation
    {
        f2x OX[NI], OY[NI], OZ[NI], PA[NI][4];
#pragma unroll
        for (int k = 0; k < NI; k++) {
            const float4 H = A.spH[pid[k]], L4 = A.spL[pid[k]];
            const float ox = (H.x - Hg.x) + (L4.x - Lg.x);
            const float oy = (H.y - Hg.y) + (L4.y - Lg.y);
            const float oz = (H.z - Hg.z) + (L4.z - Lg.z);
            OX[k] = pk2(ox, ox);
            OY[k] = pk2(oy, oy);
            OZ[k] = pk2(oz, oz);
#pragma unroll
            for (int c = 0; c < 4; c++) PA[k][c] = 0ull;
        }
        const unsigned nc = A.gr_nc[g];
        const unsigned long long co = A.gr_co[g];
        for (unsigned t = w * kJ; t < nc; t += kFWarps * kJ) {
            const int cnt = (int)min((unsigned)kJ, nc - t);
            const int cnt2 = (cnt + 2 * J - 1) / (2 * J) * (2 * J);   // <= kJ: kJ is a multiple of 2J
            // lane -> pairs P = lane, lane + 32, ..: entries a = (P / J) 2J + P mod J and
            // b = a + J; each row of a pair is one 128-bit store
#pragma unroll
            for (int h = 0; h < kJ / 64; h++) {
                const int P = lane + 32 * h;
                if (2 * P < cnt2) {
                    const int ea = (P / J) * 2 * J + (P % J), eb = ea + J;
                    float x[2], y[2], z[2], ms[2], q[2][6];
#pragma unroll
                    for (int u = 0; u < 2; u++) {
                        const int e = u ? eb : ea;
                        x[u] = 1e15f; y[u] = 1e15f; z[u] = 1e15f; ms[u] = 0.0f;   // padding: massless, far away
#pragma unroll
                        for (int c = 0; c < 6; c++) q[u][c] = 0.0f;
                        if (e < cnt) {
                            const unsigned v = A.cells[co + t + e];
                            const float4 f0 = A.nd_f[3 * v], f1 = A.nd_f[3 * v + 1];
                            x[u] = (f0.x - Hg.x) + (f1.x - Lg.x);
                            y[u] = (f0.y - Hg.y) + (f1.y - Lg.y);
                            z[u] = (f0.z - Hg.z) + (f1.z - Lg.z);
                            ms[u] = f0.w;
                            if (ORDER == 2) {
                                // the record holds -Q (so -Q d feeds the acceleration
                                // directly) without its zz element: -Qzz = Qxx + Qyy
                                const float4 f2 = A.nd_f[3 * v + 2];
                                q[u][0] = f1.w; q[u][1] = f2.x; q[u][2] = -(f1.w + f2.x);
                                q[u][3] = f2.y; q[u][4] = f2.z; q[u][5] = f2.w;
                            }
                        }
                    }
                    sP[w][0][P] = make_ulonglong2(pk2(x[0], x[1]), pk2(y[0], y[1]));
                    sP[w][1][P] = make_ulonglong2(pk2(z[0], z[1]), pk2(ms[0], ms[1]));
                    if (ORDER == 2) {        // (Qxx, Qyy), (Qzz, Qxy), (Qxz, Qyz), all negated
                        sP[w][2][P] = make_ulonglong2(pk2(q[0][0], q[1][0]), pk2(q[0][1], q[1][1]));
                        sP[w][3][P] = make_ulonglong2(pk2(q[0][2], q[1][2]), pk2(q[0][3], q[1][3]));
                        sP[w][4][P] = make_ulonglong2(pk2(q[0][4], q[1][4]), pk2(q[0][5], q[1][5]));
                    }
                }
            }
            __syncwarp();
            cells_tile_f2<NI, J, ORDER>(sP[w], s, cnt2 / 2, OX, OY, OZ, PA);
            __syncwarp();
#pragma unroll
            for (int k = 0; k < NI; k++)
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const float2 v = up2(PA[k][c]);
                    float2 a = acc[k][c][lane];
                    ff_add(a.x, a.y, v.x + v.y);
                    acc[k][c][lane] = a;
                    PA[k][c] = 0ull;
                }
        }
    }
    // ---- particle-particle: float-float differences, two list entries per
    // f32x2 operation on the Newtonian path
    {
        f2x OX[NI], OY[NI], OZ[NI], PA[NI][4];
        float invs_t[NI];
#pragma unroll
        for (int k = 0; k < NI; k++) {
            const float4 H = A.spH[pid[k]], L4 = A.spL[pid[k]];
            const float ox = (H.x - Hg.x) + (L4.x - Lg.x);
            const float oy = (H.y - Hg.y) + (L4.y - Lg.y);
            const float oz = (H.z - Hg.z) + (L4.z - Lg.z);
            OX[k] = pk2(ox, ox); OY[k] = pk2(oy, oy); OZ[k] = pk2(oz, oz);
            invs_t[k] = L4.w;                                    // 1 / s_i
#pragma unroll
            for (int c = 0; c < 4; c++) PA[k][c] = 0ull;
        }
        int nvalid = 0;
#pragma unroll
        for (int k = 0; k < NI; k++) nvalid += valid[k] ? 1 : 0;
        unsigned n_full = 0, n_fast = 0;
        const unsigned ntarg = min((unsigned)(NI * L), gr.y - i0);   // targets of this pass
        // the near segment (changeover test per iteration), then the far one
        for (int seg = 0; seg < 2; seg++) {
            const unsigned np = seg == 0 ? A.gr_np[g] : A.gr_nf[g];
            const unsigned long long po = seg == 0 ? A.gr_po[g] : A.gr_fo[g];
            for (unsigned t = w * kJ; t < np; t += kFWarps * kJ) {
                const int cnt = (int)min((unsigned)kJ, np - t);
                const int cnt2 = (cnt + 2 * J - 1) / (2 * J) * (2 * J);   // <= kJ: kJ is a multiple of 2J
#pragma unroll
                for (int h = 0; h < kJ / 64; h++) {
                    const int P = lane + 32 * h;
                    if (2 * P < cnt2) {
                        const int ea = (P / J) * 2 * J + (P % J), eb = ea + J;
                        float ox[2], oy[2], oz[2], ms[2], wj[2];
                        unsigned id[2];
#pragma unroll
                        for (int u = 0; u < 2; u++) {
                            const int e = u ? eb : ea;
                            ox[u] = 1e15f; oy[u] = 1e15f; oz[u] = 1e15f; ms[u] = 0.0f; wj[u] = 1.0f;   // padding
                            id[u] = 0xffffffffu;
                            if (e < cnt) {
                                const unsigned p = A.pp[po + t + e];
                                const float4 H = A.spH[p], L = A.spL[p];
                                ox[u] = (H.x - Hg.x) + (L.x - Lg.x);
                                oy[u] = (H.y - Hg.y) + (L.y - Lg.y);
                                oz[u] = (H.z - Hg.z) + (L.z - Lg.z);
                                ms[u] = H.w;
                                wj[u] = L.w;
                                id[u] = p;
                            }
                        }
                        sP[w][0][P] = make_ulonglong2(pk2(ox[0], ox[1]), pk2(oy[0], oy[1]));
                        sP[w][1][P] = make_ulonglong2(pk2(oz[0], oz[1]), pk2(ms[0], ms[1]));
                        if (MD) sP[w][2][P].x = pk2(wj[0], wj[1]);
                        reinterpret_cast<uint2 *>(sI[w])[P] = make_uint2(id[0], id[1]);
                    }
                }
                __syncwarp();
                if (seg == 1) {
                    pp_tile_far<NI, J>(sP[w], s, cnt2 / 2, OX, OY, OZ, PA);
                    if (lane == 0) n_fast += (unsigned)cnt * ntarg;
                } else if (NB && A.want_nb) {
                    pp_tile_f2<NI, J, true, MD>(A, sP[w], sI[w], s, cnt2 / 2, cnt, C, OX, OY, OZ,
                                                invs_t, pid, valid, nvalid, rout2, rout, PA, pa, n_full, n_fast);
                } else {
                    pp_tile_f2<NI, J, false, MD>(A, sP[w], sI[w], s, cnt2 / 2, cnt, C, OX, OY, OZ,
                                                 invs_t, pid, valid, nvalid, rout2, rout, PA, pa, n_full, n_fast);
                }
                __syncwarp();
#pragma unroll
                for (int k = 0; k < NI; k++)
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        const float2 v = up2(PA[k][c]);
                        float2 a = acc[k][c][lane];
                        ff_add(a.x, a.y, (v.x + v.y) + pa[k][c]);
                        acc[k][c][lane] = a;
                        PA[k][c] = 0ull;
                        pa[k][c] = 0.0f;
                    }
            }
        }
        n_full = warp_sum(n_full);
        n_fast = warp_sum(n_fast);
        if (lane == 0 && (n_full | n_fast)) {
            atomicAdd(&A.st->pp_full, (unsigned long long)n_full);
            atomicAdd(&A.st->pp_fast, (unsigned long long)n_fast);
        }
    }
    // ---- sum the J sub-streams of each target (float-float, fixed order),
    // then hand over to the block
#pragma unroll
    for (int k = 0; k < NI; k++)
#pragma unroll
        for (int c = 0; c < 4; c++) {
            float2 v = acc[k][c][lane];
#pragma unroll
            for (int o = L; o < 32; o <<= 1) {
                const float2 u = make_float2(__shfl_xor_sync(0xffffffffu, v.x, o),
                                             __shfl_xor_sync(0xffffffffu, v.y, o));
                v = (lane & o) ? ff_sum(u, v) : ff_sum(v, u);   // the same order on both lanes
            }
            if (s == 0) red[w][l + L * k][c] = v;
        }
}

// Final per-target sums of the mixed kernel (threads 0..slots-1): the warps'
// float-float partials added in a fixed order, converted to float64 once;
// removal of the self entry, output in caller order.
__device__ __forceinline__ void write_targets_ff(const ForceArgs &A, const uint2 gr, unsigned i0,
                                                 unsigned slots, double c2, float2 (*red)[kSlotMax][4],
                                                 double (&ep)[4]) {
    const unsigned t = threadIdx.x;
    if (t < slots && i0 + t < gr.y) {
        double s[4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            float2 v = red[0][t][c];
            for (int w = 1; w < kFWarps; w++) v = ff_sum(v, red[w][t][c]);
            s[c] = (double)v.x + (double)v.y;
        }
        const unsigned p = gr.x + i0 + t;
        const double m = A.sp64[p].w;
        const double P = s[3] - (A.massdep ? m * c2 / A.ssc[p] : m * c2);
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

// Final per-target sums of the float64 kernel (threads 0..slots-1): fixed-order
// float64 reduction over the warps, removal of the self entry, output in caller order.
__device__ __forceinline__ void write_targets(const ForceArgs &A, const uint2 gr, unsigned i0,
                                              unsigned slots, double c2, double (*red)[kSlotMax][4],
                                              double (&ep)[4]) {
    const unsigned t = threadIdx.x;
    if (t < slots && i0 + t < gr.y) {
        double s[4] = {0, 0, 0, 0};
        for (int w = 0; w < kFWarps; w++)
            for (int c = 0; c < 4; c++) s[c] += red[w][t][c];
        const unsigned p = gr.x + i0 + t;
        const double m = A.sp64[p].w;
        // remove the self entry m_i 2 / (s_i (r_out + r_in))
        const double P = s[3] - (A.massdep ? m * c2 / A.ssc[p] : m * c2);
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
    const int w = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 4; c++) ep[c] = warp_sum(ep[c]);
    if ((threadIdx.x & 31) == 0)
        for (int c = 0; c < 4; c++) ered[w][c] = ep[c];
    __syncthreads();
    if (threadIdx.x == 0) {
        double e[4] = {0, 0, 0, 0};
        for (int k = 0; k < kFWarps; k++)
            for (int c = 0; c < 4; c++) e[c] += ered[k][c];
        A.gpart[g] = make_double4(e[0], e[1], e[2], e[3]);
    }
}

// Configuration class of a group's first pass (0: more than 64 targets, more
// than one pass or the 96-slot one; then 64, 48, 32, 24 and 16 slots), in the
// order the mixed kernel takes the groups.
__device__ __forceinline__ int pass_class(unsigned n) {
    return n > 64 ? 0 : n > 48 ? 1 : n > 32 ? 2 : n > 24 ? 3 : n > 16 ? 4 : 5;
}
constexpr int kPassClasses = 6;

// Pass configuration for `rem` remaining targets: returns the slot count and
// runs the matching instantiation.
template <int ORDER, bool NB, bool MD>
__device__ unsigned mixed_pass(const ForceArgs &A, unsigned g, const uint2 gr, unsigned i0,
                               const ChgF &C, double rout2, double rout, ulonglong2 (*sP)[5][kJ / 2],
                               unsigned (*sI)[kJ], float2 (*sF)[3][4][32], float2 (*red)[kSlotMax][4]) {
    const unsigned rem = gr.y - i0;
    if (rem <= 16) { group_pass_f<2, 4, ORDER, NB, MD>(A, g, gr, i0, C, rout2, rout, sP, sI, sF, red); return 16; }
    if (rem <= 24) { group_pass_f<3, 4, ORDER, NB, MD>(A, g, gr, i0, C, rout2, rout, sP, sI, sF, red); return 24; }
    if (rem <= 32) { group_pass_f<2, 2, ORDER, NB, MD>(A, g, gr, i0, C, rout2, rout, sP, sI, sF, red); return 32; }
    if (rem <= 48) { group_pass_f<3, 2, ORDER, NB, MD>(A, g, gr, i0, C, rout2, rout, sP, sI, sF, red); return 48; }
    if (rem <= 64) { group_pass_f<2, 1, ORDER, NB, MD>(A, g, gr, i0, C, rout2, rout, sP, sI, sF, red); return 64; }
    group_pass_f<3, 1, ORDER, NB, MD>(A, g, gr, i0, C, rout2, rout, sP, sI, sF, red);
    return 96;
}

template <int ORDER, bool NB, bool MD, bool TAIL>
__global__ void __launch_bounds__(kFThreads, PT_FORCE_MIN_BLOCKS) k_force_mixed(ForceArgs A) {
    __shared__ ulonglong2 sP[kFWarps][5][kJ / 2];
    __shared__ float2 sF[kFWarps][3][4][32];
    __shared__ unsigned sI[kFWarps][kJ];
    __shared__ float2 red[kFWarps][kSlotMax][4];
    __shared__ double ered[kFWarps][4];
    __shared__ unsigned gsh;
    // the group's changeover constants, formed once per group by thread 0
    // (float64 divisions and a square root: slow on this part's FP64 pipe)
    __shared__ ChgF sC;
    __shared__ double sRout2, sRout, sC2;
    // lists left unusable by the walk (one-pass arrays exhausted, stack
    // overflow): do nothing, the host re-runs the walk and the force
    if (A.st->flags & (kErrListCap | kErrStack)) return;
    const unsigned ng = A.st->ngroups;
    for (unsigned it = 0;; it++) {
        unsigned gi;
        if constexpr (!TAIL) {
            if (A.direct_groups) {               // one group per CTA, in group order
                if (it > 0 || blockIdx.x >= ng) break;
                gi = blockIdx.x;
            } else {                             // persistent CTAs
                __syncthreads();
                if (threadIdx.x == 0) gsh = (unsigned)atomicAdd(&A.st->work[2], 1ull);
                __syncthreads();
                gi = gsh;
                if (gi >= ng) break;
            }
        } else {
            // the CTA's own group first, then the groups beyond a grid sized
            // from a count hint (a separate instantiation: the loop that may
            // run again compiled the single-set kernel 2.4% slower)
            if (it == 0 && A.direct_groups && blockIdx.x < ng) {
                gi = blockIdx.x;
            } else {
                if (A.direct_groups >= ng) break;
                __syncthreads();
                if (threadIdx.x == 0) gsh = A.direct_groups + (unsigned)atomicAdd(&A.st->work[2], 1ull);
                __syncthreads();
                gi = gsh;
                if (gi >= ng) break;
            }
        }
        const unsigned g = A.gr_ord[gi];
        const uint2 gr = A.gr_r[g];
        if (threadIdx.x == 0) {
            const Chg C64 = make_chg(A.sets[A.gr_a[g].w]);
            ChgF C;
            C.invw = (float)C64.invw;
            C.c0 = (float)C64.c0;
            C.c2 = (float)C64.c2;
            C.k0 = (float)(70.0 * C64.ri / (C64.ro + C64.ri));   // 35 (1 - Lambda), no cancellation
            C.w0 = (float)(14.0 * C64.lam);
            C.w1 = (float)(-28.0 * C64.lam);
            C.w2 = (float)(20.0 * C64.lam);
            C.w3 = (float)(-5.0 * C64.lam);
            C.tiny = fmaxf((float)C64.tiny, 1e-36f);
            C.rout2m = vote_rout2(A.gr_a[g], A.gr_b[g], A.sets[A.gr_a[g].w]);
            sC = C;
            sRout2 = C64.rout2;
            sRout = C64.ro;
            sC2 = C64.c2;
        }
        __syncthreads();
        const ChgF C = sC;
        const double rout2 = sRout2, rout = sRout, c2 = sC2;
        double ep[4] = {0, 0, 0, 0};
        for (unsigned i0 = 0; i0 < gr.y;) {
            const unsigned slots = mixed_pass<ORDER, NB, MD>(A, g, gr, i0, C, rout2, rout, sP, sI, sF, red);
            __syncthreads();
            write_targets_ff(A, gr, i0, slots, c2, red, ep);
            __syncthreads();
            i0 += slots;
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

template <int NI, bool NB, bool MD>
__device__ __forceinline__ void pp_tile_d(const ForceArgs &A, const double4 *sP, const unsigned *sI,
                                          const double *sS, int cnt, const Chg &C,
                                          const double (&xx)[2], const double (&xy)[2],
                                          const double (&xz)[2], const double (&st)[2],
                                          const unsigned (&pid)[2], const bool (&valid)[2],
                                          double (&pa)[2][4]) {
    for (int j = 0; j < cnt; j++) {
        const double4 P = sP[j];
#pragma unroll
        for (int s = 0; s < NI; s++) {
            const double dx = __dsub_rn(P.x, xx[s]), dy = __dsub_rn(P.y, xy[s]), dz = __dsub_rn(P.z, xz[s]);
            const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            double rout2 = C.rout2, sij = 1.0;
            if (MD) {                       // pair radii s_ij (r_in, r_out), s_ij = max(s_i, s_j)
                sij = fmax(st[s], sS[j]);
                const double ro = __dmul_rn(C.ro, sij);
                rout2 = __dmul_rn(ro, ro);
            }
            if (NB && r2 < rout2) {
                const unsigned pj = sI[j];
                if (valid[s] && pj != pid[s]) emit_pair(A, pid[s], pj);
            }
            const double r2c = fmax(r2, C.tiny);
            const double rinv = rsqrt(r2c);
            const double r = MD ? (r2c * rinv) / sij : r2c * rinv;     // r / s_ij
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

// Far PP entries in float64 (every pair at least r_out apart: K = W = 0):
// plain Newtonian pairs.
template <int NI>
__device__ __forceinline__ void pp_tile_d_far(const double4 *sP, int cnt, const double (&xx)[2],
                                              const double (&xy)[2], const double (&xz)[2],
                                              double (&pa)[2][4]) {
    for (int j = 0; j < cnt; j++) {
        const double4 P = sP[j];
#pragma unroll
        for (int s = 0; s < NI; s++) {
            const double dx = P.x - xx[s], dy = P.y - xy[s], dz = P.z - xz[s];
            const double rinv = rsqrt(fma(dz, dz, fma(dy, dy, dx * dx)));
            const double mr = P.w * rinv;
            const double fk = mr * (rinv * rinv);
            pa[s][0] = fma(fk, dx, pa[s][0]);
            pa[s][1] = fma(fk, dy, pa[s][1]);
            pa[s][2] = fma(fk, dz, pa[s][2]);
            pa[s][3] += mr;
        }
    }
}

template <int NI, int ORDER, bool NB, bool MD>
__device__ void group_pass_d(const ForceArgs &A, unsigned g, const uint2 gr, unsigned i0,
                             const Chg &C, double4 (*sA)[kJD], double4 (*sB)[kJD],
                             double2 (*sC)[kJD], unsigned (*sI)[kJD], double (*sS)[kJD],
                             double (*red)[kSlotMax][4]) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double xx[2], xy[2], xz[2], st[2];
    unsigned pid[2];
    bool valid[2];
#pragma unroll
    for (int s = 0; s < 2; s++) {
        const unsigned idx = i0 + lane + 32 * s;
        valid[s] = idx < gr.y;
        pid[s] = gr.x + (valid[s] ? idx : 0u);
        const double4 P = A.sp64[pid[s]];
        xx[s] = P.x; xy[s] = P.y; xz[s] = P.z;
        st[s] = MD ? A.ssc[pid[s]] : 1.0;
    }
    double pa[2][4];
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int c = 0; c < 4; c++) pa[s][c] = 0.0;
    const unsigned nc = A.gr_nc[g];
    const unsigned long long co = A.gr_co[g];
    for (unsigned t = w * kJD; t < nc; t += kFWarps * kJD) {
        const int cnt = (int)min((unsigned)kJD, nc - t);
#pragma unroll
        for (int h = 0; h < kJD / 32; h++) {
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
    // near PP segment (changeover and neighbour test per pair), then the far
    // one (plain Newtonian pairs)
    for (int seg = 0; seg < 2; seg++) {
        const unsigned np = seg == 0 ? A.gr_np[g] : A.gr_nf[g];
        const unsigned long long po = seg == 0 ? A.gr_po[g] : A.gr_fo[g];
        for (unsigned t = w * kJD; t < np; t += kFWarps * kJD) {
            const int cnt = (int)min((unsigned)kJD, np - t);
#pragma unroll
            for (int h = 0; h < kJD / 32; h++) {
                const int e = lane + 32 * h;
                if (e < cnt) {
                    const unsigned p = A.pp[po + t + e];
                    sA[w][e] = A.sp64[p];
                    sI[w][e] = p;
                    if (MD) sS[w][e] = A.ssc[p];
                }
            }
            __syncwarp();
            if (seg == 1)
                pp_tile_d_far<NI>(sA[w], cnt, xx, xy, xz, pa);
            else if (NB && A.want_nb)
                pp_tile_d<NI, true, MD>(A, sA[w], sI[w], sS[w], cnt, C, xx, xy, xz, st, pid, valid, pa);
            else
                pp_tile_d<NI, false, MD>(A, sA[w], sI[w], sS[w], cnt, C, xx, xy, xz, st, pid, valid, pa);
            __syncwarp();
        }
    }
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int c = 0; c < 4; c++) red[w][lane + 32 * s][c] = (s < NI) ? pa[s][c] : 0.0;
}

template <int ORDER, bool NB, bool MD, bool TAIL>
__global__ void __launch_bounds__(kFThreads) k_force_fp64(ForceArgs A) {
    __shared__ double4 sA[kFWarps][kJD];
    __shared__ double4 sB[kFWarps][kJD];
    __shared__ double2 sC[kFWarps][kJD];
    __shared__ unsigned sI[kFWarps][kJD];
    __shared__ double sS[kFWarps][MD ? kJD : 1];
    __shared__ double red[kFWarps][kSlotMax][4];
    __shared__ double ered[kFWarps][4];
    __shared__ unsigned gsh;
    // lists left unusable by the walk (one-pass arrays exhausted, stack
    // overflow): do nothing, the host re-runs the walk and the force
    if (A.st->flags & (kErrListCap | kErrStack)) return;
    const unsigned ng = A.st->ngroups;
    for (unsigned it = 0;; it++) {
        unsigned g;
        if constexpr (!TAIL) {
            if (A.direct_groups) {               // one group per CTA
                if (it > 0 || blockIdx.x >= ng) break;
                g = blockIdx.x;
            } else {
                __syncthreads();
                if (threadIdx.x == 0) gsh = (unsigned)atomicAdd(&A.st->work[2], 1ull);
                __syncthreads();
                g = gsh;
                if (g >= ng) break;
            }
        } else {                                 // see the mixed kernel
            if (it == 0 && A.direct_groups && blockIdx.x < ng) {
                g = blockIdx.x;
            } else {
                if (A.direct_groups >= ng) break;
                __syncthreads();
                if (threadIdx.x == 0) gsh = A.direct_groups + (unsigned)atomicAdd(&A.st->work[2], 1ull);
                __syncthreads();
                g = gsh;
                if (g >= ng) break;
            }
        }
        const uint2 gr = A.gr_r[g];
        const Chg C = make_chg(A.sets[A.gr_a[g].w]);
        double ep[4] = {0, 0, 0, 0};
        for (unsigned i0 = 0; i0 < gr.y; i0 += kIB) {
            if (gr.y - i0 > 32)
                group_pass_d<2, ORDER, NB, MD>(A, g, gr, i0, C, sA, sB, sC, sI, (double (*)[kJD])sS, red);
            else
                group_pass_d<1, ORDER, NB, MD>(A, g, gr, i0, C, sA, sB, sC, sI, (double (*)[kJD])sS, red);
            __syncthreads();
            write_targets(A, gr, i0, kIB, C.c2, red, ep);
            __syncthreads();
        }
        group_partials(A, g, ep, ered);
    }
}

// ===========================================================================
// Totals over groups (fixed-order reduction, one block)
// ===========================================================================

// Energy / momentum sums and interaction counts over the groups, in two
// launches with a fixed reduction order (the same sums every run on a given
// device): each of nb = min(SMs, kRedBlocksMax) blocks reduces a contiguous
// range of groups, then one warp adds the blocks' partials in block order.
constexpr int kRedThreads = 256;

__global__ void __launch_bounds__(kRedThreads) k_force_partials(const double4 *gpart, const uint2 *gr_r,
                                                                const unsigned *gr_nc, const unsigned *gr_np,
                                                                const unsigned *gr_nf, double4 *red_e,
                                                                unsigned long long *red_c, const Status *st) {
    __shared__ double se[kRedThreads / 32][4];
    __shared__ unsigned long long si[kRedThreads / 32][2];
    const unsigned ng = st->ngroups, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned per = (ng + gridDim.x - 1) / gridDim.x;
    const unsigned b = min(blockIdx.x * per, ng), e = min(b + per, ng);
    double acc[4] = {0, 0, 0, 0};
    unsigned long long ci = 0, pi = 0;
    for (unsigned g = b + threadIdx.x; g < e; g += blockDim.x) {
        const double4 p = gpart[g];
        acc[0] += p.x; acc[1] += p.y; acc[2] += p.z; acc[3] += p.w;
        const unsigned long long n = gr_r[g].y;
        ci += n * gr_nc[g];
        pi += n * (gr_np[g] + gr_nf[g]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int c = 0; c < 4; c++) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
        ci += __shfl_xor_sync(0xffffffffu, ci, o);
        pi += __shfl_xor_sync(0xffffffffu, pi, o);
    }
    if (lane == 0) {
        for (int c = 0; c < 4; c++) se[w][c] = acc[c];
        si[w][0] = ci;
        si[w][1] = pi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[4] = {0, 0, 0, 0};
        unsigned long long tc = 0, tp = 0;
        for (int k = 0; k < kRedThreads / 32; k++) {
            for (int c = 0; c < 4; c++) t[c] += se[k][c];
            tc += si[k][0];
            tp += si[k][1];
        }
        red_e[blockIdx.x] = make_double4(t[0], t[1], t[2], t[3]);
        red_c[2 * blockIdx.x] = tc;
        red_c[2 * blockIdx.x + 1] = tp;
    }
}

__global__ void __launch_bounds__(32) k_force_reduce(const double4 *red_e, const unsigned long long *red_c,
                                                     int nb, Status *st) {
    const unsigned lane = threadIdx.x;
    double acc[4] = {0, 0, 0, 0};
    unsigned long long ci = 0, pi = 0;
    for (int b = lane; b < nb; b += 32) {
        const double4 p = red_e[b];
        acc[0] += p.x; acc[1] += p.y; acc[2] += p.z; acc[3] += p.w;
        ci += red_c[2 * b];
        pi += red_c[2 * b + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int c = 0; c < 4; c++) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
        ci += __shfl_xor_sync(0xffffffffu, ci, o);
        pi += __shfl_xor_sync(0xffffffffu, pi, o);
    }
    if (lane == 0) {
        st->energy = acc[0];
        st->mom[0] = acc[1];
        st->mom[1] = acc[2];
        st->mom[2] = acc[3];
        st->cell_inter = ci;
        st->pp_inter = pi;
    }
}

// Order in which the mixed kernel takes the groups: class by class (largest
// pass configuration first), group order within a class.  Consecutive groups
// then run the same instantiation, which keeps one code path in the SMs'
// instruction caches, and the largest groups start first, which shortens the
// tail of the atomic work queue.  One CTA: thread t classifies a contiguous
// chunk of groups, a block-wide exclusive scan per class gives each chunk its
// output positions, and a second pass over the chunk writes them (stable).
__global__ void __launch_bounds__(1024) k_group_order(const uint2 *gr_r, unsigned *gr_ord,
                                                      const Status *st) {
    __shared__ unsigned wsum[32][kPassClasses];
    __shared__ unsigned base[kPassClasses];
    const unsigned ng = st->ngroups;
    const unsigned t = threadIdx.x, lane = t & 31, w = t >> 5;
    const unsigned per = (ng + 1023) / 1024;
    const unsigned b = min(t * per, ng), e = min(b + per, ng);
    unsigned c[kPassClasses], x[kPassClasses];
#pragma unroll
    for (int k = 0; k < kPassClasses; k++) c[k] = 0;
#pragma unroll 4
    for (unsigned g = b; g < e; g++) {
        const int k = pass_class(gr_r[g].y);
#pragma unroll
        for (int j = 0; j < kPassClasses; j++) c[j] += j == k ? 1u : 0u;   // stays in registers
    }
#pragma unroll
    for (int k = 0; k < kPassClasses; k++) {       // inclusive scan within the warp
        unsigned v = c[k];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned u = __shfl_up_sync(0xffffffffu, v, d);
            if (lane >= (unsigned)d) v += u;
        }
        x[k] = v;
        if (lane == 31) wsum[w][k] = v;
    }
    __syncthreads();
    if (w == 0) {                                   // inclusive scan over the warps
        unsigned v[kPassClasses];
#pragma unroll
        for (int k = 0; k < kPassClasses; k++) v[k] = wsum[lane][k];
#pragma unroll
        for (int k = 0; k < kPassClasses; k++) {
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned u = __shfl_up_sync(0xffffffffu, v[k], d);
                if (lane >= (unsigned)d) v[k] += u;
            }
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < kPassClasses; k++) wsum[lane][k] = v[k];
    }
    __syncthreads();
    if (t == 0) {
        unsigned sum = 0;
        for (int k = 0; k < kPassClasses; k++) {
            base[k] = sum;
            sum += wsum[31][k];
        }
    }
    __syncthreads();
    unsigned o[kPassClasses];
#pragma unroll
    for (int k = 0; k < kPassClasses; k++) o[k] = base[k] + (w ? wsum[w - 1][k] : 0u) + x[k] - c[k];
    for (unsigned g = b; g < e; g++) {
        const int k = pass_class(gr_r[g].y);
        unsigned pos = 0;
#pragma unroll
        for (int j = 0; j < kPassClasses; j++)      // register-indexed: no local-memory array
            if (j == k) pos = o[j]++;
        gr_ord[pos] = g;
    }
}

// One CTA per group when the host knows the group count (CTAs then retire
// group by group, so kernels of other streams -- other batches of a server --
// get SMs within a group's time instead of waiting for the whole launch),
// else a persistent grid that takes groups from an atomic counter.
template <bool TAIL>
static void force_launch_t(const ForceArgs &A, int precision, int blocks, cudaStream_t st) {
    const bool md = A.massdep != 0;
    if (precision == 1) {
        if (A.order == 2) {
            if (md) k_force_mixed<2, true, true, TAIL><<<blocks, kFThreads, 0, st>>>(A);
            else k_force_mixed<2, true, false, TAIL><<<blocks, kFThreads, 0, st>>>(A);
        } else {
            if (md) k_force_mixed<0, true, true, TAIL><<<blocks, kFThreads, 0, st>>>(A);
            else k_force_mixed<0, true, false, TAIL><<<blocks, kFThreads, 0, st>>>(A);
        }
    } else {
        if (A.order == 2) {
            if (md) k_force_fp64<2, true, true, TAIL><<<blocks, kFThreads, 0, st>>>(A);
            else k_force_fp64<2, true, false, TAIL><<<blocks, kFThreads, 0, st>>>(A);
        } else {
            if (md) k_force_fp64<0, true, true, TAIL><<<blocks, kFThreads, 0, st>>>(A);
            else k_force_fp64<0, true, false, TAIL><<<blocks, kFThreads, 0, st>>>(A);
        }
    }
}

int force_launch(const ForceArgs &A, int precision, cudaStream_t st) {
    const int blocks = A.direct_groups ? (int)A.direct_groups : sm_count() * 8;
    if (precision == 1) k_group_order<<<1, 1024, 0, st>>>(A.gr_r, A.gr_ord, A.st);
    if (A.count_hint && A.direct_groups) force_launch_t<true>(A, precision, blocks, st);
    else force_launch_t<false>(A, precision, blocks, st);
    return precision == 1 ? 2 : 1;
}

int force_reduce_launch(const ForceArgs &A, cudaStream_t st) {
    const int nb = std::min(sm_count(), kRedBlocksMax);
    k_force_partials<<<nb, kRedThreads, 0, st>>>(A.gpart, A.gr_r, A.gr_nc, A.gr_np, A.gr_nf, A.red_e,
                                                 A.red_c, A.st);
    k_force_reduce<<<1, 32, 0, st>>>(A.red_e, A.red_c, nb, A.st);
    return 2;
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
    k_nb_keys<<<sm_count() * 4, 256, 0, st>>>(A);
    int nk = radix_sort(A.keys, A.vals, A.keys_sorted, A.vals_sorted, A.npairs_dev,
                        (unsigned)A.pair_cap, 0, A.key_bits, nullptr, 0, A.sort_tmp, st);
    k_nb_csr<<<sm_count() * 4, 256, 0, st>>>(A);
    return nk + 2;
}

}  // namespace pt
