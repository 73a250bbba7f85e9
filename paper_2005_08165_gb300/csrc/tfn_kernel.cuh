// tfn_kernel.cuh -- the fused Three-Filters-to-Normal kernel for sm_103a.
//
// A persistent kernel of independent warps.  A work item is a band of 128
// pixel columns x TH rows of one frame; warp w takes items w, w + W, ... of a
// queue spanning every frame of the launch.  A lane owns 4 adjacent columns
// and rolls down the item's rows keeping three sample rows (above, at, below)
// in registers, so the edges between two rows are computed once for both.
// The rows reach shared memory through a per-warp ring of TMA 2D copies
// (boxes of CR rows x 128 columns plus a 16-byte halo each side, one mbarrier
// per stage); normals and mask leave through vectorised streaming stores.
// Holes decode to 2^100 (see kHole), and the TMA zero fill outside the image
// (rows above the first and past the last, columns beyond the edges) is a
// hole, so borders need no special case.
//
// Arithmetic (Sec. III of Fan et al.):
//   filters          FD on depth: G = 1/Z_{+1} - 1/Z_{-1} = (Z_{-1} - Z_{+1}) /
//                    (Z_{-1} Z_{+1}) in one pass; Sobel, Scharr, Prewitt:
//                    G = sum_k c_k (w_{k,+1} - w_{k,-1}) with w = 1/Z per sample
//                    as wh + wl (hardware reciprocal plus its FMA residual) and
//                    exact tap differences (Knuth's TwoSum); normalisation
//                    dropped (the normal's direction is homogeneous in
//                    (G_u, G_v)); disparity: the same on d (Eq. nx2_ny2_nz3);
//   candidates       c_j = A + R_j, A = (u-u0) G_u + (v-v0) G_v,
//                    R_j = (du G_u + dv G_v) rho_j, rho_j = Z_j / (Z_j - Z_i)
//                    (Eq. nx2_ny2_nz2 with the back-projection of Eq. intrinsic
//                    substituted: fx and fy cancel); disparity: rho_j =
//                    d_i / (d_i - d_j).  1/(Z_j - Z_i) is computed once per
//                    edge of the pixel grid and shared by its two end pixels;
//   Phi              mean over the kept candidates, or the median through a
//                    19-comparator network over the 8 slots, empty slots filled
//                    alternately with +inf / -inf so the median sits at sorted
//                    position 3 (odd count) or 3 and 4 (even count);
//   output           n = -n'/|n'|, n' = (fx G_u, fy G_v, -(A + Phi)).
//
// Accuracy: each candidate carries a few units of FP32 rounding relative to
// itself, and each gradient a known relative error.  What remains is
// cancellation inside the candidate sum (mean) or between the two middle
// candidates (even median), and the effect of the gradient error; each pixel
// bounds both, and the rare pixels whose bound exceeds the threshold are
// redone in double-float arithmetic (refine_pixel): by the main kernel itself
// for the FD mean (a per-warp queue, 32 pixels at a time) and for the short
// items of small launches (at the end of each item), otherwise by
// refine_kernel after the main kernel, from a list.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tfn_internal.h"
#include "tfn_items.h"

namespace tfn {
namespace dev {

constexpr float kValidLo = 1.52587890625e-05f;  // 2^-16
constexpr float kValidHi = 65536.0f;            // 2^16
constexpr long long kWaitCycles = 4000000000LL;    // ~2 s at 2 GHz
constexpr long long kDrainCycles = 2000000LL;      // ~1 ms: the drain after a failed wait
constexpr long long kTestWaitCycles = 2000000LL;   // ~1 ms: the wait of TFN_FLAG_TEST_WAIT_TIMEOUT

// ---------------------------------------------------------------- numerics

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

struct df {  // unevaluated sum h + l
    float h, l;
};

// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ df two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// Dekker's Fast2Sum, valid when |a| >= |b| or a == 0.
__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// Error-free product through FMA: p + e == a * b exactly.
__device__ __forceinline__ df two_prod(float a, float b)
{
    float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df df_neg(df a) { return {-a.h, -a.l}; }

__device__ __forceinline__ df df_add(df a, df b)
{
    df s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ df df_mul_f(df a, float b)
{
    df p = two_prod(a.h, b);
    return fast_two_sum(p.h, __fmaf_rn(a.l, b, p.l));
}

__device__ __forceinline__ df df_mul(df a, df b)
{
    df p = two_prod(a.h, b.h);
    return fast_two_sum(p.h, __fadd_rn(p.l, __fmaf_rn(a.h, b.l, __fmul_rn(a.l, b.h))));
}

// Long division in double-float (Dekker's): q1 = a_h / b_h from the
// hardware reciprocal (within about 2u), the residual a - b q1 in
// double-float (nearly exact), and its quotient as the correction; h + l is
// then within a few u^2 of a / b, relative, for operands and residuals in
// the normal range.  No branch: the refinement's eight quotients can overlap.
__device__ __forceinline__ df df_div(df a, df b)
{
    const float rb = rcp_approx(b.h);
    const float q1 = __fmul_rn(a.h, rb);
    const df r = df_add(a, df_neg(df_mul_f(b, q1)));
    const float q2 = __fmul_rn(r.h, rb);
    return fast_two_sum(q1, q2);
}

// Unnormalised double-float for the long weighted sums of the 5x5 filters:
// the high parts are added exactly (TwoSum) or multiplied exactly (FMA
// residual), the low parts and those errors are accumulated in FP32, and the
// pair is not renormalised after each step (8 and 3 operations instead of 11
// and 6).  h + l keeps the terms' sum to about u^2 of their magnitudes, as
// the normalised operations do; df_norm renormalises (exactly) at the end.
__device__ __forceinline__ df dfl_add(df a, df b)
{
    const df s = two_sum(a.h, b.h);
    return {s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l))};
}
__device__ __forceinline__ df dfl_sub(df a, df b) { return dfl_add(a, df_neg(b)); }
__device__ __forceinline__ df dfl_mul_f(df a, float b)
{
    const float p = __fmul_rn(a.h, b);
    return {p, __fmaf_rn(a.l, b, __fmaf_rn(a.h, b, -p))};
}
__device__ __forceinline__ df df_norm(df a) { return two_sum(a.h, a.l); }

__device__ __forceinline__ float df_val(df a) { return __fadd_rn(a.h, a.l); }

// ------------------------------------------------------------ pixel pairs
//
// The 3x3 kernels write a lane's four pixels as two pairs (see row_step2).
// An f2 holds one value of each pixel of a pair, and these helpers apply the
// same correctly rounded operation to both: two scalar operations each,
// never contracted or reassociated, so a pair computes exactly what two
// scalar pixels would.
typedef float2 f2;

__device__ __forceinline__ f2 pk(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ f2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float lane_of(f2 a, int l) { return l == 0 ? a.x : a.y; }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return pk(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return pk(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y)); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return pk(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return pk(__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y)); }
__device__ __forceinline__ f2 neg2(f2 a) { return pk(-a.x, -a.y); }
__device__ __forceinline__ f2 rcp2(f2 a) { return pk(rcp_approx(a.x), rcp_approx(a.y)); }

// w_b - w_a for depths a, b > 0, i.e. (a - b) / (a b), as h + l with error
// ~u^2: exact difference (TwoSum), exact product (FMA), and the division
// residual d - q P - q Pe folded into the low part.
__device__ __forceinline__ df inv_diff(float a, float b)
{
    df d = two_sum(a, -b);
    float P = __fmul_rn(a, b);
    float Pe = __fmaf_rn(a, b, -P);
    float r = rcp_approx(P);
    float q = __fmul_rn(d.h, r);
    float e = __fmaf_rn(-q, P, d.h);
    e = __fadd_rn(e, d.l);
    e = __fmaf_rn(-q, Pe, e);
    return {q, __fmul_rn(e, r)};
}

template <int KIND>
struct KindTraits;
template <>
struct KindTraits<KIND_DEPTH_F32> {
    typedef float T;
    static constexpr bool disparity = false;
    static constexpr bool exact_diff = false;
};
template <>
struct KindTraits<KIND_DEPTH_F16> {
    typedef __half T;
    static constexpr bool disparity = false;
    static constexpr bool exact_diff = false;
};
template <>
struct KindTraits<KIND_DISP_U16> {
    typedef uint16_t T;
    static constexpr bool disparity = true;
    static constexpr bool exact_diff = true;  // integer differences are exact in FP32
};
template <>
struct KindTraits<KIND_DISP_F32> {
    typedef float T;
    static constexpr bool disparity = true;
    static constexpr bool exact_diff = false;
};

// Gradient term between taps a (the -1 side) and b (the +1 side).
template <int KIND>
__device__ __forceinline__ df grad_term(float a, float b)
{
    if (KindTraits<KIND>::disparity) {
        if (KindTraits<KIND>::exact_diff) return {__fsub_rn(b, a), 0.f};
        return two_sum(b, -a);
    }
    return inv_diff(a, b);
}

// Weighted filter sum G = c0 T0 + c1 T1 + c2 T2 (row weights of Sec. III's
// filters, normalisation dropped), compensated.
template <int GRAD>
__device__ __forceinline__ df filter_sum(df t0, df t1, df t2)
{
    if (GRAD == GRAD_FD) return t1;
    if (GRAD == GRAD_SOBEL || GRAD == GRAD_PREWITT) {
        const float c1 = GRAD == GRAD_SOBEL ? 2.f : 1.f;  // exact scalings
        df s = two_sum(t0.h, c1 * t1.h);
        df s2 = two_sum(s.h, t2.h);
        float lo = __fadd_rn(__fadd_rn(s.l, s2.l), __fadd_rn(__fadd_rn(t0.l, t2.l), c1 * t1.l));
        return {s2.h, lo};
    }
    // Scharr (3, 10, 3): the scaled terms need error-free products.
    df p0 = two_prod(3.f, t0.h), p1 = two_prod(10.f, t1.h), p2 = two_prod(3.f, t2.h);
    df s = two_sum(p0.h, p1.h);
    df s2 = two_sum(s.h, p2.h);
    float lo = __fadd_rn(__fadd_rn(s.l, s2.l), __fadd_rn(__fadd_rn(p0.l, p1.l), p2.l));
    lo = __fadd_rn(lo, __fmaf_rn(3.f, __fadd_rn(t0.l, t2.l), 10.f * t1.l));
    return {s2.h, lo};
}

// Weighted filter sum G = w0 T0 + w1 T1 + w2 T2 with the caller's row weights
// (the weighted family), compensated like Scharr's: error-free products and
// sums.  A zero-weight row drops out entirely (its taps may be holes).
__device__ __forceinline__ df filter_sum_w(df t0, df t1, df t2, float w0, float w1, float w2)
{
    const df z = {0.f, 0.f};
    const df a = w0 != 0.f ? t0 : z, b = w1 != 0.f ? t1 : z, c = w2 != 0.f ? t2 : z;
    const df p0 = two_prod(w0, a.h), p1 = two_prod(w1, b.h), p2 = two_prod(w2, c.h);
    const df s = two_sum(p0.h, p1.h);
    const df s2 = two_sum(s.h, p2.h);
    float lo = __fadd_rn(__fadd_rn(s.l, s2.l), __fadd_rn(__fadd_rn(p0.l, p1.l), p2.l));
    lo = __fadd_rn(lo, __fmaf_rn(w0, a.l, __fmaf_rn(w1, b.l, __fmul_rn(w2, c.l))));
    return {s2.h, lo};
}

template <int KIND, int GRAD>
__device__ __forceinline__ void gradients(const float (&z)[3][3], df &Gu, df &Gv, float w0, float w1, float w2)
{
    if (GRAD == GRAD_FD) {
        Gu = grad_term<KIND>(z[1][0], z[1][2]);
        Gv = grad_term<KIND>(z[0][1], z[2][1]);
    } else if (GRAD == GRAD_WEIGHTED) {
        Gu = filter_sum_w(grad_term<KIND>(z[0][0], z[0][2]), grad_term<KIND>(z[1][0], z[1][2]),
                          grad_term<KIND>(z[2][0], z[2][2]), w0, w1, w2);
        Gv = filter_sum_w(grad_term<KIND>(z[0][0], z[2][0]), grad_term<KIND>(z[0][1], z[2][1]),
                          grad_term<KIND>(z[0][2], z[2][2]), w0, w1, w2);
    } else {
        Gu = filter_sum<GRAD>(grad_term<KIND>(z[0][0], z[0][2]), grad_term<KIND>(z[1][0], z[1][2]),
                              grad_term<KIND>(z[2][0], z[2][2]));
        Gv = filter_sum<GRAD>(grad_term<KIND>(z[0][0], z[2][0]), grad_term<KIND>(z[0][1], z[2][1]),
                              grad_term<KIND>(z[0][2], z[2][2]));
    }
}

// Neighbour slots: pair p holds offset j_p = (du, dv) and -j_p.
//   p = 0: (1, 0)   p = 1: (0, 1)   p = 2: (1, 1)   p = 3: (1, -1)
__device__ __forceinline__ int pair_du(int p) { return p == 1 ? 0 : 1; }
__device__ __forceinline__ int pair_dv(int p) { return p == 0 ? 0 : (p == 3 ? -1 : 1); }

template <int GRAD>
__device__ __forceinline__ bool evaluable(const bool (&ok)[3][3])
{
    bool e = ok[1][1] && ok[1][0] && ok[1][2] && ok[0][1] && ok[2][1];
    if (GRAD != GRAD_FD) e = e && ok[0][0] && ok[0][2] && ok[2][0] && ok[2][2];
    return e;
}

// ------------------------------------------------------------ refinement

// The whole pixel again in double-float: exact differences, compensated
// products and quotients for every candidate, compensated accumulation.
// Used for the rare pixels whose FP32 error bound is too loose (or for all
// with TFN_FLAG_REFINE_ALL).
struct Vec3 {
    float x, y, z;
};

// The window travels by value (9 samples + 9 validity bits) so that the
// caller keeps it in registers; a reference would force it to local memory.
// The candidates, Phi and the normal in double-float, given the gradients.
template <int KIND, int PHI>
__device__ __forceinline__ Vec3 refine_candidates(const float (&z)[3][3], const bool (&ok)[3][3], df Gu, df Gv, int u,
                                                  int v, float fx, float fy, float u0, float v0)
{
    const float zi = z[1][1];
    // the candidates in fixed slots q = 2 p + side (pair p's neighbour j_p,
    // then -j_p), so that they stay in registers; kept[q]: the neighbour is
    // valid and differs from the centre
    df R[8];
    bool kept[8];
    int m = 0;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int du = pair_du(p), dv = pair_dv(p);
        df num = Gu;
        if (p == 1) num = Gv;
        if (p == 2) num = df_add(Gu, Gv);
        if (p == 3) num = df_add(Gu, df_neg(Gv));
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int a = 1 + (side ? -dv : dv), b = 1 + (side ? -du : du), q = 2 * p + side;
            const float zj = z[a][b];
            const df nj = side ? df_neg(num) : num;
            kept[q] = ok[a][b] && zj != zi;
            // (computed for every slot, without a branch, so that the eight
            // quotients overlap; a dropped slot's value may be inf or NaN
            // and is never selected)
            if (KindTraits<KIND>::disparity)  // Z_j / dz_j = d_i / (d_i - d_j)
                R[q] = df_div(df_mul_f(nj, zi), two_sum(zi, -zj));
            else
                R[q] = df_div(df_mul_f(nj, zj), two_sum(zj, -zi));
            m += kept[q] ? 1 : 0;
        }
    }
    df F = {0.f, 0.f};
    if (PHI == PHI_MEAN) {
        // the kept candidates summed pairwise (a dropped slot adds an exact 0)
        df t[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) t[q] = kept[q] ? R[q] : df{0.f, 0.f};
#pragma unroll
        for (int w = 1; w < 8; w *= 2)
#pragma unroll
            for (int q = 0; q < 8; q += 2 * w) t[q] = df_add(t[q], t[q + w]);
        F = df_div(t[0], df{(float)m, 0.f});
    } else {
        // The kept candidates in ascending order of their leading parts, ties
        // in slot order (a stable sort), by a sorting network over all 8
        // slots keyed on (leading part, slot): a dropped slot holds a
        // sentinel, +inf, -inf, +inf, ... in turn, so that the kept ones
        // always straddle the middle slots 3 and 4.
        float sh[8], sl[8];
        int si[8];
        float sent = __uint_as_float(0x7f800000u);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            sh[q] = kept[q] ? R[q].h : sent;
            sl[q] = kept[q] ? R[q].l : 0.f;
            si[q] = q;
            sent = kept[q] ? sent : -sent;
        }
#define TFN_CE2(i, j)                                                            \
    {                                                                            \
        const bool sw_ = sh[i] > sh[j] || (sh[i] == sh[j] && si[i] > si[j]);     \
        const float h_ = sw_ ? sh[j] : sh[i], l_ = sw_ ? sl[j] : sl[i];          \
        const int i_ = sw_ ? si[j] : si[i];                                      \
        sh[j] = sw_ ? sh[i] : sh[j];                                             \
        sl[j] = sw_ ? sl[i] : sl[j];                                             \
        si[j] = sw_ ? si[i] : si[j];                                             \
        sh[i] = h_;                                                              \
        sl[i] = l_;                                                              \
        si[i] = i_;                                                              \
    }
        TFN_CE2(0, 2) TFN_CE2(1, 3) TFN_CE2(4, 6) TFN_CE2(5, 7)
        TFN_CE2(0, 4) TFN_CE2(1, 5) TFN_CE2(2, 6) TFN_CE2(3, 7)
        TFN_CE2(0, 1) TFN_CE2(2, 3) TFN_CE2(4, 5) TFN_CE2(6, 7)
        TFN_CE2(2, 4) TFN_CE2(3, 5)
        TFN_CE2(1, 4) TFN_CE2(3, 6)
        TFN_CE2(1, 2) TFN_CE2(3, 4) TFN_CE2(5, 6)
#undef TFN_CE2
        // m kept: the middle one is slot 3 (m odd), the middle two slots 3
        // and 4 (m even)
        if (m > 0) {
            F = df{sh[3], sl[3]};
            if (!(m & 1)) {
                F = df_add(df{sh[3], sl[3]}, df{sh[4], sl[4]});
                F = {0.5f * F.h, 0.5f * F.l};
            }
        }
    }
    const df uc = two_sum((float)u, -u0), vc = two_sum((float)v, -v0);
    const df A = df_add(df_mul(uc, Gu), df_mul(vc, Gv));
    const float nzp = -df_val(df_add(A, F));
    const float nxp = df_val(df_mul_f(Gu, fx));
    const float nyp = df_val(df_mul_f(Gv, fy));
    // normalise with an exact power-of-two prescale (no over/underflow)
    float mx = fmaxf(fabsf(nxp), fmaxf(fabsf(nyp), fabsf(nzp)));
    int ex;
    frexpf(mx, &ex);
    const float x = ldexpf(nxp, -ex), y = ldexpf(nyp, -ex), w = ldexpf(nzp, -ex);
    const float rs = rsqrt_approx(x * x + y * y + w * w);
    return {-x * rs, -y * rs, -w * rs};
}

template <int KIND, int GRAD, int PHI>
__device__ __noinline__ Vec3 refine_pixel(float z00, float z01, float z02, float z10, float z11, float z12, float z20,
                                          float z21, float z22, unsigned okbits, int u, int v, float fx, float fy,
                                          float u0, float v0, float w0, float w1, float w2)
{
    const float z[3][3] = {{z00, z01, z02}, {z10, z11, z12}, {z20, z21, z22}};
    bool ok[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) ok[a][b] = (okbits >> (3 * a + b)) & 1u;
    df Gu, Gv;
    gradients<KIND, GRAD>(z, Gu, Gv, w0, w1, w2);
    return refine_candidates<KIND, PHI>(z, ok, Gu, Gv, u, v, fx, fy, u0, v0);
}

// ------------------------------------------------------------ main path

// 2^-110: below the square of the smallest non-zero difference of two valid
// samples (|delta| >= 2^-39, so delta^2 >= 2^-78) by 2^-32.
constexpr float kEdgeEps = 7.703719777548943e-34f;

// 2^-60: the one-pass FD mean's n_z' offset that gives a flat pixel its
// (0, 0, -1) without a test (row_step2).
constexpr float kFlatEps = 8.673617379884035e-19f;

// r = 1/delta and k = delta * r (1 for delta != 0, 0 for delta == 0) without
// a branch: delta / (delta^2 + eps) is 1/delta to a relative 2^-32 for every
// non-zero difference of valid samples and exactly 0 for delta == 0, which is
// how a neighbour at the centre's depth drops out of the candidates.
struct EdgeR {
    float r, k;
};
__device__ __forceinline__ EdgeR edge_recip(float delta)
{
    const float r = __fmul_rn(delta, rcp_approx(__fmaf_rn(delta, delta, kEdgeEps)));
    return {r, __fmul_rn(delta, r)};
}

// edge_recip on a pair of edges, keeping delta (d) instead of k: its users
// form k = delta r inside their sums.
struct EdgeR2 {
    f2 r, d;
};
__device__ __forceinline__ EdgeR2 edge_recip2(f2 delta)
{
    return {mul2(delta, rcp2(fma2(delta, delta, bc(kEdgeEps)))), delta};
}

// A hole's stand-in value, 2^100.  Its difference with any valid sample
// (<= 2^16) has a square that overflows to +inf, whose reciprocal is 0, so an
// edge that touches a hole gets r = 0 and k = 0 with no test (two holes give
// delta = 0: the same).  Valid samples are <= kValidHi, holes are above it.
constexpr float kHole = 1.2676506002282294e30f;

template <int KIND>
__device__ __forceinline__ float decode(typename KindTraits<KIND>::T raw)
{
    if constexpr (KIND == KIND_DISP_U16) {
        const float v = (float)raw;
        return v != 0.f ? v : kHole;
    } else {
        float v;
        if constexpr (KIND == KIND_DEPTH_F16)
            v = __half2float(raw);
        else
            v = raw;
        // finite and in [2^-16, 2^16]: one unsigned compare on the bit pattern
        // (negatives, infinities and NaNs have patterns above 2^16's)
        return (uint32_t)(__float_as_uint(v) - 0x37800000u) <= (0x47800000u - 0x37800000u) ? v : kHole;
    }
}

template <class T>
__device__ __forceinline__ T from_bits16(uint32_t b)
{
    if constexpr (sizeof(T) == 2) {
        const uint16_t s = (uint16_t)b;
        return *reinterpret_cast<const T *>(&s);
    } else {
        return T();
    }
}

// One sample row of a lane's window: image columns x0-1 .. x0+4 around the
// lane's 4 pixel columns x0 .. x0+3.  Depth rows that feed a compensated
// (Sobel-type) filter also carry w = 1/Z per sample as wh + wl.
template <int KIND, int GRAD>
struct Row {
    static constexpr bool kW = !KindTraits<KIND>::disparity && GRAD != GRAD_FD && GRAD != GRAD_SEP5 &&
                               GRAD != GRAD_PLANEPCA;
    float z[6];
    float wh[kW ? 6 : 1], wl[kW ? 6 : 1];
};

// Sample c (0 .. 5) of a row.
template <int KIND, int GRAD>
__device__ __forceinline__ float sample(const Row<KIND, GRAD> &R, int c)
{
    return R.z[c];
}

// The sample pair (z_i, z_{i+2}) of a row: row_step2 takes a lane's pixels
// 1 and 3, then 2 and 4, as pairs, whose windows sit on these pairs.
template <int KIND, int GRAD>
__device__ __forceinline__ f2 zpair(const Row<KIND, GRAD> &R, int i)
{
    return pk(R.z[i], R.z[i + 2]);
}

// Fills a row with its 6 decoded samples.
template <int KIND, int GRAD>
__device__ __forceinline__ void set_row(Row<KIND, GRAD> &R, const float (&z)[6])
{
#pragma unroll
    for (int c = 0; c < 6; ++c) R.z[c] = z[c];
}

// Reads row `jr` of a staged box (BOXW samples per row, the lane's pixels at
// column PADX + 4 lane) and decodes it.
template <int KIND, int GRAD, int BOXW, int PADX>
__device__ __forceinline__ void load_row(const unsigned char *stage, int jr, int lane, Row<KIND, GRAD> &R)
{
    typedef typename KindTraits<KIND>::T T;
    const T *p = reinterpret_cast<const T *>(stage) + jr * BOXW + PADX + 4 * lane;
    T raw[6];
    raw[0] = p[-1];
    if constexpr (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        raw[1] = q.x;
        raw[2] = q.y;
        raw[3] = q.z;
        raw[4] = q.w;
    } else {
        const uint2 q = *reinterpret_cast<const uint2 *>(p);
        raw[1] = from_bits16<T>(q.x & 0xffffu);
        raw[2] = from_bits16<T>(q.x >> 16);
        raw[3] = from_bits16<T>(q.y & 0xffffu);
        raw[4] = from_bits16<T>(q.y >> 16);
    }
    raw[5] = p[4];
    float z[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) z[c] = decode<KIND>(raw[c]);
    set_row(R, z);
    if constexpr (Row<KIND, GRAD>::kW) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const float wh = rcp_approx(z[c]);
            R.wh[c] = wh;
            R.wl[c] = __fmul_rn(__fmaf_rn(-wh, z[c], 1.f), wh);
        }
    }
}

// The FD gradient term between taps a (the -1 side) and b (the +1 side) of
// both pixels of a pair, as h + l.  Depth: 1/Z_b - 1/Z_a = d / P with d =
// Z_a - Z_b (exact for neighbouring depths within a factor 2) and P = Z_a
// Z_b; h = d rcp(P), and l is h's residual against the exact product P + Pe
// divided by P, so h + l is the quotient to about u^2 relative, as a
// difference of compensated reciprocals would be; h is 0 exactly when the
// taps are equal.  With ONE_PASS (the mean on depth when kFdOnePassMean is
// set) only h: within 5u of the quotient (the difference exact or rounded
// once, the product rounded once, the reciprocal within one ulp, the product
// with it rounded once; no operand or result subnormal for samples in
// [2^-16, 2^16]).  Disparity: d_b - d_a (exact for integer samples; TwoSum for
// float ones).
struct df2 {
    f2 h, l;
};
template <int KIND, bool ONE_PASS>
__device__ __forceinline__ df2 fd_term2(f2 a, f2 b)
{
    if constexpr (KindTraits<KIND>::disparity) {
        if constexpr (KindTraits<KIND>::exact_diff) return {sub2(b, a), bc(0.f)};
        // TwoSum(b, -a): s = b - a, bb = s - b, e = (b - (s - bb)) - (a + bb)
        const f2 sm = sub2(b, a);
        const f2 bb = sub2(sm, b);
        return {sm, sub2(sub2(b, sub2(sm, bb)), add2(a, bb))};
    } else if constexpr (ONE_PASS) {
        return {mul2(sub2(a, b), rcp2(mul2(a, b))), bc(0.f)};
    } else {
        const f2 d = sub2(a, b);
        const f2 P = mul2(a, b);
        const f2 Pe = fma2(a, b, neg2(P));
        const f2 r = rcp2(P);
        const f2 q = mul2(d, r);
        const f2 nq = neg2(q);
        const f2 e = fma2(nq, Pe, fma2(nq, P, d));
        return {q, mul2(e, r)};
    }
}

// Exact difference of two compensated taps, w_b - w_a as h + l.
template <int KIND, int GRAD>
__device__ __forceinline__ df tap_diff(const Row<KIND, GRAD> &A, int ca, const Row<KIND, GRAD> &B, int cb)
{
    if constexpr (KindTraits<KIND>::disparity) {
        if constexpr (KindTraits<KIND>::exact_diff) return {__fsub_rn(B.z[cb], A.z[ca]), 0.f};
        return two_sum(B.z[cb], -A.z[ca]);
    } else {
        const float lo = __fsub_rn(B.wl[cb], A.wl[ca]);
        const df h = two_sum(B.wh[cb], -A.wh[ca]);
        return {h.h, __fadd_rn(h.l, lo)};
    }
}

// rho of the two end pixels of an edge p -> q (p first in raster order),
// r = 1/(s_q - s_p): rho_fwd is q's rho seen from p, rho_bwd is p's rho seen
// from q.  Depth: rho_j = Z_j / (Z_j - Z_i); disparity: d_i / (d_i - d_j).
template <int KIND>
__device__ __forceinline__ float rho_fwd(float sp, float sq, float r)
{
    if constexpr (KindTraits<KIND>::disparity)
        return -__fmul_rn(sp, r);
    else
        return __fmul_rn(sq, r);
}
template <int KIND>
__device__ __forceinline__ float rho_bwd(float sp, float sq, float r)
{
    if constexpr (KindTraits<KIND>::disparity)
        return __fmul_rn(sq, r);
    else
        return -__fmul_rn(sp, r);
}

// rho of the neighbours above a row's 4 pixels, known from the previous row
// pair: up, up-left, up-right, and how many of the three are kept.
struct UpCarry {
    float ru[4], rul[4], rur[4], ku[4];
};

// Edges between sample rows C (above) and N (below) as seen from N's pixels:
// the carry for the row of N.
template <int KIND, int GRAD>
__device__ __forceinline__ void carry_down(const Row<KIND, GRAD> &C, const Row<KIND, GRAD> &N, UpCarry &cy)
{
#pragma unroll
    for (int c = 1; c <= 4; ++c) {
        const EdgeR v = edge_recip(__fsub_rn(N.z[c], C.z[c]));          // (y, c)   -> (y+1, c)
        const EdgeR d = edge_recip(__fsub_rn(N.z[c], C.z[c - 1]));      // (y, c-1) -> (y+1, c)
        const EdgeR a = edge_recip(__fsub_rn(N.z[c], C.z[c + 1]));      // (y, c+1) -> (y+1, c)
        cy.ru[c - 1] = rho_bwd<KIND>(C.z[c], N.z[c], v.r);
        cy.rul[c - 1] = rho_bwd<KIND>(C.z[c - 1], N.z[c], d.r);
        cy.rur[c - 1] = rho_bwd<KIND>(C.z[c + 1], N.z[c], a.r);
        cy.ku[c - 1] = __fadd_rn(__fadd_rn(v.k, d.k), a.k);
    }
}

// Whether a 3x3 kernel keeps its rows' horizontal tap differences in the
// shared-memory ring (computed once per sample row, read by the three output
// rows that use them) instead of computing them for each output row:
// Sobel, Scharr and Prewitt, 4-7% faster with it (means) and up to 2.5%
// (medians) on the 256-frame batch; the weighted family measured 1% slower
// (its row step spills with it).
constexpr bool uses_dring(int grad, int phi)
{
    return (grad == GRAD_SOBEL || grad == GRAD_SCHARR || grad == GRAD_PREWITT) && (phi == PHI_MEAN || phi == PHI_MEDIAN);
}

// A row's horizontal tap differences w[c+1] - w[c-1] (exact, as h + l) at the
// columns of pair h (1 + h and 3 + h).
template <int KIND, int GRAD>
__device__ __forceinline__ df2 hdiff_pair(const Row<KIND, GRAD> &R, int h)
{
    const df a = tap_diff(R, h, R, h + 2), b = tap_diff(R, h + 2, R, h + 4);
    return {pk(a.h, b.h), pk(a.l, b.l)};
}

// The 3x3 filters: the carry of the pixel pairs (pair 0: pixels 1 and 3, pair 1: pixels
// 2 and 4): the magnitudes B of the rho of the up, up-left and up-right
// neighbours (rho = -B on depth, +B on disparity) and how many of the three
// are kept.  It lives in shared memory, this lane's slots of its warp's
// buffer (kCarry3Bytes): pair h at q[64 h] = (B_u, B_ul) and q[64 h + 32] =
// (B_ur, k_u), so that a pair's carry occupies registers only between its
// load and its store in row_step2.
struct UpCarry2 {
    float4 *q;
    // (smoothed filters) the ring of horizontal tap differences: row slot t,
    // pair h at d[32 (2 t + h)] = (D.h of both pixels, D.l of both); the slot of
    // the current P row is p0, then C and N follow cyclically
    float4 *d;
    int p0;
    bool ring;  // whether the ring is used (a constant of the kernel: uses_dring)
    __device__ __forceinline__ void dget(int t, int h, df2 &D) const
    {
        const float4 a = d[32 * (2 * t + h)];
        D = {pk(a.x, a.y), pk(a.z, a.w)};
    }
    __device__ __forceinline__ void dput(int t, int h, const df2 &D) const
    {
        d[32 * (2 * t + h)] = make_float4(D.h.x, D.h.y, D.l.x, D.l.y);
    }
    __device__ __forceinline__ void get(int h, f2 &bu, f2 &bul, f2 &bur, f2 &ku) const
    {
        const float4 a = q[64 * h], b = q[64 * h + 32];
        bu = pk(a.x, a.y);
        bul = pk(a.z, a.w);
        bur = pk(b.x, b.y);
        ku = pk(b.z, b.w);
    }
    __device__ __forceinline__ void put(int h, f2 bu, f2 bul, f2 bur, f2 ku) const
    {
        q[64 * h] = make_float4(bu.x, bu.y, bul.x, bul.y);
        q[64 * h + 32] = make_float4(bur.x, bur.y, ku.x, ku.y);
    }
};
template <int GRAD, bool PAIR = grad_is_pair(GRAD)>
struct CarryOf {
    typedef UpCarry type;
};
template <int GRAD>
struct CarryOf<GRAD, true> {
    typedef UpCarry2 type;
};

// carry_down for the 3x3 filters' rows.  Edge p -> q with r = 1/(s_q - s_p):
// seen from q, rho = -s_p r on depth and s_q r on disparity (rho_bwd).
template <int KIND, int GRAD>
__device__ __forceinline__ void carry_down(const Row<KIND, GRAD> &C, const Row<KIND, GRAD> &N, UpCarry2 &cy)
{
    constexpr bool disp = KindTraits<KIND>::disparity;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const f2 Cl = zpair(C, h), Cc = zpair(C, 1 + h), Cr = zpair(C, 2 + h), Nc = zpair(N, 1 + h);
        const EdgeR2 v = edge_recip2(sub2(Nc, Cc));  // (y, c)   -> (y+1, c)
        const EdgeR2 d = edge_recip2(sub2(Nc, Cl));  // (y, c-1) -> (y+1, c)
        const EdgeR2 a = edge_recip2(sub2(Nc, Cr));  // (y, c+1) -> (y+1, c)
        cy.put(h, mul2(disp ? Nc : Cc, v.r), mul2(disp ? Nc : Cl, d.r), mul2(disp ? Nc : Cr, a.r),
               fma2(v.d, v.r, fma2(d.d, d.r, mul2(a.d, a.r))));
        if (GRAD != GRAD_FD && cy.ring) {  // the first two rows' horizontal tap differences
            cy.dput(0, h, hdiff_pair(C, h));
            cy.dput(1, h, hdiff_pair(N, h));
        }
    }
    cy.p0 = 0;
}

// One row of a lane's 4 pixels (Sec. III end to end) for the 5x5 filters
// (the 3x3 filters run row_step2), given the sample rows above (P), at (C)
// and below (N) and the carry from the row above; leaves the carry for the
// next row in `cy`.  Outputs the normal components, the mask bits and the
// bits of the pixels whose FP32 error bound is too loose.  Every product is
// an explicit __fmul_rn and every fused multiply-add an explicit __fmaf_rn
// (never a contraction), so a pixel's bits do not depend on how the compiler
// schedules this code in a given instantiation.
template <int KIND, int GRAD, int PHI>
__device__ __forceinline__ void row_step(const Row<KIND, GRAD> &P, const Row<KIND, GRAD> &C, const Row<KIND, GRAD> &N,
                                         UpCarry &cy, const float (&uc)[4], float vc, float fx, float fy, float thr,
                                         const float (&wts)[3], const df (&gin_u)[4], const df (&gin_v)[4],
                                         float (&ox)[4], float (&oy)[4], float (&oz)[4], uint32_t &mword,
                                         unsigned &rbits)
{
    static_assert(GRAD == GRAD_SEP5, "the 3x3 filters run row_step2");
    // edges of this row (c -> c+1) and to the row below, computed pixel by
    // pixel: pixel c needs those of columns c-1 and c only
    EdgeR h[5], ed[5], ea[5];
    h[0] = edge_recip(__fsub_rn(C.z[1], C.z[0]));
    ed[0] = edge_recip(__fsub_rn(N.z[1], C.z[0]));  // (y, 0) -> (y+1, 1)
    ea[0] = edge_recip(__fsub_rn(N.z[0], C.z[1]));  // (y, 1) -> (y+1, 0)
    mword = 0;
    rbits = 0;
#pragma unroll
    for (int c = 1; c <= 4; ++c) {
        const int k = c - 1;
        h[c] = edge_recip(__fsub_rn(C.z[c + 1], C.z[c]));
        ed[c] = edge_recip(__fsub_rn(N.z[c + 1], C.z[c]));  // (y, c)   -> (y+1, c+1)
        ea[c] = edge_recip(__fsub_rn(N.z[c], C.z[c + 1]));  // (y, c+1) -> (y+1, c)
        const EdgeR ev = edge_recip(__fsub_rn(N.z[c], C.z[c]));  // (y, c) -> (y+1, c)
        const float zi = C.z[c];
        const float rr = rho_fwd<KIND>(zi, C.z[c + 1], h[c].r);
        const float rl = rho_bwd<KIND>(C.z[c - 1], zi, h[c - 1].r);
        const float rd = rho_fwd<KIND>(zi, N.z[c], ev.r);
        const float rdr = rho_fwd<KIND>(zi, N.z[c + 1], ed[c].r);
        const float rdl = rho_fwd<KIND>(zi, N.z[c - 1], ea[c - 1].r);
        const float ru = cy.ru[k], rul = cy.rul[k], rur = cy.rur[k];
        const float m = __fadd_rn(__fadd_rn(__fadd_rn(h[c].k, h[c - 1].k), __fadd_rn(ev.k, ed[c].k)),
                                  __fadd_rn(ea[c - 1].k, cy.ku[k]));

        // the 5x5 gradients come from the caller as h + l, NaN where a needed
        // tap is a hole; evaluability and the special case
        const df Gu = gin_u[k], Gv = gin_v[k];
        const bool ev_ok = zi <= kValidHi && Gu.h == Gu.h && Gv.h == Gv.h;
        // Sec. III special case: both gradients exactly zero (an h + l pair
        // vanishes only when both parts do)
        bool flat = Gu.h == 0.f && Gu.l == 0.f && Gv.h == 0.f && Gv.l == 0.f;
        // (a non-evaluable pixel's gradient may be NaN, from two hole taps: keep n' finite)
        const float gu = ev_ok ? __fadd_rn(Gu.h, Gu.l) : 0.f, gv = ev_ok ? __fadd_rn(Gv.h, Gv.l) : 0.f;
        // numerators of the diagonal pairs from the parts (they can cancel)
        const float n2 = __fadd_rn(__fadd_rn(Gu.h, Gv.h), __fadd_rn(Gu.l, Gv.l));
        const float n3 = __fadd_rn(__fsub_rn(Gu.h, Gv.h), __fsub_rn(Gu.l, Gv.l));

        float mF, mbound, scale;
        bool none;  // no neighbour gives a candidate
        if constexpr (PHI == PHI_MEAN) {
            // sum over the pairs (j, -j) of num_p (rho_j - rho_-j), carried
            // unnormalised: n' scaled by m > 0 keeps its direction
            const float S = __fmaf_rn(gu, __fsub_rn(rr, rl),
                                      __fmaf_rn(gv, __fsub_rn(rd, ru),
                                                __fmaf_rn(n2, __fsub_rn(rdr, rul), __fmul_rn(n3, __fsub_rn(rur, rdl)))));
            // bound of the candidate sum's rounding: sum_p |num_p| (|rho_j| + |rho_-j|)
            mbound = __fmaf_rn(fabsf(gu), __fadd_rn(fabsf(rr), fabsf(rl)),
                               __fmaf_rn(fabsf(gv), __fadd_rn(fabsf(rd), fabsf(ru)),
                                         __fmaf_rn(fabsf(n2), __fadd_rn(fabsf(rdr), fabsf(rul)),
                                                   __fmul_rn(fabsf(n3), __fadd_rn(fabsf(rur), fabsf(rdl))))));
            mF = S;
            scale = m;
            none = m == 0.f;
        } else {
            const float rho8[8] = {rr, rl, rd, ru, rdr, rul, rur, rdl};
            const float num8[8] = {gu, -gu, gv, -gv, n2, -n2, n3, -n3};
            float s[8];
            float sent = __uint_as_float(0x7f800000u);  // the next sentinel: +inf, -inf, +inf, ...
            int cnt = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const bool kept = rho8[q] != 0.f;
                cnt += kept;
                s[q] = kept ? __fmul_rn(num8[q], rho8[q]) : sent;
                sent = kept ? sent : -sent;
            }
#define TFN_CE(i, j)                         \
    {                                        \
        const float lo_ = fminf(s[i], s[j]); \
        s[j] = fmaxf(s[i], s[j]);            \
        s[i] = lo_;                          \
    }
            TFN_CE(0, 2) TFN_CE(1, 3) TFN_CE(4, 6) TFN_CE(5, 7)
            TFN_CE(0, 4) TFN_CE(1, 5) TFN_CE(2, 6) TFN_CE(3, 7)
            TFN_CE(0, 1) TFN_CE(2, 3) TFN_CE(4, 5) TFN_CE(6, 7)
            TFN_CE(2, 4) TFN_CE(3, 5)
            TFN_CE(1, 4) TFN_CE(3, 6)
            TFN_CE(1, 2) TFN_CE(3, 4) TFN_CE(5, 6)
#undef TFN_CE
            const bool odd = sent < 0.f;  // (8 - cnt missing: odd with cnt)
            none = cnt == 0;
            mF = odd ? s[3] : __fmul_rn(0.5f, __fadd_rn(s[3], s[4]));
            mbound = odd ? fabsf(s[3]) : fmaxf(fabsf(s[3]), fabsf(s[4]));
            scale = 1.f;
        }
        // Sec. III special case when every valid neighbour shares the centre's
        // depth: with 3x3 filters the gradients are then zero (flat already);
        // a 5x5 filter can still see a depth change in its outer taps
        if constexpr (GRAD == GRAD_SEP5) flat = flat || none;
        const float gxo = GRAD == GRAD_SEP5 && flat ? 0.f : gu, gyo = GRAD == GRAD_SEP5 && flat ? 0.f : gv;
        const float A = __fmaf_rn(uc[k], gu, __fmul_rn(vc, gv));
        const float nxp = __fmul_rn(__fmul_rn(scale, fx), gxo), nyp = __fmul_rn(__fmul_rn(scale, fy), gyo);
        // (a non-evaluable pixel's median may be a +-inf sentinel: keep n' finite so that rs = 0 zeroes it)
        const float nzp = (flat || !ev_ok) ? 1.f : -__fmaf_rn(scale, A, mF);
        const float nn = __fmaf_rn(nxp, nxp, __fmaf_rn(nyp, nyp, __fmul_rn(nzp, nzp)));
        const float rs = ev_ok ? rsqrt_approx(nn) : 0.f;
        // refine unless bound <= thr |n'|; written so that a NaN (|n'|
        // overflowed) also refines, and thr < 0 refines every pixel
        const bool refine = ev_ok && !flat && !(mbound <= __fmul_rn(thr, __fmul_rn(nn, rs)));
        // -n'/|n'|, with +0 (not -0) for zero components and for non-evaluable pixels
        ox[k] = __fmaf_rn(-nxp, rs, 0.f);
        oy[k] = __fmaf_rn(-nyp, rs, 0.f);
        oz[k] = __fmaf_rn(-nzp, rs, 0.f);
        mword |= ev_ok ? 1u << (8 * k) : 0u;
        rbits |= refine ? 1u << k : 0u;

        // the carry for the pixel below: its up, up-left and up-right neighbours
        cy.ru[k] = rho_bwd<KIND>(zi, N.z[c], ev.r);
        cy.rul[k] = rho_bwd<KIND>(C.z[c - 1], N.z[c], ed[c - 1].r);
        cy.rur[k] = rho_bwd<KIND>(C.z[c + 1], N.z[c], ea[c].r);
        cy.ku[k] = __fadd_rn(__fadd_rn(ev.k, ed[c - 1].k), ea[c].k);
    }
}

// The smoothed 3x3 filters' gradients of a pair's two pixels (columns 1 + h
// and 3 + h of the lane's window), each as the scalar step computes them:
// exact tap differences and the compensated filter sum (weighted: the
// caller's row weights); and each pixel's evaluability (every tap with a
// non-zero weight in either filter inside the frame and valid).
template <int KIND, int GRAD>
__device__ __forceinline__ void grad_pair(const Row<KIND, GRAD> &P, const Row<KIND, GRAD> &C, const Row<KIND, GRAD> &N,
                                          int h, const UpCarry2 &cy, const float (&wts)[3], df2 &Gu, df2 &Gv,
                                          bool (&ev_ok)[2])
{
    // the horizontal tap differences: rows P and C from the ring and N's into
    // it, or all three computed here
    df2 DP, DC, DN = hdiff_pair(N, h);
    if (cy.ring) {
        const int tc = cy.p0 == 2 ? 0 : cy.p0 + 1, tn = tc == 2 ? 0 : tc + 1;
        cy.dget(cy.p0, h, DP);
        cy.dget(tc, h, DC);
        cy.dput(tn, h, DN);
    } else {
        DP = hdiff_pair(P, h);
        DC = hdiff_pair(C, h);
    }
    df gu[2], gv[2];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        const int c = 1 + h + 2 * l;
        const df dp = {lane_of(DP.h, l), lane_of(DP.l, l)}, dc = {lane_of(DC.h, l), lane_of(DC.l, l)},
                 dn = {lane_of(DN.h, l), lane_of(DN.l, l)};
        if constexpr (GRAD == GRAD_WEIGHTED) {
            const float w0 = wts[0], w1 = wts[1], w2 = wts[2];
            gu[l] = filter_sum_w(dp, dc, dn, w0, w1, w2);
            gv[l] = filter_sum_w(tap_diff(P, c - 1, N, c - 1), tap_diff(P, c, N, c), tap_diff(P, c + 1, N, c + 1), w0,
                                 w1, w2);
            // tap (row a, column b) is needed when its row's weight is non-zero in the horizontal
            // filter (outer columns) or its column's weight in the vertical one (outer rows)
            const bool n0 = w0 != 0.f, n1 = w1 != 0.f, n2 = w2 != 0.f;
            float mx = C.z[c];
            mx = fmaxf(mx, n0 ? P.z[c - 1] : 0.f);
            mx = fmaxf(mx, (n0 || n2) ? P.z[c + 1] : 0.f);
            mx = fmaxf(mx, (n0 || n2) ? N.z[c - 1] : 0.f);
            mx = fmaxf(mx, n2 ? N.z[c + 1] : 0.f);
            mx = fmaxf(mx, n1 ? fmaxf(fmaxf(P.z[c], N.z[c]), fmaxf(C.z[c - 1], C.z[c + 1])) : 0.f);
            ev_ok[l] = mx <= kValidHi;
        } else {
            gu[l] = filter_sum<GRAD>(dp, dc, dn);
            gv[l] = filter_sum<GRAD>(tap_diff(P, c - 1, N, c - 1), tap_diff(P, c, N, c), tap_diff(P, c + 1, N, c + 1));
            const float mp = fmaxf(fmaxf(P.z[c - 1], P.z[c]), P.z[c + 1]);
            const float mc = fmaxf(fmaxf(C.z[c - 1], C.z[c]), C.z[c + 1]);
            const float mn = fmaxf(fmaxf(N.z[c - 1], N.z[c]), N.z[c + 1]);
            ev_ok[l] = fmaxf(fmaxf(mp, mc), mn) <= kValidHi;
        }
    }
    Gu = {pk(gu[0].h, gu[1].h), pk(gu[0].l, gu[1].l)};
    Gv = {pk(gv[0].h, gv[1].h), pk(gv[0].l, gv[1].l)};
}

// The row step of the 3x3 filters, two pixels at a time.  A lane's pixels 1
// and 3 form one pair and pixels 2 and 4 the other: their windows sit on the
// same sample pairs (zpair), so each edge, rho and sum is written once for a
// pair (add2, mul2, fma2), and the pair's carry lives in shared memory
// between rows (UpCarry2).  The gradients: FD's quotients on the pairs
// (fd_term2; one-pass for the mean on depth when kFdOnePassMean is set), the
// smoothed filters' per pixel as the scalar step computes them (grad_pair:
// exact tap differences, compensated filter sums).
//
// rho of the neighbours: an edge p -> q with r = 1/(s_q - s_p) gives p the
// rho s_q r (depth) or -s_p r (disparity), and q the rho -s_p r or s_q r; the
// pairs keep the magnitudes F (forward: right, down, down-right, down-left)
// and B (backward: left, up, up-left, up-right), with rho = sF forward and
// -sB backward, s = +1 on depth and -1 on disparity.  Then rho_j - rho_-j of
// the pairs (right, left), (down, up), (down-right, up-left) is s (F + B), and
// that of (up-right, down-left) -s (B + F): the candidate sum is s T with T
// below (n3n = G_v - G_u = -n3), and the candidates are s times the products
// num F or num B.
//
// NOREF: the launch's frames are known never to need refinement (FP16 depth,
// see refinement_idle on the host), so the error bound and the refinement
// test are not computed; every other operation, and so every result bit, is
// that of NOREF = false.
template <int KIND, int GRAD, int PHI, bool NOREF>
__device__ __forceinline__ void row_step2(const Row<KIND, GRAD> &P, const Row<KIND, GRAD> &C, const Row<KIND, GRAD> &N,
                                          UpCarry2 &cy, const f2 (&uc2)[2], float vc, float fx, float fy, float thr,
                                          const float (&wts)[3], float (&ox)[4], float (&oy)[4], float (&oz)[4],
                                          uint32_t &mword, unsigned &rbits)
{
    static_assert(grad_is_pair(GRAD), "row_step2 runs the 3x3 filters");
    constexpr bool disp = KindTraits<KIND>::disparity;
    constexpr bool one_pass = GRAD == GRAD_FD && kFdOnePassMean && PHI == PHI_MEAN && !disp;
    // Whether the mean's special case and flat test come from n_z' = kFlatEps -
    // Q and the bound (below).  For FD and the symmetric filters a non-zero
    // gradient always has a kept neighbour in a pair of non-zero weight.  The
    // weighted family keeps the explicit test: with w0 != w2 that need not
    // hold, and its row step spilled with the change (0.6% slower; Sobel's
    // 2.5% faster).
    constexpr bool flat_by_bound = PHI == PHI_MEAN && !NOREF && GRAD != GRAD_WEIGHTED;
    const f2 vc2 = bc(vc), fx2 = bc(fx), fy2 = bc(fy);
    // the edges to column c-1 of pixels c = 1, 3 (the next pair's come from this pair)
    EdgeR2 ehm = edge_recip2(sub2(zpair(C, 1), zpair(C, 0)));  // (y, c-1) -> (y, c)
    EdgeR2 edm = edge_recip2(sub2(zpair(N, 1), zpair(C, 0)));  // (y, c-1) -> (y+1, c)
    EdgeR2 eam = edge_recip2(sub2(zpair(N, 0), zpair(C, 1)));  // (y, c)   -> (y+1, c-1)
    mword = 0;
    rbits = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const f2 Cl = zpair(C, h), Cc = zpair(C, 1 + h), Cr = zpair(C, 2 + h);
        const f2 Nl = zpair(N, h), Nc = zpair(N, 1 + h), Nr = zpair(N, 2 + h), Pc = zpair(P, 1 + h);
        const EdgeR2 eh = edge_recip2(sub2(Cr, Cc));  // (y, c)   -> (y, c+1)
        const EdgeR2 ed = edge_recip2(sub2(Nr, Cc));  // (y, c)   -> (y+1, c+1)
        const EdgeR2 ea = edge_recip2(sub2(Nc, Cr));  // (y, c+1) -> (y+1, c)
        const EdgeR2 ev = edge_recip2(sub2(Nc, Cc));  // (y, c)   -> (y+1, c)
        const f2 Fr = mul2(disp ? Cc : Cr, eh.r);
        const f2 Bl = mul2(disp ? Cc : Cl, ehm.r);
        const f2 Fd = mul2(disp ? Cc : Nc, ev.r);
        const f2 Fdr = mul2(disp ? Cc : Nr, ed.r);
        const f2 Fdl = mul2(disp ? Cc : Nl, eam.r);
        f2 Bu, Bul, Bur, ku;
        cy.get(h, Bu, Bul, Bur, ku);
        // the candidate count: delta r over the 8 edges (1 to a few ulp for a
        // kept neighbour, 0 for a dropped one), the up edges' sum carried
        const f2 m = fma2(eh.d, eh.r, fma2(ehm.d, ehm.r, fma2(ev.d, ev.r, fma2(ed.d, ed.r, fma2(eam.d, eam.r, ku)))));

        // gradients (as h + l), evaluability and the special case, per pixel
        df2 Gu, Gv;
        bool ev_ok[2], flat[2];
        if constexpr (GRAD == GRAD_FD) {
            Gu = fd_term2<KIND, one_pass>(Cl, Cr);
            Gv = fd_term2<KIND, one_pass>(Pc, Nc);
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                ev_ok[l] = fmaxf(fmaxf(fmaxf(lane_of(Cl, l), lane_of(Cc, l)), lane_of(Cr, l)),
                                 fmaxf(lane_of(Pc, l), lane_of(Nc, l))) <= kValidHi;
                // Sec. III special case: both gradients exactly zero (an FD term's
                // low part is 0 whenever its high part is)
                flat[l] = lane_of(Gu.h, l) == 0.f && lane_of(Gv.h, l) == 0.f;
            }
        } else {
            grad_pair<KIND, GRAD>(P, C, N, h, cy, wts, Gu, Gv, ev_ok);
#pragma unroll
            for (int l = 0; l < 2; ++l)  // (an h + l pair vanishes only when both parts do)
                flat[l] = lane_of(Gu.h, l) == 0.f && lane_of(Gu.l, l) == 0.f && lane_of(Gv.h, l) == 0.f &&
                          lane_of(Gv.l, l) == 0.f;
        }
        f2 gu, gv, n2, n3n;
        if constexpr (one_pass) {
            // (one-pass quotients are finite on hole taps; a non-evaluable
            // pixel's output is zeroed through rs below)
            gu = Gu.h;
            gv = Gv.h;
            n2 = add2(gu, gv);
            n3n = sub2(gv, gu);
        } else {
            // (a non-evaluable pixel's gradient may be NaN, from two hole taps: keep n' finite)
            const f2 su = add2(Gu.h, Gu.l), sv = add2(Gv.h, Gv.l);
            gu = pk(ev_ok[0] ? su.x : 0.f, ev_ok[1] ? su.y : 0.f);
            gv = pk(ev_ok[0] ? sv.x : 0.f, ev_ok[1] ? sv.y : 0.f);
            // numerators of the diagonal pairs from the parts (they can cancel)
            n2 = add2(add2(Gu.h, Gv.h), add2(Gu.l, Gv.l));
            n3n = add2(sub2(Gv.h, Gu.h), sub2(Gv.l, Gu.l));
        }

        f2 mF, scale;
        float mbound[2] = {};
        if constexpr (PHI == PHI_MEAN) {
            // sum over the pairs (j, -j) of num_p (rho_j - rho_-j) = s T,
            // carried unnormalised: n' scaled by m > 0 keeps its direction
            const f2 T = fma2(gu, add2(Fr, Bl), fma2(gv, add2(Fd, Bu), fma2(n2, add2(Fdr, Bul), mul2(n3n, add2(Bur, Fdl)))));
            mF = disp ? neg2(T) : T;
#pragma unroll
            for (int l = 0; l < 2 && !NOREF; ++l) {
                // bound of the candidate sum's rounding: sum_p |num_p| (|rho_j| + |rho_-j|),
                // which the host's threshold multiplies by K1 u.  One-pass gradients
                // (within 5u each) put up to 5u (|G_u| + |G_v|) on a diagonal
                // numerator, whose cancellation can leave it large against the
                // numerator: its weight grows by 0.3 (|G_u| + |G_v|) (5u / (K1 u)
                // with this path's K1 = 17, see refine_threshold)
                float w2 = fabsf(lane_of(n2, l)), w3 = fabsf(lane_of(n3n, l));
                if constexpr (one_pass) {
                    const float sg = __fadd_rn(fabsf(lane_of(gu, l)), fabsf(lane_of(gv, l)));
                    w2 = __fmaf_rn(0.3f, sg, w2);
                    w3 = __fmaf_rn(0.3f, sg, w3);
                }
                mbound[l] = __fmaf_rn(fabsf(lane_of(gu, l)), __fadd_rn(fabsf(lane_of(Fr, l)), fabsf(lane_of(Bl, l))),
                            __fmaf_rn(fabsf(lane_of(gv, l)), __fadd_rn(fabsf(lane_of(Fd, l)), fabsf(lane_of(Bu, l))),
                            __fmaf_rn(w2, __fadd_rn(fabsf(lane_of(Fdr, l)), fabsf(lane_of(Bul, l))),
                                      __fmul_rn(w3, __fadd_rn(fabsf(lane_of(Bur, l)), fabsf(lane_of(Fdl, l)))))));
            }
            scale = m;
        } else {
            // the candidates, s times these products
            const f2 pr[8] = {mul2(gu, Fr), mul2(gu, Bl), mul2(gv, Fd), mul2(gv, Bu),
                              mul2(n2, Fdr), mul2(n2, Bul), mul2(n3n, Bur), mul2(n3n, Fdl)};
            const f2 mag[8] = {Fr, Bl, Fd, Bu, Fdr, Bul, Bur, Fdl};
            float med[2];
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                float sv[8];
                float sent = __uint_as_float(0x7f800000u);  // the next sentinel: +inf, -inf, +inf, ...
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const bool kept = lane_of(mag[q], l) != 0.f;
                    sv[q] = kept ? lane_of(pr[q], l) : sent;
                    sent = kept ? sent : -sent;
                }
#define TFN_CE(i, j)                           \
    {                                          \
        const float lo_ = fminf(sv[i], sv[j]); \
        sv[j] = fmaxf(sv[i], sv[j]);           \
        sv[i] = lo_;                           \
    }
                TFN_CE(0, 2) TFN_CE(1, 3) TFN_CE(4, 6) TFN_CE(5, 7)
                TFN_CE(0, 4) TFN_CE(1, 5) TFN_CE(2, 6) TFN_CE(3, 7)
                TFN_CE(0, 1) TFN_CE(2, 3) TFN_CE(4, 5) TFN_CE(6, 7)
                TFN_CE(2, 4) TFN_CE(3, 5)
                TFN_CE(1, 4) TFN_CE(3, 6)
                TFN_CE(1, 2) TFN_CE(3, 4) TFN_CE(5, 6)
#undef TFN_CE
                // (the median of s times the products is s times theirs: the
                // sentinels keep the middle slots on the kept candidates)
                // the count of kept candidates, 8 minus the missing ones, is odd
                // when an odd number is missing: when the next sentinel is -inf
                const bool odd = sent < 0.f;
                const float md = odd ? sv[3] : __fmul_rn(0.5f, __fadd_rn(sv[3], sv[4]));
                med[l] = disp ? -md : md;
                if constexpr (!NOREF) mbound[l] = odd ? fabsf(sv[3]) : fmaxf(fabsf(sv[3]), fabsf(sv[4]));
            }
            mF = pk(med[0], med[1]);
            scale = bc(1.f);
        }
        const f2 A = fma2(uc2[h], gu, mul2(vc2, gv));
        const f2 nxp = PHI == PHI_MEAN ? mul2(mul2(scale, fx2), gu) : mul2(fx2, gu);
        const f2 nyp = PHI == PHI_MEAN ? mul2(mul2(scale, fy2), gv) : mul2(fy2, gv);
        const f2 Q = PHI == PHI_MEAN ? fma2(scale, A, mF) : add2(A, mF);  // -n_z'
        f2 nzp;
        if constexpr (one_pass) {
            // Sec. III special case without a test: n_z' = kFlatEps - Q.  A flat
            // pixel (G_u = G_v = 0) has n' = (0, 0, kFlatEps) exactly, so the
            // output below is exactly (0, 0, -1) (rsqrt of kFlatEps^2 = 2^-120 is
            // exact); any other pixel has |n'| >= m fx |G_u| or m fy |G_v|, far
            // above 2^-60, and nz' moves only where |Q| < 2^-35, by less than
            // 2^-33 of |n'|.  Every value here is finite for the one-pass
            // quotients, so a non-evaluable pixel is still zeroed through rs.
            nzp = sub2(bc(kFlatEps), Q);
        } else if constexpr (flat_by_bound) {
            // The same for the other means, whose non-evaluable pixels may
            // carry a NaN gradient part (from two hole taps) and so keep the
            // select on evaluability: the flat test's four compares go.
            nzp = pk(ev_ok[0] ? __fsub_rn(kFlatEps, Q.x) : 1.f, ev_ok[1] ? __fsub_rn(kFlatEps, Q.y) : 1.f);
        } else {
            // (a non-evaluable pixel's median may be a +-inf sentinel: keep n' finite so that rs = 0 zeroes it)
            nzp = pk((flat[0] || !ev_ok[0]) ? 1.f : -Q.x, (flat[1] || !ev_ok[1]) ? 1.f : -Q.y);
        }
        const f2 nn = fma2(nxp, nxp, fma2(nyp, nyp, mul2(nzp, nzp)));
        const f2 rs = pk(ev_ok[0] ? rsqrt_approx(nn.x) : 0.f, ev_ok[1] ? rsqrt_approx(nn.y) : 0.f);
        const f2 lim = NOREF ? bc(0.f) : mul2(bc(thr), mul2(nn, rs));
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const int k = h + 2 * l;
            const float r = lane_of(rs, l);
            // refine unless bound <= thr |n'|; written so that a NaN (|n'|
            // overflowed) also refines, and thr < 0 refines every pixel
            // (the means but the weighted family's: an evaluable pixel is flat
            // exactly when its bound is 0, every weight being 0; otherwise a
            // kept neighbour makes it > 0)
            const bool notflat = flat_by_bound ? mbound[l] > 0.f : !flat[l];
            const bool refine = !NOREF && ev_ok[l] && notflat && !(mbound[l] <= lane_of(lim, l));
            // -n'/|n'|, with +0 (not -0) for zero components and for non-evaluable pixels
            ox[k] = __fmaf_rn(-lane_of(nxp, l), r, 0.f);
            oy[k] = __fmaf_rn(-lane_of(nyp, l), r, 0.f);
            oz[k] = __fmaf_rn(-lane_of(nzp, l), r, 0.f);
            mword |= ev_ok[l] ? 1u << (8 * k) : 0u;
            rbits |= refine ? 1u << k : 0u;
        }

        // the carry for the pixels below: their up, up-left and up-right neighbours
        cy.put(h, mul2(disp ? Nc : Cc, ev.r), mul2(disp ? Nc : Cl, edm.r), mul2(disp ? Nc : Cr, ea.r),
               fma2(ev.d, ev.r, fma2(edm.d, edm.r, mul2(ea.d, ea.r))));
        // this pair's edges to column c+1 are the next pair's to column c-1
        ehm = eh;
        edm = ed;
        eam = ea;
    }
    if (GRAD != GRAD_FD && cy.ring) cy.p0 = cy.p0 == 2 ? 0 : cy.p0 + 1;  // (the ring: C becomes P)
}

// ------------------------------------------------------------ 5x5 filters
//
// The separable 5x5 gradient filters: an antisymmetric derivative profile
// (d1 at offsets +-1, d2 at +-2) along the filter's axis times a symmetric
// smoothing profile (s0, s1, s2) across it.  As each sample row arrives, a
// lane computes at its 4 columns the row's derivative Dh = d1 (w_{+1} -
// w_{-1}) + d2 (w_{+2} - w_{-2}) and smoothing Sh = s0 w_0 + s1 (w_{-1} +
// w_{+1}) + s2 (w_{-2} + w_{+2}) (w = 1/Z or the disparity), both as
// unnormalised double-float pairs (exact tap differences, then the dfl_
// operations), and keeps them for 5 rows; then G_u = sum_a s_|a| Dh(y + a)
// and G_v = d1 (Sh(y+1) - Sh(y-1)) + d2 (Sh(y+2) - Sh(y-2)), renormalised
// once at the end.  The common
// normalisation is dropped (it cancels from the direction).  A value whose
// needed taps include a hole is NaN, which marks the pixels that use it as
// not evaluable; zero-weight terms are never read.

struct Sep5W {
    float d1, d2, s0, s1, s2;
};

__device__ __forceinline__ float f4_at(const float4 &v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }

__device__ __forceinline__ df df_nan() { return {__int_as_float(0x7fc00000), __int_as_float(0x7fc00000)}; }

// One sample row of a lane's 5x5 window: image columns x0-2 .. x0+5.
template <int KIND, int BOXW, int PADX>
__device__ __forceinline__ void load_row8(const unsigned char *stage, int jr, int lane, float (&z)[8])
{
    typedef typename KindTraits<KIND>::T T;
    static_assert(PADX >= 2, "the box halo must hold 2 columns");
    const T *p = reinterpret_cast<const T *>(stage) + jr * BOXW + PADX + 4 * lane;
    T raw[8];
    raw[0] = p[-2];
    raw[1] = p[-1];
    if constexpr (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        raw[2] = q.x;
        raw[3] = q.y;
        raw[4] = q.z;
        raw[5] = q.w;
    } else {
        const uint2 q = *reinterpret_cast<const uint2 *>(p);
        raw[2] = from_bits16<T>(q.x & 0xffffu);
        raw[3] = from_bits16<T>(q.x >> 16);
        raw[4] = from_bits16<T>(q.y & 0xffffu);
        raw[5] = from_bits16<T>(q.y >> 16);
    }
    raw[6] = p[4];
    raw[7] = p[5];
#pragma unroll
    for (int c = 0; c < 8; ++c) z[c] = decode<KIND>(raw[c]);
}

// Dh and Sh of one sample row at the lane's 4 columns (sample c + 2 of z is
// column x0 + c).
template <int KIND>
__device__ __forceinline__ void sep5_row(const float (&z)[8], const Sep5W &w, df (&Dh)[4], df (&Sh)[4])
{
    float wh[8], wl[8];
    bool ok[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        ok[i] = z[i] <= kValidHi;
        if constexpr (KindTraits<KIND>::disparity) {
            wh[i] = z[i];
            wl[i] = 0.f;
        } else {  // 1/Z as wh + wl: hardware reciprocal plus its FMA residual
            wh[i] = rcp_approx(z[i]);
            wl[i] = __fmul_rn(__fmaf_rn(-wh[i], z[i], 1.f), wh[i]);
        }
    }
    // w_b - w_a, exact up to the low parts' rounding
    auto diff = [&](int a, int b) -> df {
        if constexpr (KindTraits<KIND>::exact_diff) {
            return {__fsub_rn(wh[b], wh[a]), 0.f};
        } else {
            const df h = two_sum(wh[b], -wh[a]);
            return {h.h, __fadd_rn(h.l, __fsub_rn(wl[b], wl[a]))};
        }
    };
    auto val = [&](int a) -> df { return {wh[a], wl[a]}; };
    const df zero = {0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int c = k + 2;
        const bool ok1 = ok[c - 1] && ok[c + 1], ok2 = ok[c - 2] && ok[c + 2];
        // (unnormalised pairs: the ring keeps them so, the vertical sums renormalise)
        const df t1 = w.d1 != 0.f ? dfl_mul_f(diff(c - 1, c + 1), w.d1) : zero;
        const df t2 = w.d2 != 0.f ? dfl_mul_f(diff(c - 2, c + 2), w.d2) : zero;
        const bool dok = (w.d1 == 0.f || ok1) && (w.d2 == 0.f || ok2);
        Dh[k] = dok ? dfl_add(t1, t2) : df_nan();
        const df a0 = w.s0 != 0.f ? dfl_mul_f(val(c), w.s0) : zero;
        const df a1 = w.s1 != 0.f ? dfl_mul_f(dfl_add(val(c - 1), val(c + 1)), w.s1) : zero;
        const df a2 = w.s2 != 0.f ? dfl_mul_f(dfl_add(val(c - 2), val(c + 2)), w.s2) : zero;
        const bool sok = (w.s0 == 0.f || ok[c]) && (w.s1 == 0.f || ok1) && (w.s2 == 0.f || ok2);
        Sh[k] = sok ? dfl_add(a0, dfl_add(a1, a2)) : df_nan();
    }
}

// ------------------------------------------------------------ PlanePCA
//
// The comparison estimator of Sec. II-A (Eq. planepca): the normal is the
// eigenvector of the smallest eigenvalue of the scatter matrix of the 9
// back-projected points of the 3x3 neighbourhood, centred on their mean,
// turned to face the camera.  The points are taken relative to the centre
// pixel's in the algebraic form (dx = (dz (u - u0) + Z_j du)/fx, likewise dy,
// with dz = Z_j - Z_i exact for depths within a factor 2, or computed as
// f t_c (d_i - d_j)/(d_i d_j) for disparity), so that the FP32 coordinates
// keep their accuracy relative to the neighbourhood's size.  The smallest
// eigenvalue comes from Newton's method on the characteristic polynomial
// started at 0 (below it; the iterates rise monotonically to it), and the
// eigenvector from the largest cross product of two rows of M - lambda I.

constexpr int kPcaNewton = 12;

template <int KIND>
__device__ __forceinline__ void pca_pixel(const float (&w)[3][3], float uc, float vc, float rfx, float rfy, float ztc,
                                          float &nx, float &ny, float &nz, bool &ok)
{
    ok = fmaxf(fmaxf(fmaxf(w[0][0], w[0][1]), fmaxf(w[0][2], w[1][0])),
               fmaxf(fmaxf(w[1][1], w[1][2]), fmaxf(fmaxf(w[2][0], w[2][1]), w[2][2]))) <= kValidHi;
    const float si = w[1][1];
    float rx[9], ry[9], rz[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int j = 3 * a + b;
            const float sj = w[a][b];
            float dz, Zj;
            if constexpr (KindTraits<KIND>::disparity) {
                // Z = ztc / s: dz = ztc (s_i - s_j) / (s_i s_j)
                Zj = __fdiv_rn(ztc, sj);
                dz = __fdiv_rn(__fmul_rn(ztc, __fsub_rn(si, sj)), __fmul_rn(si, sj));
            } else {
                Zj = sj;
                dz = __fsub_rn(sj, si);
            }
            const float du = (float)(b - 1), dv = (float)(a - 1);
            rx[j] = __fmul_rn(__fmaf_rn(dz, uc, __fmul_rn(du, Zj)), rfx);
            ry[j] = __fmul_rn(__fmaf_rn(dz, vc, __fmul_rn(dv, Zj)), rfy);
            rz[j] = dz;
        }
    float mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        mx = __fadd_rn(mx, rx[j]);
        my = __fadd_rn(my, ry[j]);
        mz = __fadd_rn(mz, rz[j]);
    }
    const float r9 = 1.f / 9.f;
    mx = __fmul_rn(mx, r9);
    my = __fmul_rn(my, r9);
    mz = __fmul_rn(mz, r9);
    float m00 = 0.f, m01 = 0.f, m02 = 0.f, m11 = 0.f, m12 = 0.f, m22 = 0.f;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const float x = __fsub_rn(rx[j], mx), y = __fsub_rn(ry[j], my), z = __fsub_rn(rz[j], mz);
        m00 = __fmaf_rn(x, x, m00);
        m01 = __fmaf_rn(x, y, m01);
        m02 = __fmaf_rn(x, z, m02);
        m11 = __fmaf_rn(y, y, m11);
        m12 = __fmaf_rn(y, z, m12);
        m22 = __fmaf_rn(z, z, m22);
    }
    // trace 1 (the direction does not depend on the scale; this keeps the
    // cubic's coefficients in range)
    const float tr = __fadd_rn(__fadd_rn(m00, m11), m22);
    const float s = ok && tr > 0.f ? __frcp_rn(tr) : 0.f;
    m00 = __fmul_rn(m00, s);
    m01 = __fmul_rn(m01, s);
    m02 = __fmul_rn(m02, s);
    m11 = __fmul_rn(m11, s);
    m12 = __fmul_rn(m12, s);
    m22 = __fmul_rn(m22, s);
    // det(M - l I) = c0 - c1 l + c2 l^2 - l^3, c2 = 1
    const float k0 = __fmaf_rn(m11, m22, -__fmul_rn(m12, m12));
    const float k1 = __fmaf_rn(m01, m22, -__fmul_rn(m12, m02));
    const float k2 = __fmaf_rn(m01, m12, -__fmul_rn(m11, m02));
    const float c0 = __fmaf_rn(m00, k0, __fmaf_rn(-m01, k1, __fmul_rn(m02, k2)));
    const float c1 = __fadd_rn(__fadd_rn(k0, __fmaf_rn(m00, m22, -__fmul_rn(m02, m02))),
                               __fmaf_rn(m00, m11, -__fmul_rn(m01, m01)));
    float l = 0.f;
#pragma unroll
    for (int it = 0; it < kPcaNewton; ++it) {
        const float p = __fmaf_rn(-l, __fmaf_rn(-l, __fsub_rn(1.f, l), c1), c0);  // c0 - l (c1 - l (1 - l))
        const float dp = __fmaf_rn(l, __fmaf_rn(-3.f, l, 2.f), -c1);               // -c1 + l (2 - 3 l)
        l = dp < 0.f ? __fmaf_rn(-p, rcp_approx(dp), l) : l;  // (the step need not be exact: the Rayleigh step below fixes l)
    }
    // The eigenvector of an eigenvalue l: the largest cross product of two
    // rows of A = M - l I, normalised.
    auto vec_for = [&](float lv, float &x, float &y, float &z) {
        const float a00 = __fsub_rn(m00, lv), a11 = __fsub_rn(m11, lv), a22 = __fsub_rn(m22, lv);
        float v[3][3];
        // a0 x a1, a0 x a2, a1 x a2 with a0 = (a00, m01, m02), a1 = (m01, a11, m12), a2 = (m02, m12, a22)
        v[0][0] = __fmaf_rn(m01, m12, -__fmul_rn(m02, a11));
        v[0][1] = __fmaf_rn(m02, m01, -__fmul_rn(a00, m12));
        v[0][2] = __fmaf_rn(a00, a11, -__fmul_rn(m01, m01));
        v[1][0] = __fmaf_rn(m01, a22, -__fmul_rn(m02, m12));
        v[1][1] = __fmaf_rn(m02, m02, -__fmul_rn(a00, a22));
        v[1][2] = __fmaf_rn(a00, m12, -__fmul_rn(m01, m02));
        v[2][0] = __fmaf_rn(a11, a22, -__fmul_rn(m12, m12));
        v[2][1] = __fmaf_rn(m12, m02, -__fmul_rn(m01, a22));
        v[2][2] = __fmaf_rn(m01, m12, -__fmul_rn(a11, m02));
        float best = -1.f;
        x = 0.f, y = 0.f, z = 1.f;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float n2 = __fmaf_rn(v[q][0], v[q][0], __fmaf_rn(v[q][1], v[q][1], __fmul_rn(v[q][2], v[q][2])));
            const bool take = n2 > best;
            best = take ? n2 : best;
            x = take ? v[q][0] : x;
            y = take ? v[q][1] : y;
            z = take ? v[q][2] : z;
        }
        const float rs = ok && best > 0.f ? rsqrt_approx(best) : 0.f;
        x = __fmul_rn(x, rs);
        y = __fmul_rn(y, rs);
        z = __fmul_rn(z, rs);
    };
    // its Rayleigh quotient b^T M b / b^T b, never below the smallest eigenvalue
    auto rayleigh = [&](float x, float y, float z) -> float {
        const float mbx = __fmaf_rn(m00, x, __fmaf_rn(m01, y, __fmul_rn(m02, z)));
        const float mby = __fmaf_rn(m01, x, __fmaf_rn(m11, y, __fmul_rn(m12, z)));
        const float mbz = __fmaf_rn(m02, x, __fmaf_rn(m12, y, __fmul_rn(m22, z)));
        const float num = __fmaf_rn(x, mbx, __fmaf_rn(y, mby, __fmul_rn(z, mbz)));
        const float den = __fmaf_rn(x, x, __fmaf_rn(y, y, __fmul_rn(z, z)));
        return den > 0.f ? __fmul_rn(num, rcp_approx(den)) : 0.f;  // (den is 1 to a few u: no exact division)
    };
    // Two candidates: the vector of the Newton eigenvalue, and that of l = 0
    // (the adjugate's largest column).  det(M) carries an absolute error of
    // about u tr^3, which can throw the cubic's root past lambda_2 when
    // lambda_2 / tr is below about u^(1/2) (a window across a steep slope);
    // l = 0 is then the better start.  The candidate nearer the smallest
    // eigenvector has the smaller Rayleigh quotient.  Two steps of l = the
    // Rayleigh quotient, then the cross products again, refine it.
    float xn, yn, zn, x0, y0, z0;
    vec_for(l, xn, yn, zn);
    vec_for(0.f, x0, y0, z0);
    const float qn = rayleigh(xn, yn, zn), q0 = rayleigh(x0, y0, z0);
    const bool newton = qn <= q0;
    float bx = newton ? xn : x0, by = newton ? yn : y0, bz = newton ? zn : z0;
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) vec_for(rayleigh(bx, by, bz), bx, by, bz);
    // face the camera: n . (uc / fx, vc / fy, 1) < 0; ties by n_z, n_y, n_x < 0
    const float d = __fmaf_rn(bx, __fmul_rn(uc, rfx), __fmaf_rn(by, __fmul_rn(vc, rfy), bz));
    const float key = d != 0.f ? d : bz != 0.f ? bz : by != 0.f ? by : bx;
    const float sg = key > 0.f ? -1.f : 1.f;
    // (a non-evaluable pixel's arithmetic may have overflowed: its output is 0)
    nx = ok ? __fmaf_rn(sg, bx, 0.f) : 0.f;
    ny = ok ? __fmaf_rn(sg, by, 0.f) : 0.f;
    nz = ok ? __fmaf_rn(sg, bz, 0.f) : 0.f;
}

// A lane's 4 pixels of one row by PlanePCA (P, C, N: the sample rows above,
// at and below; uc = u - u0 per column, vc = v - v0).
template <int KIND, int GRAD>
__device__ __forceinline__ void pca_row(const Row<KIND, GRAD> &P, const Row<KIND, GRAD> &C, const Row<KIND, GRAD> &N,
                                        const float (&uc)[4], float vc, float rfx, float rfy, float ztc,
                                        float (&ox)[4], float (&oy)[4], float (&oz)[4], uint32_t &mword)
{
    mword = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int c = k + 1;
        const float w[3][3] = {{P.z[c - 1], P.z[c], P.z[c + 1]},
                               {C.z[c - 1], C.z[c], C.z[c + 1]},
                               {N.z[c - 1], N.z[c], N.z[c + 1]}};
        bool ok;
        pca_pixel<KIND>(w, uc[k], vc, rfx, rfy, ztc, ox[k], oy[k], oz[k], ok);
        mword |= ok ? 1u << (8 * k) : 0u;
    }
}

// ------------------------------------------------------------ TMA / mbarrier

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bounded wait for the phase with parity `phase`; false if it did not
// complete within kWaitCycles.
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t phase)
{
    uint32_t done;
    // the suspend-time hint (ns) lets a waiting warp sleep instead of spinning
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(bar), "r"(phase), "r"(20000)
        : "memory");
    return done != 0;
}

// Bounded wait for the phase with parity `phase`; false if it did not
// complete within kWaitCycles (the clock is read every 16 polls).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, long long limit = kWaitCycles)
{
    if (mbar_try(bar, phase)) return true;
    const long long t0 = clock64();
    for (;;) {
#pragma unroll 1
        for (int k = 0; k < 16; ++k)
            if (mbar_try(bar, phase)) return true;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void fence_tensormap_acquire(const CUtensorMap *map)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}

__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ------------------------------------------------------------ stores

// Where a tile's results go (copied to registers once per tile).
struct OutDesc {
    char *out;
    int64_t out_pitch, out_plane;
    uint8_t *mask;
    int64_t mask_pitch;
};

__device__ __forceinline__ uint32_t pack2(float a, float b, int fmt)
{
    if (fmt == OUT_F16 || fmt == OUT_F16X4) {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// Octahedral code of a unit normal (Cigolle et al., JCGT 2014, the "oct"
// map): p = (x, y) / (|x| + |y| + |z|), folded over the square's corners where
// z < 0 (sign +1 for 0), each component as round-to-nearest-even(p * 32767),
// packed as two int16 (x in the low half).  The zero vector of a
// non-evaluable pixel gives (0, 0).
__device__ __forceinline__ uint32_t oct16(float x, float y, float z)
{
    const float s = __fadd_rn(__fadd_rn(fabsf(x), fabsf(y)), fabsf(z));
    const float is = s > 0.f ? rcp_approx(s) : 0.f;
    const float px = __fmul_rn(x, is), py = __fmul_rn(y, is);
    float qx = px, qy = py;
    if (z < 0.f) {
        qx = px >= 0.f ? __fsub_rn(1.f, fabsf(py)) : -__fsub_rn(1.f, fabsf(py));
        qy = py >= 0.f ? __fsub_rn(1.f, fabsf(px)) : -__fsub_rn(1.f, fabsf(px));
    }
    const int cx = __float2int_rn(__fmul_rn(fminf(fmaxf(qx, -1.f), 1.f), 32767.f));
    const int cy = __float2int_rn(__fmul_rn(fminf(fmaxf(qy, -1.f), 1.f), 32767.f));
    return ((uint32_t)cx & 0xffffu) | ((uint32_t)cy << 16);
}

// Back-projected points of 4 consecutive pixels of row v (n of them inside
// the frame f): Z = the sample (disparity: ztc / sample), X = Z (u - u0)/fx,
// Y = Z (v - v0)/fy; holes give (0, 0, 0).  Out of line, reading what it
// needs from the frame's descriptor, so that the row loop keeps neither the
// code nor the registers of this rare output.
template <int KIND>
__device__ __noinline__ void store_points4(const FrameDesc *f, int u, int v, int n, float z1, float z2, float z3,
                                           float z4)
{
    char *pts = (char *)__ldg((const unsigned long long *)&f->pts);
    const int64_t pitch = __ldg(&f->pts_pitch), plane = __ldg(&f->pts_plane);
    const float fx = __ldg(&f->fx), fy = __ldg(&f->fy), u0 = __ldg(&f->u0), v0 = __ldg(&f->v0);
    const float ztc = __ldg(&f->ztc);
    const float z[4] = {z1, z2, z3, z4};
    const float vcf = __fdiv_rn(__fsub_rn((float)v, v0), fy);
    float X[4], Y[4], Z[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float ucf = __fdiv_rn(__fsub_rn((float)(u + k), u0), fx);
        const float s = z[k];
        const bool ok = s <= kValidHi;
        const float Zk = KindTraits<KIND>::disparity ? __fdiv_rn(ztc, s) : s;
        X[k] = ok ? __fmul_rn(Zk, ucf) : 0.f;
        Y[k] = ok ? __fmul_rn(Zk, vcf) : 0.f;
        Z[k] = ok ? Zk : 0.f;
    }
    char *row = pts + (int64_t)v * pitch;
    if (n == 4) {
        __stcs(reinterpret_cast<float4 *>(row + (int64_t)u * 4), make_float4(X[0], X[1], X[2], X[3]));
        __stcs(reinterpret_cast<float4 *>(row + plane + (int64_t)u * 4), make_float4(Y[0], Y[1], Y[2], Y[3]));
        __stcs(reinterpret_cast<float4 *>(row + 2 * plane + (int64_t)u * 4), make_float4(Z[0], Z[1], Z[2], Z[3]));
        return;
    }
    for (int k = 0; k < n; ++k) {
        reinterpret_cast<float *>(row)[u + k] = X[k];
        reinterpret_cast<float *>(row + plane)[u + k] = Y[k];
        reinterpret_cast<float *>(row + 2 * plane)[u + k] = Z[k];
    }
}

// Stores 4 consecutive pixels (n valid of them, starting at column u) in the
// rarer cases (octahedral and packed layouts, a row's last pixels): out of
// line, so that the row loop's code stays small (the row loop is bound by
// instruction issue and fetch).
static __device__ __noinline__ void store4_cold(OutDesc fd, int fmt, int u, int v, int n, float x0, float x1, float x2, float x3,
                                        float y0, float y1, float y2, float y3, float z0, float z1, float z2, float z3,
                                        uint32_t mw)
{
    const float x[4] = {x0, x1, x2, x3}, y[4] = {y0, y1, y2, y3}, zz[4] = {z0, z1, z2, z3};
    char *row = fd.out + (int64_t)v * fd.out_pitch;
    uint8_t *mrow = fd.mask + (int64_t)v * fd.mask_pitch;
    if (n == 4) {
        if (fmt == OUT_F32) {
            __stcs(reinterpret_cast<float4 *>(row + (int64_t)u * 4), make_float4(x[0], x[1], x[2], x[3]));
            __stcs(reinterpret_cast<float4 *>(row + fd.out_plane + (int64_t)u * 4), make_float4(y[0], y[1], y[2], y[3]));
            __stcs(reinterpret_cast<float4 *>(row + 2 * fd.out_plane + (int64_t)u * 4),
                   make_float4(zz[0], zz[1], zz[2], zz[3]));
        } else if (fmt == OUT_OCT16) {
            __stcs(reinterpret_cast<uint4 *>(row + (int64_t)u * 4),
                   make_uint4(oct16(x[0], y[0], zz[0]), oct16(x[1], y[1], zz[1]), oct16(x[2], y[2], zz[2]),
                              oct16(x[3], y[3], zz[3])));
        } else if (fmt == OUT_F16 || fmt == OUT_BF16) {
            __stcs(reinterpret_cast<uint2 *>(row + (int64_t)u * 2), make_uint2(pack2(x[0], x[1], fmt), pack2(x[2], x[3], fmt)));
            __stcs(reinterpret_cast<uint2 *>(row + fd.out_plane + (int64_t)u * 2),
                   make_uint2(pack2(y[0], y[1], fmt), pack2(y[2], y[3], fmt)));
            __stcs(reinterpret_cast<uint2 *>(row + 2 * fd.out_plane + (int64_t)u * 2),
                   make_uint2(pack2(zz[0], zz[1], fmt), pack2(zz[2], zz[3], fmt)));
        } else {
            uint4 a = make_uint4(pack2(x[0], y[0], fmt), pack2(zz[0], 0.f, fmt), pack2(x[1], y[1], fmt),
                                 pack2(zz[1], 0.f, fmt));
            uint4 b = make_uint4(pack2(x[2], y[2], fmt), pack2(zz[2], 0.f, fmt), pack2(x[3], y[3], fmt),
                                 pack2(zz[3], 0.f, fmt));
            __stcs(reinterpret_cast<uint4 *>(row + (int64_t)u * 8), a);
            __stcs(reinterpret_cast<uint4 *>(row + (int64_t)u * 8 + 16), b);
        }
        __stcs(reinterpret_cast<unsigned int *>(mrow + u), mw);
        return;
    }
    for (int k = 0; k < n; ++k) {
        const int uu = u + k;
        if (fmt == OUT_F32) {
            reinterpret_cast<float *>(row)[uu] = x[k];
            reinterpret_cast<float *>(row + fd.out_plane)[uu] = y[k];
            reinterpret_cast<float *>(row + 2 * fd.out_plane)[uu] = zz[k];
        } else if (fmt == OUT_OCT16) {
            reinterpret_cast<uint32_t *>(row)[uu] = oct16(x[k], y[k], zz[k]);
        } else if (fmt == OUT_F16 || fmt == OUT_BF16) {
            const uint32_t px = pack2(x[k], y[k], fmt), pz = pack2(zz[k], 0.f, fmt);
            reinterpret_cast<uint16_t *>(row)[uu] = (uint16_t)(px & 0xffff);
            reinterpret_cast<uint16_t *>(row + fd.out_plane)[uu] = (uint16_t)(px >> 16);
            reinterpret_cast<uint16_t *>(row + 2 * fd.out_plane)[uu] = (uint16_t)(pz & 0xffff);
        } else {
            reinterpret_cast<uint2 *>(row)[uu] = make_uint2(pack2(x[k], y[k], fmt), pack2(zz[k], 0.f, fmt));
        }
        mrow[uu] = (uint8_t)(mw >> (8 * k));
    }
}

// Normals and mask of a full quad of row v in a planar layout (fmt OUT_F32,
// OUT_F16 or OUT_BF16).
__device__ __forceinline__ void store4_planar(const OutDesc &fd, int fmt, int u, int v, const float (&x)[4],
                                              const float (&y)[4], const float (&zz)[4], uint32_t mw)
{
    char *row = fd.out + (int64_t)v * fd.out_pitch;
    uint8_t *mrow = fd.mask + (int64_t)v * fd.mask_pitch;
    if (fmt == OUT_F32) {
        __stcs(reinterpret_cast<float4 *>(row + (int64_t)u * 4), make_float4(x[0], x[1], x[2], x[3]));
        __stcs(reinterpret_cast<float4 *>(row + fd.out_plane + (int64_t)u * 4), make_float4(y[0], y[1], y[2], y[3]));
        __stcs(reinterpret_cast<float4 *>(row + 2 * fd.out_plane + (int64_t)u * 4), make_float4(zz[0], zz[1], zz[2], zz[3]));
    } else {
        // (one branch on the launch's format, so that each pair is converted once)
        auto put = [&](int ff) {
            __stcs(reinterpret_cast<uint2 *>(row + (int64_t)u * 2), make_uint2(pack2(x[0], x[1], ff), pack2(x[2], x[3], ff)));
            __stcs(reinterpret_cast<uint2 *>(row + fd.out_plane + (int64_t)u * 2),
                   make_uint2(pack2(y[0], y[1], ff), pack2(y[2], y[3], ff)));
            __stcs(reinterpret_cast<uint2 *>(row + 2 * fd.out_plane + (int64_t)u * 2),
                   make_uint2(pack2(zz[0], zz[1], ff), pack2(zz[2], zz[3], ff)));
        };
        if (fmt == OUT_F16)
            put(OUT_F16);
        else
            put(OUT_BF16);
    }
    __stcs(reinterpret_cast<unsigned int *>(mrow + u), mw);
}

// Normals and mask of 4 pixels of row v: FP32 and FP16/BF16 planar full
// quads inline, everything else through store4_cold.
__device__ __forceinline__ void store4(const OutDesc &fd, int fmt, int u, int v, int n, const float (&x)[4],
                                       const float (&y)[4], const float (&zz)[4], uint32_t mw)
{
    if (n == 4 && fmt <= OUT_BF16) {
        store4_planar(fd, fmt, u, v, x, y, zz, mw);
        return;
    }
    store4_cold(fd, fmt, u, v, n, x[0], x[1], x[2], x[3], y[0], y[1], y[2], y[3], zz[0], zz[1], zz[2], zz[3], mw);
}


// Stores one pixel's normal (the mask is already written).
__device__ __forceinline__ void store1(const OutDesc &fd, int fmt, int u, int v, Vec3 n)
{
    char *row = fd.out + (int64_t)v * fd.out_pitch;
    if (fmt == OUT_F32) {
        reinterpret_cast<float *>(row)[u] = n.x;
        reinterpret_cast<float *>(row + fd.out_plane)[u] = n.y;
        reinterpret_cast<float *>(row + 2 * fd.out_plane)[u] = n.z;
    } else if (fmt == OUT_OCT16) {
        reinterpret_cast<uint32_t *>(row)[u] = oct16(n.x, n.y, n.z);
    } else if (fmt == OUT_F16 || fmt == OUT_BF16) {
        const uint32_t px = pack2(n.x, n.y, fmt), pz = pack2(n.z, 0.f, fmt);
        reinterpret_cast<uint16_t *>(row)[u] = (uint16_t)(px & 0xffff);
        reinterpret_cast<uint16_t *>(row + fd.out_plane)[u] = (uint16_t)(px >> 16);
        reinterpret_cast<uint16_t *>(row + 2 * fd.out_plane)[u] = (uint16_t)(pz & 0xffff);
    } else {
        reinterpret_cast<uint2 *>(row)[u] = make_uint2(pack2(n.x, n.y, fmt), pack2(n.z, 0.f, fmt));
    }
}

// The double-float path for pixel (x, y), reading its 3x3 window again from
// the input image (taps outside the image and holes are invalid).  Called
// for the rare refined pixels after a work item's rows are done, so that the
// main loop never waits on it.
template <int KIND, int GRAD, int PHI>
__device__ __noinline__ Vec3 refine_from_input(const void *in, int64_t pitch, int H, int W, int x, int y, float fx,
                                               float fy, float u0, float v0, float w0, float w1, float w2)
{
    typedef typename KindTraits<KIND>::T T;
    float z[9];
    unsigned okb = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int yy = y - 1 + a, xx = x - 1 + b;
            float v = kHole;
            if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                v = decode<KIND>(reinterpret_cast<const T *>(static_cast<const char *>(in) + (int64_t)yy * pitch)[xx]);
            z[3 * a + b] = v;
            okb |= (v <= kValidHi ? 1u : 0u) << (3 * a + b);
        }
    return refine_pixel<KIND, GRAD, PHI>(z[0], z[1], z[2], z[3], z[4], z[5], z[6], z[7], z[8], okb, x, y, fx, fy, u0,
                                         v0, w0, w1, w2);
}

// The same for a 5x5 filter: the gradients from the 5x5 window in
// double-float (per row or column the weighted differences of the taps at
// +-1 and +-2, then the smoothing profile across), then the candidates of
// the 3x3 window.  Zero-weight taps are never read.
template <int KIND, int PHI>
__device__ __noinline__ Vec3 refine_from_input_sep5(const void *in, int64_t pitch, int H, int W, int x, int y, float fx,
                                                    float fy, float u0, float v0, float d1, float d2, float s0,
                                                    float s1, float s2)
{
    typedef typename KindTraits<KIND>::T T;
    float z[5][5];
    for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b) {
            const int yy = y - 2 + a, xx = x - 2 + b;
            float v = kHole;
            if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                v = decode<KIND>(reinterpret_cast<const T *>(static_cast<const char *>(in) + (int64_t)yy * pitch)[xx]);
            z[a][b] = v;
        }
    const float sw[5] = {s2, s1, s0, s1, s2};
    df Gu = {0.f, 0.f}, Gv = {0.f, 0.f};
    for (int a = 0; a < 5; ++a) {
        if (sw[a] == 0.f) continue;
        df hu = {0.f, 0.f}, hv = {0.f, 0.f};
        if (d1 != 0.f) {
            hu = df_add(hu, df_mul_f(grad_term<KIND>(z[a][1], z[a][3]), d1));
            hv = df_add(hv, df_mul_f(grad_term<KIND>(z[1][a], z[3][a]), d1));
        }
        if (d2 != 0.f) {
            hu = df_add(hu, df_mul_f(grad_term<KIND>(z[a][0], z[a][4]), d2));
            hv = df_add(hv, df_mul_f(grad_term<KIND>(z[0][a], z[4][a]), d2));
        }
        Gu = df_add(Gu, df_mul_f(hu, sw[a]));
        Gv = df_add(Gv, df_mul_f(hv, sw[a]));
    }
    float zi[3][3];
    bool ok[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            zi[a][b] = z[a + 1][b + 1];
            ok[a][b] = zi[a][b] <= kValidHi;
        }
    return refine_candidates<KIND, PHI>(zi, ok, Gu, Gv, x, y, fx, fy, u0, v0);
}

// ------------------------------------------------------------ item -> frame

// frame_of (tfn_items.h) over the launch's frame descriptors.
__device__ __forceinline__ int frame_of_item(const FrameDesc *frames, int nframes, int t, int from)
{
    return frame_of([frames](int i) { return __ldg(&frames[i].tile_begin); }, nframes, t, from);
}

// ------------------------------------------------------------ refinement list
//
// Except for the FD mean and the short items of small launches, which refine
// in the main kernel (see normals_kernel), the main kernel does not refine: a
// pixel whose FP32 error bound is too loose keeps its FP32 normal, gets bit 1
// set in its mask byte, and is appended to the launch's refinement list
// (frame index << 32 | y << 16 | x).  refine_kernel, launched after it on the
// same stream, redoes the listed pixels in double-float and clears their bit,
// and its last block zeroes the count for the list's next launch.  Keeping
// the double-float code out of the row loop's kernel leaves that loop its
// registers and instruction cache.  A list that overflows its capacity is not
// lost: the count still grows, and refine_kernel then finds the flagged pixels
// by their mask bit instead.

// Appends the flagged pixels (bit k of rb: column x0 + k) of row y of frame fi.
static __device__ __noinline__ void list_for_refinement(unsigned long long *rlist, unsigned long long *rcount, int rcap,
                                                 int fi, int x0, int y, unsigned rb)
{
    const unsigned long long base = atomicAdd(rcount, (unsigned long long)__popc(rb));
    const unsigned long long e0 = ((unsigned long long)(unsigned)fi << 32) | ((unsigned)y << 16) | (unsigned)x0;
    for (unsigned long long j = base; rb; ++j, rb &= rb - 1u)
        if (j < (unsigned long long)rcap) rlist[j] = e0 + (unsigned)(__ffs(rb) - 1);
}

// Refines one flagged pixel (x, y) of frame fi of the launch, and clears its
// mask bit 1 when CLEAR (the refinement kernel's pixels; a kernel that refines
// its own pixels never sets the bit).
template <int KIND, int GRAD, int PHI, bool CLEAR>
__device__ __forceinline__ void refine_at(const LaunchArgs &args, int fi, int x, int y)
{
    const FrameDesc *f = args.frames + fi;
    OutDesc out;
    out.out = (char *)__ldg((const unsigned long long *)&f->out);
    out.out_pitch = __ldg(&f->out_pitch);
    out.out_plane = __ldg(&f->out_plane);
    out.mask = (uint8_t *)__ldg((const unsigned long long *)&f->mask);
    out.mask_pitch = __ldg(&f->mask_pitch);
    const void *in = (const void *)__ldg((const unsigned long long *)&f->in);
    const int64_t in_pitch = __ldg(&f->in_pitch);
    const int H = __ldg(&f->H), W = __ldg(&f->W);
    const float fx = __ldg(&f->fx), fy = __ldg(&f->fy), u0 = __ldg(&f->u0), v0 = __ldg(&f->v0);
    Vec3 nr;
    if constexpr (GRAD == GRAD_SEP5)
        nr = refine_from_input_sep5<KIND, PHI>(in, in_pitch, H, W, x, y, fx, fy, u0, v0, args.w[0], args.w[1],
                                               args.w[2], args.w[3], args.w[4]);
    else
        nr = refine_from_input<KIND, GRAD, PHI>(in, in_pitch, H, W, x, y, fx, fy, u0, v0, args.w[0], args.w[1],
                                                args.w[2]);
    store1(out, args.out_fmt, x, y, nr);
    if (CLEAR) out.mask[(int64_t)y * out.mask_pitch + x] = 1;
}

// ------------------------------------------------------------ the kernel

// Persistent kernel of independent warps.  The work item is a band of 128
// pixel columns x TH rows of one frame (items are numbered frame by frame,
// row band by row band, left to right); warp w of the grid takes items w,
// w + W, w + 2W, ... (W warps in the grid).  A lane owns 4 adjacent columns
// and rolls down the item's rows with three sample rows in registers, so the
// edges between two rows are computed once for both.  Each warp streams its
// items' rows through a ring of NST shared-memory stages of CR rows each
// (box: 128 columns plus a 16-byte halo on each side), filled by TMA 2D
// copies that lane 0 issues and completed on one mbarrier per stage; a stage
// is refilled with the chunk NST ahead as soon as the warp has read its last
// row.  No warp ever waits for another.  The TMA zero fill outside the frame
// (above the first row, past the last, beyond the edges) reads as holes, so
// borders need no special case.
template <int KIND, int GRAD, int PHI, int CFG, bool NOREF>
__global__ void __launch_bounds__(32 * cta_warps(CFG, GRAD), grad_is_pair(GRAD) ? ctas3_per_sm(CFG) : 0)
    normals_kernel(const __grid_constant__ LaunchArgs args)
{
    static_assert(!NOREF || (GRAD == GRAD_FD && KIND == KIND_DEPTH_F16), "only FP16 depth with FD has a NOREF form");
    typedef typename KindTraits<KIND>::T T;
    typedef Row<KIND, GRAD> R;
    constexpr int TH = kCfgs[CFG].th, CR = kCfgs[CFG].cr, NST = cfg_nst(CFG, GRAD), NW = cta_warps(CFG, GRAD);
    constexpr bool SEP5 = GRAD == GRAD_SEP5;
    // the short-item shape (launches of few items, e.g. one frame) refines
    // in place at the end of each item: a second launch would cost more there
    constexpr bool INPLACE = refines_in_place(CFG);
    // the FD mean in the other shapes refines its flagged pixels in this
    // kernel too, through a per-warp queue that the lanes drain 32 at a time
    // (not the NOREF form, which flags none)
    constexpr bool QUEUE = refines_by_queue(CFG, GRAD, PHI) && !NOREF;
    constexpr bool INKERNEL = INPLACE || QUEUE;
    constexpr int HR = SEP5 ? 2 : 1;                  // halo rows above and below an item
    constexpr int NCH = (TH + 2 * HR + CR - 1) / CR;  // chunks per item: rows y0-HR .. y0+TH-1+HR
    static_assert(SEP5 || (TH + 2) % CR == 0, "3x3 items' chunks tile their rows exactly");
    static_assert(kCfgs[CFG].tw == 128, "a band is 32 lanes x 4 columns");
    static_assert(TH <= 32, "pending-refinement bits hold 32 rows");
    constexpr int PADX = 16 / (int)sizeof(T);
    constexpr int BOXW = 128 + 2 * PADX;
    constexpr uint32_t BOX_BYTES = BOXW * CR * sizeof(T);
    constexpr uint32_t STRIDE = (BOX_BYTES + 127) & ~127u;

    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long full[NW][NST];
    // (QUEUE) each warp's queue of flagged pixels: frame index << 32 | y << 16 | x
    __shared__ unsigned long long rqueue[NW][QUEUE ? 32 : 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // (an offset from smem_raw keeps the compiler's knowledge that this is shared memory)
    unsigned char *const sbase = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    unsigned char *ring = sbase + warp * NST * STRIDE;
    // (5x5 filters) this lane's slots of the per-warp ring of row derivatives and smoothings
    float4 *const dring = reinterpret_cast<float4 *>(sbase + NW * NST * STRIDE + warp * kSep5RingBytes) + lane;
    // (FD) this lane's slots of the per-warp carry buffer
    float4 *const carry3 = reinterpret_cast<float4 *>(sbase + NW * NST * STRIDE + warp * carry_bytes(GRAD)) + lane;
    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < NST; ++s) mbar_init(smem_addr(&full[warp][s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_shared();
    }
    __syncwarp();
    // The refinement kernel that follows on the stream (a programmatic
    // dependent launch) may be scheduled now: its blocks take the SMs this
    // grid leaves, and wait for the grid's completion before reading the
    // list.  (No dependent, no effect.)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    const int gw = blockIdx.x * NW + warp, nw = gridDim.x * NW, total = args.total_tiles;

    if ((args.flags & TFN_FLAG_TEST_WAIT_TIMEOUT) && gw == 0) {
        // (test hook) wait on a barrier that nothing completes, before this
        // warp issues any copy, and give up as a copy that never landed
        // would: the launch reports the failed wait, this warp's items stay
        // unprocessed, and no copy of this warp is in flight
        __shared__ __align__(8) unsigned long long never;
        if (lane == 0) {
            mbar_init(smem_addr(&never), 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            if (!mbar_wait(smem_addr(&never), 0, kTestWaitCycles)) atomicOr(args.status, DEVERR_TMA_WAIT);
        }
        __syncwarp();
        return;
    }

    // Producer (lane 0): chunk number cc of this warp's sequence is chunk
    // cc % NCH of its (cc / NCH)-th item and goes to stage cc % NST.
    int pf = 0, fenced = -1;
    auto issue = [&](int cc) {
        const int t = gw + (cc / NCH) * nw;
        if (t >= total) return;
        pf = frame_of_item(args.frames, args.nframes, t, pf);
        const FrameDesc *f = args.frames + pf;
        const int lt = t - __ldg(&f->tile_begin), txs = __ldg(&f->tiles_x);
        const int x = (lt % txs) * 128 - PADX;
        const int y = (lt / txs) * TH - HR + (cc % NCH) * CR;
        const uint32_t bar = smem_addr(&full[warp][cc % NST]);
        // (a chunk partly or wholly past the bottom row is copied too: the
        // copy fills those rows with zeros, which decode as holes)
        const CUtensorMap *map = args.maps + pf;
        if (pf != fenced) {
            fence_tensormap_acquire(map);
            fenced = pf;
        }
        mbar_expect_tx(bar, BOX_BYTES);
        tma_load_2d(smem_addr(ring + (cc % NST) * STRIDE), map, x, y, bar);
    };
    if (lane == 0)
#pragma unroll
        for (int cc = 0; cc < NST; ++cc) issue(cc);

    const bool refine_all = args.flags & TFN_FLAG_REFINE_ALL;  // a negative threshold refines every pixel
    const float wts[3] = {args.w[0], args.w[1], args.w[2]};  // GRAD_WEIGHTED's row weights
    const Sep5W sw = {args.w[0], args.w[1], args.w[2], args.w[3], args.w[4]};  // GRAD_SEP5's profiles
    int cf = 0, fail_cc = 0;
    unsigned nref = 0;  // (INPLACE, QUEUE) pixels refined by this lane
    int qn = 0;         // (QUEUE) entries in the warp's queue (the same in every lane)
    bool failed = false;
    for (int i = 0; !failed; ++i) {
        const int t = gw + i * nw;
        if (t >= total) break;
        cf = frame_of_item(args.frames, args.nframes, t, cf);
        const FrameDesc *f = args.frames + cf;
        OutDesc out;
        out.out = (char *)__ldg((const unsigned long long *)&f->out);
        out.out_pitch = __ldg(&f->out_pitch);
        out.out_plane = __ldg(&f->out_plane);
        out.mask = (uint8_t *)__ldg((const unsigned long long *)&f->mask);
        out.mask_pitch = __ldg(&f->mask_pitch);
        const int H = __ldg(&f->H), W = __ldg(&f->W), txs = __ldg(&f->tiles_x);
        const float fx = __ldg(&f->fx), fy = __ldg(&f->fy), u0 = __ldg(&f->u0), v0 = __ldg(&f->v0);
        const float thr = refine_all ? -1.f : __ldg(&f->thr);
        const bool has_pts = __ldg((const unsigned long long *)&f->pts) != 0;  // (the fused point cloud)
        const float ztc = __ldg(&f->ztc);
        const float rfx = __frcp_rn(fx), rfy = __frcp_rn(fy);  // (PlanePCA)
        const int lt = t - __ldg(&f->tile_begin);
        const int x0 = (lt % txs) * 128 + 4 * lane, y0 = (lt / txs) * TH;
        const int nvalid = min(4, W - x0);  // pixels of this lane inside the frame (may be <= 0)
        float uc[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) uc[k] = __fsub_rn((float)(x0 + k), u0);
        const f2 uc2[2] = {pk(uc[0], uc[2]), pk(uc[1], uc[3])};  // (FD: the pixel pairs)

        // Sample row j (0 .. TH+2HR-1) of the item is image row y0 - HR + j;
        // rows at or past the bottom arrive as the copy's zero fill (holes).
        // The rows arrive in order, so the chunk state advances
        // incrementally: row jr of chunk cc.
        int jr = 0, cc = i * NCH;
        const unsigned char *stage = ring;
        // (the row loops that fetch one row at a time: load() reads row jr of `stage` into registers)
        auto fetch_with = [&](auto &&load, int j) -> bool {
            if (jr == 0) {
                const int st = cc % NST;
                stage = ring + st * STRIDE;
                if (!__all_sync(0xffffffffu, mbar_wait(smem_addr(&full[warp][st]), (uint32_t)((cc / NST) & 1)))) {
                    fail_cc = cc;
                    return false;
                }
            }
            load();
            if (++jr == CR) {  // the stage's last row is in registers: refill it
                __syncwarp();
                if (lane == 0) {
                    fence_async_shared();
                    issue(cc + NST);
                }
                jr = 0;
                ++cc;
            }
            return true;
        };
        unsigned long long pend_a = 0, pend_b = 0;  // (INPLACE, QUEUE) bit 4 s + k: row y0 + s, column x0 + k
        typename CarryOf<GRAD>::type cy;
        if constexpr (grad_is_pair(GRAD)) {
            cy.q = carry3;
            cy.d = carry3 + kCarry3Bytes / 16;  // (smoothed filters: the tap-difference ring after it)
            cy.p0 = 0;
            cy.ring = uses_dring(GRAD, PHI);
        }
        // output row y0 + s from sample rows P (above), C and N (below); the
        // 5x5 filters' gradients come in gu, gv
        auto emit = [&](const R &P, const R &C, const R &N, int s, const df(&gu)[4], const df(&gv)[4]) {
            const int y = y0 + s;
            float ox[4], oy[4], oz[4];
            uint32_t mw;
            unsigned rb;
            if constexpr (GRAD == GRAD_PLANEPCA) {
                pca_row<KIND, GRAD>(P, C, N, uc, __fsub_rn((float)y, v0), rfx, rfy, ztc, ox, oy, oz, mw);
                rb = 0;
            } else if constexpr (grad_is_pair(GRAD)) {
                row_step2<KIND, GRAD, PHI, NOREF>(P, C, N, cy, uc2, __fsub_rn((float)y, v0), fx, fy, thr, wts, ox, oy,
                                                  oz, mw, rb);
            } else {
                row_step<KIND, GRAD, PHI>(P, C, N, cy, uc, __fsub_rn((float)y, v0), fx, fy, thr, wts, gu, gv, ox, oy,
                                          oz, mw, rb);
            }
            // The common case under one test: a full quad of a row inside the
            // frame, planar output, no point cloud, nothing to refine.
            if (y < H && nvalid == 4 && !has_pts && rb == 0 && args.out_fmt <= OUT_BF16) {
                store4_planar(out, args.out_fmt, x0, y, ox, oy, oz, mw);
            } else if (y < H && nvalid > 0) {
                rb &= (1u << min(nvalid, 4)) - 1u;
                // pixels whose FP32 error bound is too loose: mask bit 1 set
                // (bit k of rb to bit 8k + 1), and listed for refine_kernel
                if constexpr (!INKERNEL) mw |= ((rb * 0x00204081u) & 0x01010101u) << 1;
                store4(out, args.out_fmt, x0, y, nvalid, ox, oy, oz, mw);
                if (has_pts)  // the fused point cloud of this row
                    store_points4<KIND>(f, x0, y, nvalid, sample(C, 1), sample(C, 2), sample(C, 3), sample(C, 4));
                if constexpr (INKERNEL) {  // (redone after the item)
                    if (s < 16)
                        pend_a |= (unsigned long long)rb << (4 * s);
                    else
                        pend_b |= (unsigned long long)rb << (4 * (s - 16));
                } else if (rb) {
                    list_for_refinement(args.rlist, args.rcount, args.rcap, cf, x0, y, rb);
                }
            }
        };
        if constexpr (!SEP5) {
            const df g0[4] = {};  // (3x3 filters compute their gradients in row_step)
            R P, C, N;
            // Two forms of the row loop, each the faster for its Phi (measured on
            // the 256-frame batch): the median's row step, the larger, runs
            // best in one flat loop that fetches row by row; the mean's in a
            // loop over chunks with a rolled loop over each chunk's rows.
            if constexpr (PHI == PHI_MEDIAN) {
                auto fetch = [&](R &row, int j) -> bool {
                    return fetch_with([&]() { load_row<KIND, GRAD, BOXW, PADX>(stage, jr, lane, row); }, j);
                };
                if (!fetch(C, 0) || !fetch(N, 1)) {
                    failed = true;
                    break;
                }
                if constexpr (GRAD != GRAD_PLANEPCA) carry_down(C, N, cy);
                P = C;
                C = N;
                for (int s = 0; s < TH; ++s) {
                    if (!fetch(N, s + 2)) {
                        failed = true;
                        break;
                    }
                    emit(P, C, N, s, g0, g0);
                    P = C;
                    C = N;
                }
            } else {
                // Chunk by chunk (the item's TH + 2 sample rows fill NCH chunks
                // exactly): wait for the chunk's stage, roll through its rows,
                // then refill the stage; the first chunk's first two rows start
                // the window.  (Rolled loops: unrolling the row loop to rotate the
                // roles of P, C, N costs more in instruction fetch than the row
                // copies it saves.)
                int s = 0;  // output row of the item
                for (int ch = 0; ch < NCH; ++ch, ++cc) {
                    const int st = cc % NST;
                    const unsigned char *const stg = ring + st * STRIDE;
                    if (!__all_sync(0xffffffffu, mbar_wait(smem_addr(&full[warp][st]), (uint32_t)((cc / NST) & 1)))) {
                        fail_cc = cc;
                        failed = true;
                        break;
                    }
                    int r = 0;
                    if (ch == 0) {
                        load_row<KIND, GRAD, BOXW, PADX>(stg, 0, lane, C);
                        load_row<KIND, GRAD, BOXW, PADX>(stg, 1, lane, N);
                        if constexpr (GRAD != GRAD_PLANEPCA) carry_down(C, N, cy);
                        P = C;
                        C = N;
                        r = 2;
                    }
#pragma unroll 1
                    for (; r < CR; ++r, ++s) {
                        load_row<KIND, GRAD, BOXW, PADX>(stg, r, lane, N);
                        emit(P, C, N, s, g0, g0);
                        P = C;
                        C = N;
                    }
                    __syncwarp();
                    if (lane == 0) {  // every row of the stage has been read: refill it
                        fence_async_shared();
                        issue(cc + NST);
                    }
                }
            }
        } else {
            // 5x5 filters: sample row j's derivative and smoothing go to ring
            // slot j % 5 (4 float4 per lane: Dh.h, Dh.l, Sh.h, Sh.l); output
            // row y0 + s is made once sample row s + 4 has arrived, from
            // slots s .. s + 4 and the sample rows P, C, N (image rows
            // y0 + s - 1 .. y0 + s + 1).
            int wslot = 0;
            float z8[8];
            auto take = [&](R &row, int j) -> bool {
                if (!fetch_with([&]() { load_row8<KIND, BOXW, PADX>(stage, jr, lane, z8); }, j)) return false;
                df Dh[4], Sh[4];
                sep5_row<KIND>(z8, sw, Dh, Sh);
                float4 *q = dring + wslot * (4 * 32);
                q[0] = make_float4(Dh[0].h, Dh[1].h, Dh[2].h, Dh[3].h);
                q[32] = make_float4(Dh[0].l, Dh[1].l, Dh[2].l, Dh[3].l);
                q[64] = make_float4(Sh[0].h, Sh[1].h, Sh[2].h, Sh[3].h);
                q[96] = make_float4(Sh[0].l, Sh[1].l, Sh[2].l, Sh[3].l);
                wslot = wslot == 4 ? 0 : wslot + 1;
#pragma unroll
                for (int c = 0; c < 6; ++c) row.z[c] = z8[c + 1];
                return true;
            };
            R P, C, N, X;
            if (!take(X, 0) || !take(P, 1) || !take(C, 2) || !take(N, 3)) {
                failed = true;
                break;
            }
            carry_down(P, C, cy);
            int rslot = 0;  // ring slot of sample row s
            for (int s = 0; s < TH; ++s) {
                if (!take(X, s + 4)) {
                    failed = true;
                    break;
                }
                // G_u = s0 Dh(s+2) + s1 (Dh(s+1) + Dh(s+3)) + s2 (Dh(s) + Dh(s+4)),
                // G_v = d1 (Sh(s+3) - Sh(s+1)) + d2 (Sh(s+4) - Sh(s)); the ring
                // rows are read pair by pair to keep few registers live
                auto ring_at = [&](int a, int v) -> float4 {
                    const int q = rslot + a < 5 ? rslot + a : rslot + a - 5;
                    return dring[(q * 4 + v) * 32];
                };
                const df zero = {0.f, 0.f};
                df gu[4], gv[4], t[4];
                {
                    const float4 h = ring_at(2, 0), l = ring_at(2, 1);
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        gu[k] = sw.s0 != 0.f ? dfl_mul_f(df{f4_at(h, k), f4_at(l, k)}, sw.s0) : zero;
                }
                {
                    const float4 h1 = ring_at(1, 0), l1 = ring_at(1, 1), h3 = ring_at(3, 0), l3 = ring_at(3, 1);
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        t[k] = sw.s1 != 0.f ? dfl_mul_f(dfl_add(df{f4_at(h1, k), f4_at(l1, k)}, df{f4_at(h3, k), f4_at(l3, k)}),
                                                        sw.s1)
                                            : zero;
                }
                {
                    const float4 h0 = ring_at(0, 0), l0 = ring_at(0, 1), h4 = ring_at(4, 0), l4 = ring_at(4, 1);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const df t2 = sw.s2 != 0.f ? dfl_mul_f(dfl_add(df{f4_at(h0, k), f4_at(l0, k)},
                                                                       df{f4_at(h4, k), f4_at(l4, k)}),
                                                               sw.s2)
                                                   : zero;
                        gu[k] = df_norm(dfl_add(gu[k], dfl_add(t[k], t2)));
                    }
                }
                {
                    const float4 h1 = ring_at(1, 2), l1 = ring_at(1, 3), h3 = ring_at(3, 2), l3 = ring_at(3, 3);
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        gv[k] = sw.d1 != 0.f ? dfl_mul_f(dfl_sub(df{f4_at(h3, k), f4_at(l3, k)}, df{f4_at(h1, k), f4_at(l1, k)}),
                                                         sw.d1)
                                             : zero;
                }
                {
                    const float4 h0 = ring_at(0, 2), l0 = ring_at(0, 3), h4 = ring_at(4, 2), l4 = ring_at(4, 3);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const df t2 = sw.d2 != 0.f ? dfl_mul_f(dfl_sub(df{f4_at(h4, k), f4_at(l4, k)},
                                                                       df{f4_at(h0, k), f4_at(l0, k)}),
                                                               sw.d2)
                                                   : zero;
                        gv[k] = df_norm(dfl_add(gv[k], t2));
                    }
                }
                emit(P, C, N, s, gu, gv);
                P = C;
                C = N;
                N = X;
                rslot = rslot == 4 ? 0 : rslot + 1;
            }
        }
        if (failed) break;
        if constexpr ((TH + 2 * HR) % CR != 0) {
            // the item's last chunk is partly unused: its stage is free now
            if (jr != 0) {
                __syncwarp();
                if (lane == 0) {
                    fence_async_shared();
                    issue(cc + NST);
                }
                jr = 0;
                ++cc;
            }
        }
        if constexpr (INPLACE) {
            // the double-float path for this item's flagged pixels (lanes in
            // parallel); the later store to the same pixel wins
            const void *in = (const void *)__ldg((const unsigned long long *)&f->in);
            const int64_t in_pitch = __ldg(&f->in_pitch);
            while (pend_a | pend_b) {
                int b;
                if (pend_a) {
                    b = __ffsll((long long)pend_a) - 1;
                    pend_a &= pend_a - 1;
                } else {
                    b = 64 + __ffsll((long long)pend_b) - 1;
                    pend_b &= pend_b - 1;
                }
                const int x = x0 + (b & 3), y = y0 + (b >> 2);
                Vec3 nr = {0.f, 0.f, 0.f};
                if constexpr (SEP5)
                    nr = refine_from_input_sep5<KIND, PHI>(in, in_pitch, H, W, x, y, fx, fy, u0, v0, sw.d1, sw.d2,
                                                           sw.s0, sw.s1, sw.s2);
                else if constexpr (GRAD != GRAD_PLANEPCA)  // (PlanePCA never flags a pixel)
                    nr = refine_from_input<KIND, GRAD, PHI>(in, in_pitch, H, W, x, y, fx, fy, u0, v0, wts[0], wts[1],
                                                            wts[2]);
                store1(out, args.out_fmt, x, y, nr);
                ++nref;
            }
        }
        if constexpr (QUEUE) {
            // this item's flagged pixels join the warp's queue, in rounds of
            // at most one per lane; whenever it holds 32, each lane refines
            // one (the later store to the same pixel wins: the __syncwarp
            // orders the item's stores before the lanes' refined ones)
            while (__any_sync(0xffffffffu, (pend_a | pend_b) != 0)) {
                const bool has = (pend_a | pend_b) != 0;
                const unsigned bal = __ballot_sync(0xffffffffu, has);
                const int slot = qn + __popc(bal & ((1u << lane) - 1u));
                if (has && slot < 32) {  // (a lane past the queue's end keeps its pixel for the next round)
                    int b;
                    if (pend_a) {
                        b = __ffsll((long long)pend_a) - 1;
                        pend_a &= pend_a - 1;
                    } else {
                        b = 64 + __ffsll((long long)pend_b) - 1;
                        pend_b &= pend_b - 1;
                    }
                    rqueue[warp][slot] = ((unsigned long long)(unsigned)cf << 32) |
                                         ((unsigned)(y0 + (b >> 2)) << 16) | (unsigned)(x0 + (b & 3));
                }
                qn = min(qn + __popc(bal), 32);
                if (qn == 32) {
                    __syncwarp();
                    const unsigned long long e = rqueue[warp][lane];
                    refine_at<KIND, GRAD, PHI, false>(args, (int)(e >> 32), (int)(e & 0xffffu),
                                                      (int)((e >> 16) & 0xffffu));
                    ++nref;
                    __syncwarp();  // (every lane has read its entry before the slots are refilled)
                    qn = 0;
                }
            }
        }
    }
    if (failed) {
        // a copy did not land in time: flag it, then give the copies this warp
        // may still have in flight a short bounded wait before leaving
        if (lane == 0) {
            atomicOr(args.status, DEVERR_TMA_WAIT);
            for (int cc = fail_cc; cc < fail_cc + NST; ++cc)
                if (gw + (cc / NCH) * nw < total)
                    mbar_wait(smem_addr(&full[warp][cc % NST]), (uint32_t)((cc / NST) & 1), kDrainCycles);
        }
        __syncwarp();
        return;
    }
    if constexpr (QUEUE) {  // the queue's last entries, fewer than 32
        __syncwarp();
        if (lane < qn) {
            const unsigned long long e = rqueue[warp][lane];
            refine_at<KIND, GRAD, PHI, false>(args, (int)(e >> 32), (int)(e & 0xffffu), (int)((e >> 16) & 0xffffu));
            ++nref;
        }
    }
    if constexpr (INKERNEL) {
        // count of refined pixels (diagnostics): one atomic per warp, only if any
        const unsigned tot = __reduce_add_sync(0xffffffffu, nref);
        if (lane == 0 && tot) atomicAdd(args.status + 1, tot);
    }
}

// noref: the NOREF form (FP16 depth with the FD filter only; nullptr otherwise).
// FDMEAN: the FD mean's kernels with the error bound (true), or every other
// kernel (false).  The two sets are instantiated in separate translation
// units: the code of the FD mean's refinement queue, compiled into the same
// module as the other kernels, changed how the compiler allocated their
// registers (a 48-byte stack frame in every kernel of the module; the Sobel,
// Scharr, Prewitt and weighted means ran 3-6% slower, the FP16 forms 0.5-3%),
// though none of them runs that code.
template <int KIND, bool FDMEAN>
KernelFn select_kernel(int grad, int phi, int cfg, bool noref)
{
    if ((grad == GRAD_FD && phi == PHI_MEAN && !noref) != FDMEAN) return nullptr;
    if (noref) {
        // (each kernel is instantiated in one translation unit only)
        if constexpr (KIND == KIND_DEPTH_F16 && !FDMEAN) {
#define TFN_K(P, C) \
    if (grad == GRAD_FD && phi == P && cfg == C) return &normals_kernel<KIND, GRAD_FD, P, C, true>;
#define TFN_KC(P) TFN_K(P, 0) TFN_K(P, 1) TFN_K(P, 2) TFN_K(P, 3) TFN_K(P, 4) TFN_K(P, 5)
            TFN_KC(PHI_MEAN) TFN_KC(PHI_MEDIAN)
#undef TFN_KC
#undef TFN_K
        }
        return nullptr;
    }
#define TFN_K(G, P, C)                                                                        \
    if (grad == G && phi == P && cfg == C) return &normals_kernel<KIND, G, P, C, false>;
#define TFN_KC(G, P) TFN_K(G, P, 0) TFN_K(G, P, 1) TFN_K(G, P, 2) TFN_K(G, P, 3) TFN_K(G, P, 4) TFN_K(G, P, 5)
#define TFN_KP(G) TFN_KC(G, PHI_MEAN) TFN_KC(G, PHI_MEDIAN)
    if constexpr (FDMEAN) {
        TFN_KC(GRAD_FD, PHI_MEAN)
    } else {
        TFN_KC(GRAD_FD, PHI_MEDIAN)
        TFN_KP(GRAD_SOBEL) TFN_KP(GRAD_SCHARR) TFN_KP(GRAD_PREWITT) TFN_KP(GRAD_WEIGHTED) TFN_KP(GRAD_SEP5)
        TFN_KC(GRAD_PLANEPCA, PHI_MEAN)  // (PlanePCA has no Phi)
    }
#undef TFN_KP
#undef TFN_KC
#undef TFN_K
    return nullptr;
}

// The second kernel of a launch: the pixels normals_kernel flagged, from its
// list, or (when the list overflowed) by a scan of every frame's mask for
// bit 1, 16 mask bytes per load (mask rows start on 16-byte boundaries and
// their pitch is a multiple of 16, so a row's last load stays inside its
// pitch; bytes past the frame's width are not pixels and are skipped).  Adds
// the number of refined pixels to status[1].
template <int KIND, int GRAD, int PHI>
__global__ void __launch_bounds__(kRefineThreads) refine_kernel(const __grid_constant__ LaunchArgs args)
{
    // launched as a programmatic dependent of normals_kernel: wait until that
    // grid has completed and its writes (the list, the normals) are visible
    // (returns at once in a launch without the dependency)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const unsigned long long cnt = *args.rcount;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x, nth = (long long)gridDim.x * blockDim.x;
    unsigned nref = 0;
    if (cnt <= (unsigned long long)args.rcap) {
        for (long long i = tid; i < (long long)cnt; i += nth) {
            const unsigned long long e = args.rlist[i];
            const int fi = (int)(e >> 32);
            if (fi >= args.nframes) continue;  // (not an entry of this launch's frames)
            refine_at<KIND, GRAD, PHI, true>(args, fi, (int)(e & 0xffffu), (int)((e >> 16) & 0xffffu));
            ++nref;
        }
    } else {
        for (int fi = 0; fi < args.nframes; ++fi) {
            const FrameDesc *f = args.frames + fi;
            const uint8_t *mask = (const uint8_t *)__ldg((const unsigned long long *)&f->mask);
            const int64_t mp = __ldg(&f->mask_pitch);
            const int W = __ldg(&f->W), H = __ldg(&f->H);
            const int cpr = (W + 15) >> 4;  // 16-byte chunks per row
            const long long nch = (long long)H * cpr;
            for (long long q = tid; q < nch; q += nth) {
                const int y = (int)(q / cpr), c = (int)(q - (long long)y * cpr);
                const uint4 v = *reinterpret_cast<const uint4 *>(mask + (int64_t)y * mp + 16 * c);
                const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    for (unsigned b = w[j] & 0x02020202u; b; b &= b - 1u) {
                        const int x = 16 * c + 4 * j + ((__ffs(b) - 1) >> 3);
                        if (x < W) {
                            refine_at<KIND, GRAD, PHI, true>(args, fi, x, y);
                            ++nref;
                        }
                    }
                }
            }
        }
    }
    const unsigned tot = __reduce_add_sync(0xffffffffu, nref);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(args.status + 1, tot);
    // The last block to finish (every block has read the count by then)
    // zeroes the count and the block counter for the launch's next use.
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned *done = reinterpret_cast<unsigned *>(args.rcount + 1);
        __threadfence();
        if (atomicAdd(done, 1u) == gridDim.x - 1) {
            *args.rcount = 0;
            *done = 0;
            __threadfence();
        }
    }
}

template <int KIND>
KernelFn select_refiner(int grad, int phi)
{
#define TFN_R(G, P) \
    if (grad == G && phi == P) return &refine_kernel<KIND, G, P>;
#define TFN_RP(G) TFN_R(G, PHI_MEAN) TFN_R(G, PHI_MEDIAN)
    // (the FD mean refines in its own kernel; PlanePCA never flags a pixel)
    TFN_R(GRAD_FD, PHI_MEDIAN)
    TFN_RP(GRAD_SOBEL) TFN_RP(GRAD_SCHARR) TFN_RP(GRAD_PREWITT) TFN_RP(GRAD_WEIGHTED) TFN_RP(GRAD_SEP5)
#undef TFN_RP
#undef TFN_R
    return nullptr;
}

}  // namespace dev
}  // namespace tfn
