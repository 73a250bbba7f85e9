// tfn_kernel.cuh -- the fused Three-Filters-to-Normal kernel for sm_103a.
//
// One persistent kernel walks a queue of TW x TH tiles spanning every frame
// of a launch; CTA b takes every grid-th tile starting at b.  Each tile plus a halo
// (1 row above/below, 4 or 8 columns left/right so that the box starts on a
// 16-byte boundary) is staged into shared memory by a TMA 2D copy, through a
// ring of kStages buffers (mbarrier for "landed", a release counter for
// "free"); each of the 256 threads computes 4 x PR pixels from a register
// window and writes normals and mask with vectorised streaming stores.  Out-of-image taps read the TMA
// zero fill, which is a hole, so image borders need no special case.
//
// Arithmetic (Sec. III of Fan et al.):
//   inverse depth    w = 1/Z per sample as wh + wl (hardware reciprocal plus
//                    its FMA residual), so gradients never lose the digits a
//                    difference of two rounded reciprocals would;
//   filters          G = sum_k c_k (w_{k,+1} - w_{k,-1}) with the row weights of
//                    the chosen filter (normalisation dropped: the normal's
//                    direction is homogeneous in (G_u, G_v)); disparity: the
//                    same on d (Eq. nx2_ny2_nz3);
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
// Accuracy: the gradients are compensated (w residuals, exact tap
// differences by Knuth's TwoSum where filter terms can cancel), so each
// candidate carries a few units of FP32 rounding relative to itself.  What
// remains is cancellation inside the candidate sum (mean) or between the two
// middle candidates (even median); each pixel bounds that error and the rare
// pixels whose bound exceeds the threshold go to refine_pixel(), which redoes
// the pixel in double-float arithmetic.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tfn_internal.h"

namespace tfn {
namespace dev {

constexpr float kValidLo = 1.52587890625e-05f;  // 2^-16
constexpr float kValidHi = 65536.0f;            // 2^16
constexpr long long kWaitCycles = 4000000000LL;    // ~2 s at 2 GHz

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

// Long division in double-float: q1 = a/b, correct with the residual.
__device__ __forceinline__ df df_div(df a, df b)
{
    float q1 = __fdiv_rn(a.h, b.h);
    df r = df_add(a, df_neg(df_mul_f(b, q1)));
    float q2 = __fdiv_rn(r.h, b.h);
    return fast_two_sum(q1, q2);
}

__device__ __forceinline__ float df_val(df a) { return __fadd_rn(a.h, a.l); }

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

template <int KIND, int GRAD>
__device__ __forceinline__ void gradients(const float (&z)[3][3], df &Gu, df &Gv)
{
    if (GRAD == GRAD_FD) {
        Gu = grad_term<KIND>(z[1][0], z[1][2]);
        Gv = grad_term<KIND>(z[0][1], z[2][1]);
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
template <int KIND, int GRAD, int PHI>
__device__ __noinline__ Vec3 refine_pixel(float z00, float z01, float z02, float z10, float z11, float z12, float z20,
                                          float z21, float z22, unsigned okbits, int u, int v, float fx, float fy,
                                          float u0, float v0)
{
    const float z[3][3] = {{z00, z01, z02}, {z10, z11, z12}, {z20, z21, z22}};
    bool ok[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) ok[a][b] = (okbits >> (3 * a + b)) & 1u;
    df Gu, Gv;
    gradients<KIND, GRAD>(z, Gu, Gv);
    const float zi = z[1][1];
    df R[8];
    int m = 0;
    for (int p = 0; p < 4; ++p) {
        const int du = pair_du(p), dv = pair_dv(p);
        df num = Gu;
        if (p == 1) num = Gv;
        if (p == 2) num = df_add(Gu, Gv);
        if (p == 3) num = df_add(Gu, df_neg(Gv));
        for (int side = 0; side < 2; ++side) {
            const int a = 1 + (side ? -dv : dv), b = 1 + (side ? -du : du);
            const float zj = z[a][b];
            const df nj = side ? df_neg(num) : num;
            if (!ok[a][b] || zj == zi) continue;
            df r;
            if (KindTraits<KIND>::disparity)  // Z_j / dz_j = d_i / (d_i - d_j)
                r = df_div(df_mul_f(nj, zi), two_sum(zi, -zj));
            else
                r = df_div(df_mul_f(nj, zj), two_sum(zj, -zi));
            R[m++] = r;
        }
    }
    df F = {0.f, 0.f};
    if (PHI == PHI_MEAN) {
        for (int k = 0; k < m; ++k) F = df_add(F, R[k]);
        F = df_div(F, df{(float)m, 0.f});
    } else {
        for (int i = 1; i < m; ++i) {  // insertion sort by the leading part
            df x = R[i];
            int k = i - 1;
            while (k >= 0 && R[k].h > x.h) {
                R[k + 1] = R[k];
                --k;
            }
            R[k + 1] = x;
        }
        if (m > 0) {
            F = R[m / 2];
            if (!(m & 1)) {
                F = df_add(R[m / 2 - 1], R[m / 2]);
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

// ------------------------------------------------------------ main path

// 2^-110: below the square of the smallest non-zero difference of two valid
// samples (|delta| >= 2^-39, so delta^2 >= 2^-78) by 2^-32.
constexpr float kEdgeEps = 7.703719777548943e-34f;

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

// The register window of one thread: ROWS+2 sample rows x 6 columns around
// its 4 x ROWS pixels.  Holes are stored as 0.
template <int KIND, int ROWS>
struct Win {
    float z[ROWS + 2][6];   // holes are 0, valid samples are > 0
    float wh[ROWS + 2][6];  // depth kinds: 1/Z ~ wh + wl (rcp + FMA residual)
    float wl[ROWS + 2][6];
    unsigned ok[ROWS + 2];  // bit c: column c valid
};

template <int KIND>
__device__ __forceinline__ float decode(typename KindTraits<KIND>::T raw, bool &ok)
{
    float v;
    if (KIND == KIND_DISP_U16) {
        v = (float)(uint16_t)raw;
        ok = v != 0.f;
    } else {
        if (KIND == KIND_DEPTH_F16)
            v = __half2float(*reinterpret_cast<const __half *>(&raw));
        else
            v = *reinterpret_cast<const float *>(&raw);
        // finite and in [2^-16, 2^16]: one unsigned compare on the bit pattern
        // (negatives, infinities and NaNs have patterns above 2^16's)
        ok = (uint32_t)(__float_as_uint(v) - 0x37800000u) <= (0x47800000u - 0x37800000u);
    }
    return ok ? v : 0.f;
}

template <int KIND, int ROWS>
__device__ __forceinline__ void load_window(const void *tile, int SW, int PADX, int row0, int col0, Win<KIND, ROWS> &W)
{
    typedef typename KindTraits<KIND>::T T;
    const T *t = reinterpret_cast<const T *>(tile);
#pragma unroll
    for (int a = 0; a < ROWS + 2; ++a) {
        const T *p = t + (row0 + a) * SW + PADX + col0;  // p[-1..4]
        T raw[6];
        raw[0] = p[-1];
        if (sizeof(T) == 4) {
            const uint4 q = *reinterpret_cast<const uint4 *>(p);
            raw[1] = *reinterpret_cast<const T *>(&q.x);
            raw[2] = *reinterpret_cast<const T *>(&q.y);
            raw[3] = *reinterpret_cast<const T *>(&q.z);
            raw[4] = *reinterpret_cast<const T *>(&q.w);
        } else {
            const uint2 q = *reinterpret_cast<const uint2 *>(p);
            const uint16_t h[4] = {(uint16_t)(q.x & 0xffff), (uint16_t)(q.x >> 16), (uint16_t)(q.y & 0xffff),
                                   (uint16_t)(q.y >> 16)};
#pragma unroll
            for (int c = 0; c < 4; ++c) raw[1 + c] = *reinterpret_cast<const T *>(&h[c]);
        }
        raw[5] = p[4];
        unsigned bits = 0;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            bool ok;
            W.z[a][c] = decode<KIND>(raw[c], ok);
            bits |= (unsigned)ok << c;
            if (!KindTraits<KIND>::disparity) {
                const float wh = rcp_approx(W.z[a][c]);
                W.wh[a][c] = wh;
                W.wl[a][c] = __fmaf_rn(-wh, W.z[a][c], 1.f) * wh;
            }
        }
        W.ok[a] = bits;
    }
}

// Edge between samples (a1,c1) < (a2,c2) (raster order): 1/(s2 - s1); for
// disparity, an edge touching a hole is given delta = 0 so that it drops out.
template <int KIND, int ROWS>
__device__ __forceinline__ EdgeR edge(const Win<KIND, ROWS> &W, int a1, int c1, int a2, int c2)
{
    float d = W.z[a2][c2] - W.z[a1][c1];
    if (KindTraits<KIND>::disparity) d = (W.z[a1][c1] != 0.f && W.z[a2][c2] != 0.f) ? d : 0.f;
    return edge_recip(d);
}

// rho_j = Z_j / (Z_j - Z_i) for pixel i = (a,c) and neighbour j = (a+dv, c+du);
// disparity: d_i / (d_i - d_j).  k is the edge's candidate indicator.
template <int KIND, int ROWS>
__device__ __forceinline__ float rho(const Win<KIND, ROWS> &W, int a, int c, int dv, int du, float &k)
{
    const int a2 = a + dv, c2 = c + du;
    const bool fwd = dv > 0 || (dv == 0 && du > 0);  // i precedes j in raster order
    const EdgeR e = fwd ? edge<KIND, ROWS>(W, a, c, a2, c2) : edge<KIND, ROWS>(W, a2, c2, a, c);
    k = e.k;
    if (KindTraits<KIND>::disparity) return fwd ? -__fmul_rn(W.z[a][c], e.r) : __fmul_rn(W.z[a][c], e.r);
    return fwd ? __fmul_rn(W.z[a2][c2], e.r) : -__fmul_rn(W.z[a2][c2], e.r);
}

// Exact difference of two taps as h + l (w-differences carry the w residuals).
template <int KIND, int ROWS>
__device__ __forceinline__ df tap_diff(const Win<KIND, ROWS> &W, int a1, int c1, int a2, int c2, bool exact_needed)
{
    if (KindTraits<KIND>::disparity) {
        if (KindTraits<KIND>::exact_diff) return {W.z[a2][c2] - W.z[a1][c1], 0.f};
        return two_sum(W.z[a2][c2], -W.z[a1][c1]);
    }
    const float lo = __fsub_rn(W.wl[a2][c2], W.wl[a1][c1]);
    if (!exact_needed) return {__fsub_rn(W.wh[a2][c2], W.wh[a1][c1]), lo};
    const df h = two_sum(W.wh[a2][c2], -W.wh[a1][c1]);
    return {h.h, __fadd_rn(h.l, lo)};
}

template <int KIND, int GRAD, int ROWS>
__device__ __forceinline__ void gradients_win(const Win<KIND, ROWS> &W, int a, int c, df &Gu, df &Gv)
{
    if (GRAD == GRAD_FD) {
        // a single difference: no cancellation between terms to protect
        Gu = tap_diff<KIND, ROWS>(W, a, c - 1, a, c + 1, false);
        Gv = tap_diff<KIND, ROWS>(W, a - 1, c, a + 1, c, false);
    } else {
        Gu = filter_sum<GRAD>(tap_diff<KIND, ROWS>(W, a - 1, c - 1, a - 1, c + 1, true),
                              tap_diff<KIND, ROWS>(W, a, c - 1, a, c + 1, true),
                              tap_diff<KIND, ROWS>(W, a + 1, c - 1, a + 1, c + 1, true));
        Gv = filter_sum<GRAD>(tap_diff<KIND, ROWS>(W, a - 1, c - 1, a + 1, c - 1, true),
                              tap_diff<KIND, ROWS>(W, a - 1, c, a + 1, c, true),
                              tap_diff<KIND, ROWS>(W, a - 1, c + 1, a + 1, c + 1, true));
    }
}

struct PixelResult {
    float x, y, z;
    bool valid, refine;
};

// Main FP32 path of one pixel, branch-free: every lane runs the same
// instructions; invalid pixels, the special case and pixels that need the
// double-float path are resolved by selects at the end.  Every product is an
// explicit __fmul_rn (never contracted into an FMA), so a pixel's bits do not
// depend on which row of a thread's window it sits in or on the tile shape.
template <int KIND, int GRAD, int PHI, int ROWS>
__device__ __forceinline__ PixelResult pixel_normal(const Win<KIND, ROWS> &W, unsigned evmask, int a, int c, int u, int v,
                                                    float fx, float fy, float u0, float v0, float thr, bool refine_all)
{
    // evaluable: the centre and every filter tap valid (bit c of the row's mask)
    const bool ev = (evmask >> c) & 1u;
    df Gu, Gv;
    gradients_win<KIND, GRAD, ROWS>(W, a, c, Gu, Gv);
    const float gu = __fadd_rn(Gu.h, Gu.l), gv = __fadd_rn(Gv.h, Gv.l);
    // Sec. III special case: both gradients exactly zero (the sums h + l of an
    // exact representation vanish only when both parts do)
    const bool flat = Gu.h == 0.f && Gu.l == 0.f && Gv.h == 0.f && Gv.l == 0.f;
    float num[4];
    num[0] = gu;
    num[1] = gv;
    num[2] = __fadd_rn(__fadd_rn(Gu.h, Gv.h), __fadd_rn(Gu.l, Gv.l));
    num[3] = __fadd_rn(__fsub_rn(Gu.h, Gv.h), __fsub_rn(Gu.l, Gv.l));
    // pair p: neighbour j_p and -j_p; j = right, down, down-right, up-right
    const int du_[4] = {1, 0, 1, 1}, dv_[4] = {0, 1, 1, -1};
    float rj[4], rm[4], kj[4], km[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        rj[p] = rho<KIND, ROWS>(W, a, c, dv_[p], du_[p], kj[p]);
        rm[p] = rho<KIND, ROWS>(W, a, c, -dv_[p], -du_[p], km[p]);
    }
    // The mean is carried unnormalised: n' scaled by m (> 0) has the same
    // direction, so no 1/m is needed.
    float mF, mbound, scale;
    if (PHI == PHI_MEAN) {
        float S = 0.f, Sabs = 0.f, m = 0.f;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            S = __fmaf_rn(num[p], __fsub_rn(rj[p], rm[p]), S);
            Sabs = __fmaf_rn(fabsf(num[p]), __fadd_rn(fabsf(rj[p]), fabsf(rm[p])), Sabs);
            if (GRAD == GRAD_FD && !KindTraits<KIND>::disparity && p >= 2) {
                // FD: a diagonal neighbour may be a hole (its rho is 0 already)
                m += (W.z[a + dv_[p]][c + du_[p]] != 0.f ? kj[p] : 0.f);
                m += (W.z[a - dv_[p]][c - du_[p]] != 0.f ? km[p] : 0.f);
            } else {
                m += kj[p] + km[p];
            }
        }
        mF = S;
        mbound = Sabs;
        scale = m;
    } else {
        float s[8];
        int cnt = 0;
        unsigned sgn = 0;  // sign bit of the next sentinel: +inf, -inf, +inf, ...
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const float cand[2] = {__fmul_rn(num[p], rj[p]), -__fmul_rn(num[p], rm[p])};
            const float rr[2] = {rj[p], rm[p]};
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const bool kept = rr[q] != 0.f;
                cnt += kept;
                s[2 * p + q] = kept ? cand[q] : __uint_as_float(0x7f800000u | sgn);
                sgn ^= kept ? 0u : 0x80000000u;
            }
        }
#define TFN_CE(i, j)                           \
    {                                          \
        const float lo_ = fminf(s[i], s[j]);   \
        s[j] = fmaxf(s[i], s[j]);              \
        s[i] = lo_;                            \
    }
        TFN_CE(0, 2) TFN_CE(1, 3) TFN_CE(4, 6) TFN_CE(5, 7)
        TFN_CE(0, 4) TFN_CE(1, 5) TFN_CE(2, 6) TFN_CE(3, 7)
        TFN_CE(0, 1) TFN_CE(2, 3) TFN_CE(4, 5) TFN_CE(6, 7)
        TFN_CE(2, 4) TFN_CE(3, 5)
        TFN_CE(1, 4) TFN_CE(3, 6)
        TFN_CE(1, 2) TFN_CE(3, 4) TFN_CE(5, 6)
#undef TFN_CE
        const bool odd = cnt & 1;
        mF = odd ? s[3] : __fmul_rn(0.5f, __fadd_rn(s[3], s[4]));
        mbound = odd ? fabsf(s[3]) : fmaxf(fabsf(s[3]), fabsf(s[4]));
        scale = 1.f;
    }
    const float A = __fmaf_rn(__fsub_rn((float)u, u0), gu, __fmul_rn(__fsub_rn((float)v, v0), gv));
    const float nxp = __fmul_rn(__fmul_rn(scale, fx), gu), nyp = __fmul_rn(__fmul_rn(scale, fy), gv);
    const float nzp = -__fmaf_rn(scale, A, mF);
    const float nn = __fmaf_rn(nxp, nxp, __fmaf_rn(nyp, nyp, __fmul_rn(nzp, nzp)));
    const float rs = rsqrt_approx(nn);
    PixelResult res;
    res.valid = ev;
    res.refine = ev && !flat && (refine_all || mbound > __fmul_rn(thr, __fmul_rn(nn, rs)));
    res.x = ev && !flat ? -__fmul_rn(nxp, rs) : 0.f;
    res.y = ev && !flat ? -__fmul_rn(nyp, rs) : 0.f;
    res.z = ev ? (flat ? -1.f : -__fmul_rn(nzp, rs)) : 0.f;
    return res;
}

// Double-float recomputation of the pixel whose 3x3 window starts at
// element `base` of the tile in shared memory (the tile is still resident:
// its buffer is released only after the refinement).  One call site keeps
// the rare path out of the main instruction stream.
template <int KIND, int GRAD, int PHI>
__device__ __noinline__ Vec3 refine_from_tile(const void *tile, int base, int SW, int u, int v, float fx, float fy,
                                              float u0, float v0)
{
    typedef typename KindTraits<KIND>::T T;
    const T *t = reinterpret_cast<const T *>(tile) + base;
    float z[9];
    unsigned okbits = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            bool ok;
            z[3 * a + b] = decode<KIND>(t[a * SW + b], ok);
            okbits |= (unsigned)ok << (3 * a + b);
        }
    return refine_pixel<KIND, GRAD, PHI>(z[0], z[1], z[2], z[3], z[4], z[5], z[6], z[7], z[8], okbits, u, v, fx, fy, u0,
                                         v0);
}

// Bit c (1..4) set iff pixel column c of window row a is evaluable: the centre
// and every tap of both filters valid.
template <int GRAD, int KIND, int ROWS>
__device__ __forceinline__ unsigned evaluable_row(const Win<KIND, ROWS> &W, int a)
{
    const unsigned m = W.ok[a];
    if (GRAD == GRAD_FD) return m & (m >> 1) & (m << 1) & W.ok[a - 1] & W.ok[a + 1];
    const unsigned t = W.ok[a - 1] & m & W.ok[a + 1];
    return t & (t >> 1) & (t << 1);
}


// ------------------------------------------------------------ TMA / mbarrier

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
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
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase)
{
    if (mbar_try(bar, phase)) return true;
    const long long t0 = clock64();
    for (;;) {
#pragma unroll 1
        for (int k = 0; k < 16; ++k)
            if (mbar_try(bar, phase)) return true;
        if (clock64() - t0 > kWaitCycles) return false;
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

// Stores 4 consecutive pixels (n valid of them, starting at column u).
__device__ __forceinline__ void store4(const OutDesc &fd, int fmt, int u, int v, int n, const float (&x)[4],
                                       const float (&y)[4], const float (&zz)[4], const uint8_t (&mk)[4])
{
    char *row = fd.out + (int64_t)v * fd.out_pitch;
    uint8_t *mrow = fd.mask + (int64_t)v * fd.mask_pitch;
    if (n == 4) {
        if (fmt == OUT_F32) {
            __stcs(reinterpret_cast<float4 *>(row + (int64_t)u * 4), make_float4(x[0], x[1], x[2], x[3]));
            __stcs(reinterpret_cast<float4 *>(row + fd.out_plane + (int64_t)u * 4), make_float4(y[0], y[1], y[2], y[3]));
            __stcs(reinterpret_cast<float4 *>(row + 2 * fd.out_plane + (int64_t)u * 4),
                   make_float4(zz[0], zz[1], zz[2], zz[3]));
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
        const uint32_t mw = (uint32_t)mk[0] | ((uint32_t)mk[1] << 8) | ((uint32_t)mk[2] << 16) | ((uint32_t)mk[3] << 24);
        __stcs(reinterpret_cast<unsigned int *>(mrow + u), mw);
        return;
    }
    for (int k = 0; k < n; ++k) {
        const int uu = u + k;
        if (fmt == OUT_F32) {
            reinterpret_cast<float *>(row)[uu] = x[k];
            reinterpret_cast<float *>(row + fd.out_plane)[uu] = y[k];
            reinterpret_cast<float *>(row + 2 * fd.out_plane)[uu] = zz[k];
        } else if (fmt == OUT_F16 || fmt == OUT_BF16) {
            const uint32_t px = pack2(x[k], y[k], fmt), pz = pack2(zz[k], 0.f, fmt);
            reinterpret_cast<uint16_t *>(row)[uu] = (uint16_t)(px & 0xffff);
            reinterpret_cast<uint16_t *>(row + fd.out_plane)[uu] = (uint16_t)(px >> 16);
            reinterpret_cast<uint16_t *>(row + 2 * fd.out_plane)[uu] = (uint16_t)(pz & 0xffff);
        } else {
            reinterpret_cast<uint2 *>(row)[uu] = make_uint2(pack2(x[k], y[k], fmt), pack2(zz[k], 0.f, fmt));
        }
        mrow[uu] = mk[k];
    }
}


// Stores one pixel's normal (the mask is already written).
__device__ __forceinline__ void store1(const OutDesc &fd, int fmt, int u, int v, Vec3 n)
{
    char *row = fd.out + (int64_t)v * fd.out_pitch;
    if (fmt == OUT_F32) {
        reinterpret_cast<float *>(row)[u] = n.x;
        reinterpret_cast<float *>(row + fd.out_plane)[u] = n.y;
        reinterpret_cast<float *>(row + 2 * fd.out_plane)[u] = n.z;
    } else if (fmt == OUT_F16 || fmt == OUT_BF16) {
        const uint32_t px = pack2(n.x, n.y, fmt), pz = pack2(n.z, 0.f, fmt);
        reinterpret_cast<uint16_t *>(row)[u] = (uint16_t)(px & 0xffff);
        reinterpret_cast<uint16_t *>(row + fd.out_plane)[u] = (uint16_t)(px >> 16);
        reinterpret_cast<uint16_t *>(row + 2 * fd.out_plane)[u] = (uint16_t)(pz & 0xffff);
    } else {
        reinterpret_cast<uint2 *>(row)[u] = make_uint2(pack2(n.x, n.y, fmt), pack2(n.z, 0.f, fmt));
    }
}

// ------------------------------------------------------------ the kernel

// Persistent kernel, 8 warps.  CTA b takes tiles b, b + grid, b + 2 grid, ...
// of the queue (interleaving spreads every CTA over all of memory).  Tile
// buffers form a kStages-deep ring.  Whoever fills a buffer also writes the
// tile's frame descriptor and origin into the buffer's info slot in shared
// memory, then arrives on the buffer's "full" mbarrier with the TMA byte
// count; consumers wait on it and read the slot, never global memory.  Every
// warp bumps the buffer's release counter when done with it, and the warp
// that completes the count refills it with the tile kStages ahead.  No warp
// ever waits for another except for data.
constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;

struct StageInfo {
    FrameDesc fd;
    int x0, y0, tile;
    int pad;
};

template <int KIND, int GRAD, int PHI, int CFG>
__global__ void __launch_bounds__(kThreads, 2) normals_kernel(const __grid_constant__ LaunchArgs args)
{
    typedef typename KindTraits<KIND>::T T;
    constexpr int TW = kCfgs[CFG].tw, TH = kCfgs[CFG].th, PR = kCfgs[CFG].pr;
    constexpr int PADX = 16 / (int)sizeof(T);
    constexpr int SW = TW + 2 * PADX, SH = TH + 2;
    constexpr uint32_t BOX_BYTES = SW * SH * sizeof(T);
    constexpr uint32_t STRIDE = (BOX_BYTES + 1023) & ~1023u;
    constexpr int TPR = TW / 4;
    static_assert(TPR * (TH / PR) == kThreads, "tile shape must match the block");

    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long full[kStages];
    __shared__ int released[kStages];
    __shared__ __align__(16) StageInfo info[kStages];
    unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    // The launch's frame table, copied once into shared memory when it fits,
    // so that refilling a buffer never waits on global memory.
    FrameDesc *ftab = reinterpret_cast<FrameDesc *>(smem + kStages * STRIDE);
    const bool ftab_smem = args.nframes <= kFrameTableMax;
    const FrameDesc *frames = ftab_smem ? ftab : args.frames;

    const int tid = threadIdx.x, lane = tid & 31;
    const int total = args.total_tiles, first = blockIdx.x, step = gridDim.x;

    if (ftab_smem) {
        const uint4 *src = reinterpret_cast<const uint4 *>(args.frames);
        uint4 *dst = reinterpret_cast<uint4 *>(ftab);
        const int words = args.nframes * (int)(sizeof(FrameDesc) / 16);
        for (int k = tid; k < words; k += kThreads) dst[k] = __ldg(src + k);
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_addr(&full[s]), 1);
            released[s] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_shared();
    }
    __syncthreads();

    // Filling side (whichever lane fills a buffer): frame cursor, last fenced map.
    int pf = 0, fenced = -1;
    auto fill = [&](int t, int s) {
        while (pf + 1 < args.nframes && frames[pf + 1].tile_begin <= t) ++pf;
        const CUtensorMap *map = args.maps + pf;
        if (pf != fenced) {
            fence_tensormap_acquire(map);
            fenced = pf;
        }
        StageInfo &si = info[s];
        const uint4 *src = reinterpret_cast<const uint4 *>(frames + pf);
        uint4 *dst = reinterpret_cast<uint4 *>(&si.fd);
#pragma unroll
        for (int k = 0; k < (int)(sizeof(FrameDesc) / 16); ++k) dst[k] = src[k];
        const int lt = t - si.fd.tile_begin;
        const int txs = si.fd.tiles_x;
        si.x0 = (lt % txs) * TW;
        si.y0 = (lt / txs) * TH;
        si.tile = t;
        const uint32_t bar = smem_addr(&full[s]);
        mbar_expect_tx(bar, BOX_BYTES);  // release: the info slot is visible with the phase
        tma_load_2d(smem_addr(smem + s * STRIDE), map, si.x0 - PADX, si.y0 - 1, bar);
    };
    if (tid == 0)
        for (int s = 0; s < kStages; ++s)
            if (first + s * step < total) fill(first + s * step, s);

    const int tx = tid % TPR, ty = tid / TPR;
    const bool refine_all = args.flags & 1;
    for (int i = 0;; ++i) {
        const int t = first + i * step;
        if (t >= total) break;
        const int s = i % kStages;
        const bool arrived = __all_sync(0xffffffffu, mbar_wait(smem_addr(&full[s]), (uint32_t)((i / kStages) & 1)));
        if (!arrived) {
            if (lane == 0) atomicOr(args.status, DEVERR_TMA_WAIT);
            return;
        }
        unsigned pending = 0;  // pixels (pr * 4 + c) that need the double-float path
        const StageInfo &si = info[s];
        const FrameDesc &fd = si.fd;
        const int W = fd.W, H = fd.H;
        OutDesc out;
        out.out = fd.out;
        out.out_pitch = fd.out_pitch;
        out.out_plane = fd.out_plane;
        out.mask = fd.mask;
        out.mask_pitch = fd.mask_pitch;
        const int x0 = si.x0 + 4 * tx;
        const int y0 = si.y0 + PR * ty;
        if (x0 < W && y0 < H) {
            const float fx = fd.fx, fy = fd.fy, u0 = fd.u0, v0 = fd.v0, thr = fd.thr;
            Win<KIND, PR> win;
            load_window<KIND, PR>(smem + s * STRIDE, SW, PADX, PR * ty, 4 * tx, win);
            const int nvalid = min(4, W - x0);
#pragma unroll
            for (int pr = 0; pr < PR; ++pr) {
                const int v = y0 + pr;
                const unsigned evm = evaluable_row<GRAD, KIND, PR>(win, pr + 1);
                float ox[4], oy[4], oz[4];
                uint8_t mk[4];
                unsigned rbits = 0;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const PixelResult r = pixel_normal<KIND, GRAD, PHI, PR>(win, evm, pr + 1, c + 1, x0 + c, v, fx, fy,
                                                                            u0, v0, thr, refine_all);
                    ox[c] = r.x;
                    oy[c] = r.y;
                    oz[c] = r.z;
                    mk[c] = r.valid ? 1 : 0;
                    rbits |= r.refine ? 1u << c : 0u;
                }
                if (v < H) {
                    store4(out, args.out_fmt, x0, v, nvalid, ox, oy, oz, mk);
                    pending |= (rbits & ((1u << nvalid) - 1u)) << (pr * 4);
                }
            }
            // Deferred refinement: rare, so it runs after the stores and off the
            // main instruction stream; a later store to the same pixel wins.
            unsigned todo = pending;
            while (todo) {
                const int b = __ffs(todo) - 1;
                todo &= todo - 1;
                const int pr = b >> 2, c = b & 3;
                const Vec3 n = refine_from_tile<KIND, GRAD, PHI>(smem + s * STRIDE, (PR * ty + pr) * SW + PADX + 4 * tx + c - 1,
                                                                 SW, x0 + c, y0 + pr, fx, fy, u0, v0);
                store1(out, args.out_fmt, x0 + c, y0 + pr, n);
            }
        }
        // count of refined pixels (diagnostics): one atomic per warp, only if any
        const unsigned nref = __reduce_add_sync(0xffffffffu, (unsigned)__popc(pending));
        if (lane == 0 && nref) atomicAdd(args.status + 1, nref);
        // release the buffer; the last warp out refills it
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            if (atomicAdd(&released[s], 1) == kWarps - 1) {
                released[s] = 0;
                __threadfence_block();
                const int tn = t + kStages * step;
                if (tn < total) {
                    fence_async_shared();
                    fill(tn, s);
                }
            }
        }
    }
}

template <int KIND>
KernelFn select_kernel(int grad, int phi, int cfg)
{
#define TFN_K(G, P, C)                                                                        \
    if (grad == G && phi == P && cfg == C) return &normals_kernel<KIND, G, P, C>;
#define TFN_KC(G, P) TFN_K(G, P, 0) TFN_K(G, P, 1) TFN_K(G, P, 2)
#define TFN_KP(G) TFN_KC(G, PHI_MEAN) TFN_KC(G, PHI_MEDIAN)
    TFN_KP(GRAD_FD) TFN_KP(GRAD_SOBEL) TFN_KP(GRAD_SCHARR) TFN_KP(GRAD_PREWITT)
#undef TFN_KP
#undef TFN_KC
#undef TFN_K
    return nullptr;
}

}  // namespace dev
}  // namespace tfn
