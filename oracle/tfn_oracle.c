/*
 * tfn_oracle.c -- plain, slow FP64 reference of Three-Filters-to-Normal (3F2N).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only tests/, __graft_entry__.smoke() and the CPU-baseline
 * leg of bench.py may load it.  It shares no code, header, table or constant
 * with the CUDA library and includes nothing from it.
 *
 * What it computes (Fan et al., "Three-Filters-to-Normal", RA-L 2021):
 *   Sec. III, Eq. (intrinsic matrix): back-projection p = (Z(u-u0)/fx, Z(v-v0)/fy, Z).
 *   Sec. III, text after Eq. (d1/z): gradient filters on the inverse-depth image 1/Z.
 *   Sec. III, Eq. (nx2_ny2_nz2):      nx = fx d(1/Z)/du, ny = fy d(1/Z)/dv,
 *                                    n_z = -Phi{ (dx_j nx + dy_j ny) / dz_j }, j = 1..8.
 *   Sec. III, special case:          equal depths -> n = [0, 0, -1].
 *   Sec. III, Eqs. (z_d), (dd_2_dz), (nx2_ny2_nz3): disparity form, Z = f t_c / d,
 *                                    nx = dd/du, ny = dd/dv, same n_z rule.
 *
 * Readings where the paper is silent (labelled R1, R2, ...):
 *   R1 a sample is valid iff it is finite and 2^-16 <= value <= 2^16 (depth in
 *      any unit, float disparity in pixels); a 16-bit fixed-point disparity is
 *      valid iff its raw value is non-zero.  Anything else is a hole.
 *   R2 a pixel is evaluable iff it is valid and every tap with a non-zero
 *      weight in either gradient filter is inside the image and valid.
 *   R3 gradients are correlations with [-1 0 1] (horizontal) and its transpose,
 *      row/column weights FD (0 1 0)/2, Sobel (1 2 1)/8, Scharr (3 10 3)/32,
 *      Prewitt (1 1 1)/6; the weighted family (the 3x3 kernels of the
 *      brute-force search, Sec. IV) takes any row weights (w0 w1 w2) /
 *      (2 (|w0| + |w1| + |w2|)).
 *   R15 filter sizes (Fig. 2 compares "types and sizes"): a 5x5 gradient filter
 *      is separable, an antisymmetric derivative profile (d1 at offsets +-1,
 *      d2 at +-2) along its axis times a symmetric smoothing profile (s0 at 0,
 *      s1 at +-1, s2 at +-2) across it, divided by
 *      2 (d1 + 2 d2) (s0 + 2 s1 + 2 s2), so that it returns the derivative of
 *      an affine image (both sums must be non-zero).  Named members: FD5
 *      (8 -1 | 1 0 0), the fourth-order central difference; Sobel5
 *      (2 1 | 6 4 1), the binomial pair; Prewitt5 (1 2 | 1 1 1), the box pair.
 *      The candidates and Phi keep the 8-connected neighbourhood (Sec. V-A).
 *   R4 candidates come from valid neighbours with dz != 0 only.
 *   R5 Phi = median of an even count is the mean of the two middle values.
 *   R6 the normal is [0, 0, -1] if both gradients are exactly zero, or if no
 *      neighbour gives a candidate, i.e. every valid neighbour shares the
 *      centre's depth (Sec. III special case).  With 3x3 filters the second
 *      implies the first (the taps are among the neighbours); a 5x5 filter can
 *      see a depth change in its outer taps only.
 *   R7 the output is n = -n'/|n'| with n' = (nx, ny, n_z): it faces the camera.
 *   R8 invalid pixels get normal (0, 0, 0) and mask 0; evaluable ones mask 1.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_DEPTH_F32 = 0, OR_DEPTH_F16 = 1, OR_DISP_U16 = 2, OR_DISP_F32 = 3, OR_DEPTH_F64 = 100 };
enum { OR_FD = 0, OR_SOBEL = 1, OR_SCHARR = 2, OR_PREWITT = 3, OR_WEIGHTED = 4, OR_SEP5 = 5, OR_FD5 = 6,
       OR_SOBEL5 = 7, OR_PREWITT5 = 8 };
enum { OR_MEAN = 0, OR_MEDIAN = 1 };
enum { OR_LITERAL = 0, OR_ALGEBRAIC = 1 };

#define OR_OK 0
#define OR_BAD_ARG 1

static const double VALID_LO = 1.0 / 65536.0; /* 2^-16, reading R1 */
static const double VALID_HI = 65536.0;       /* 2^16 */

/* IEEE 754 binary16 -> double, from the format's definition. */
static double half_to_double(uint16_t h)
{
    int sign = (h >> 15) & 1;
    int expo = (h >> 10) & 0x1f;
    int mant = h & 0x3ff;
    double v;
    if (expo == 0)
        v = ldexp((double)mant, -24); /* subnormal: mant * 2^-14 * 2^-10 */
    else if (expo == 31)
        v = mant ? NAN : INFINITY;
    else
        v = ldexp((double)(mant + 1024), expo - 25);
    return sign ? -v : v;
}

/* Reads the raw sample at (x, y) as a double, before the validity rule. */
static double read_sample(const void *in, int64_t pitch, int type, double disp_scale, int x, int y)
{
    const char *row = (const char *)in + (int64_t)y * pitch;
    switch (type) {
    case OR_DEPTH_F32:
    case OR_DISP_F32: return (double)((const float *)row)[x];
    case OR_DEPTH_F16: return half_to_double(((const uint16_t *)row)[x]);
    case OR_DISP_U16: {
        uint16_t raw = ((const uint16_t *)row)[x];
        return raw == 0 ? 0.0 : (double)raw * disp_scale;
    }
    case OR_DEPTH_F64: return ((const double *)row)[x];
    }
    return NAN;
}

static int is_valid(double s) { return isfinite(s) && s >= VALID_LO && s <= VALID_HI; }

/* Profiles of the gradient filters (readings R3, R15) on a 5x5 window: the
 * horizontal filter's tap at offset (dv, du) is rho[dv+2] * sign(du) *
 * delta[|du|] / norm, the vertical one its transpose.  The 3x3 filters use
 * the inner window only (rho[0] = rho[4] = 0, delta[2] = 0). */
static void filter_profile(int grad, const double *custom, double rho[5], double delta[3], double *norm)
{
    double w[3], d1 = 1, d2 = 0, s0, s1, s2;
    delta[0] = 0;
    switch (grad) {
    case OR_SEP5: d1 = custom[0]; d2 = custom[1]; s0 = custom[2]; s1 = custom[3]; s2 = custom[4]; break;
    case OR_FD5: d1 = 8; d2 = -1; s0 = 1; s1 = 0; s2 = 0; break;
    case OR_SOBEL5: d1 = 2; d2 = 1; s0 = 6; s1 = 4; s2 = 1; break;
    case OR_PREWITT5: d1 = 1; d2 = 2; s0 = 1; s1 = 1; s2 = 1; break;
    default:
        switch (grad) {
        case OR_WEIGHTED: w[0] = custom[0]; w[1] = custom[1]; w[2] = custom[2]; break;
        case OR_FD: w[0] = 0; w[1] = 1; w[2] = 0; break;
        case OR_SOBEL: w[0] = 1; w[1] = 2; w[2] = 1; break;
        case OR_SCHARR: w[0] = 3; w[1] = 10; w[2] = 3; break;
        default: w[0] = 1; w[1] = 1; w[2] = 1; break;
        }
        rho[0] = 0; rho[1] = w[0]; rho[2] = w[1]; rho[3] = w[2]; rho[4] = 0;
        delta[1] = 1; delta[2] = 0;
        *norm = 2 * (fabs(w[0]) + fabs(w[1]) + fabs(w[2]));
        return;
    }
    rho[0] = s2; rho[1] = s1; rho[2] = s0; rho[3] = s1; rho[4] = s2;
    delta[1] = d1; delta[2] = d2;
    *norm = 2 * (d1 + 2 * d2) * (s0 + 2 * s1 + 2 * s2);
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

typedef struct {
    const void *in;
    int64_t pitch;
    int H, W, type, grad, phi, form;
    double disp_scale, fx, fy, u0, v0, tc;
    double cw[5];          /* weights of OR_WEIGHTED (w0 w1 w2) or OR_SEP5 (d1 d2 s0 s1 s2) */
    double *normals;       /* 3 planes of H*W doubles */
    uint8_t *mask;         /* H*W */
    double *cands;         /* optional: 8 planes of H*W candidates (NAN = excluded) */
    double *nprime;        /* optional: 3 planes of H*W unnormalised n' */
} job_t;

/* One pixel.  Writes normal, mask and (optionally) candidates / n'. */
static void pixel(const job_t *J, int u, int v)
{
    const int64_t HW = (int64_t)J->H * J->W, idx = (int64_t)v * J->W + u;
    const int disparity = (J->type == OR_DISP_U16 || J->type == OR_DISP_F32);
    /* the window: 3x3 for the 3x3 filters, 5x5 for the 5x5 ones (R15) */
    double rho[5], delta[3], norm;
    filter_profile(J->grad, J->cw, rho, delta, &norm);
    const int reach = (rho[0] != 0 || rho[4] != 0 || delta[2] != 0) ? 2 : 1;
    double s[5][5]; /* samples, s[dv+2][du+2]; 0 outside the window */
    int ok[5][5];
    for (int dv = -2; dv <= 2; ++dv)
        for (int du = -2; du <= 2; ++du) {
            int x = u + du, y = v + dv;
            int inside = abs(du) <= reach && abs(dv) <= reach && x >= 0 && x < J->W && y >= 0 && y < J->H;
            double val = inside ? read_sample(J->in, J->pitch, J->type, J->disp_scale, x, y) : 0.0;
            s[dv + 2][du + 2] = val;
            /* R1: fixed-point disparity is a hole only where the raw value is 0 */
            ok[dv + 2][du + 2] = inside && (J->type == OR_DISP_U16 ? val > 0.0 : is_valid(val));
        }
    double *n0 = J->normals, *n1 = J->normals + HW, *n2 = J->normals + 2 * HW;
    if (J->cands)
        for (int j = 0; j < 8; ++j) J->cands[j * HW + idx] = NAN;
    if (J->nprime)
        for (int c = 0; c < 3; ++c) J->nprime[c * HW + idx] = 0.0;

    /* Reading R2: evaluable pixels. */
    int evaluable = ok[2][2];
    for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b) {
            int du = b - 2, dv = a - 2;
            /* tap weight in the horizontal filter: rho[dv+2] sign(du) delta[|du|]; vertical: transposed */
            int used = (rho[a] != 0 && du != 0 && delta[abs(du)] != 0) ||
                       (rho[b] != 0 && dv != 0 && delta[abs(dv)] != 0);
            if (used && !ok[a][b]) evaluable = 0;
        }
    if (!evaluable) {
        n0[idx] = n1[idx] = n2[idx] = 0.0;
        J->mask[idx] = 0;
        return;
    }

    /* Sec. III: the filters run on the inverse-depth image 1/Z (depth form) or
     * directly on the disparity image (disparity form, Eq. nx2_ny2_nz3). */
    double img[5][5];
    for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b)
            img[a][b] = ok[a][b] ? (disparity ? s[a][b] : 1.0 / s[a][b]) : 0.0;
    /* Correlation with the derivative profile: per row (column) the weighted
     * differences of the taps at +-1 and +-2, then weighted by the row
     * (column) weight.  Equal taps give an exact zero, so the special case
     * below is decided exactly. */
    double gu = 0, gv = 0;
    for (int k = 0; k < 5; ++k) {
        if (rho[k] == 0) continue;
        double hu = 0, hv = 0;
        for (int b = 1; b <= 2; ++b) {
            if (delta[b] == 0) continue;
            hu += delta[b] * (img[k][2 + b] - img[k][2 - b]);
            hv += delta[b] * (img[2 + b][k] - img[2 - b][k]);
        }
        gu += rho[k] * hu;
        gv += rho[k] * hv;
    }
    gu /= norm;
    gv /= norm;
    J->mask[idx] = 1;
    if (gu == 0.0 && gv == 0.0) { /* reading R6 / Sec. III special case */
        n0[idx] = 0.0; n1[idx] = 0.0; n2[idx] = -1.0;
        return;
    }

    /* Eq. (nx2_ny2_nz2) / (nx2_ny2_nz3). */
    double nx, ny;
    if (disparity) { nx = gu; ny = gv; }
    else { nx = J->fx * gu; ny = J->fy * gv; }

    /* Depth of every neighbour: Z directly, or Z = f t_c / d (Eq. z_d). */
    double Z[3][3]; /* the 8-connected neighbourhood, Z[dv+1][du+1] */
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            Z[a][b] = ok[a + 1][b + 1] ? (disparity ? J->fx * J->tc / s[a + 1][b + 1] : s[a + 1][b + 1]) : 0.0;

    double c[8];
    int m = 0;
    int j = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            int du = b - 1, dv = a - 1;
            if (du == 0 && dv == 0) continue;
            int slot = j++;
            if (!ok[a + 1][b + 1]) continue;
            double dz = Z[a][b] - Z[1][1];
            if (dz == 0.0) continue; /* reading R4 */
            double cand;
            if (J->form == OR_LITERAL) {
                /* Eq. (intrinsic matrix): back-project both points, r = q - p. */
                double px = Z[1][1] * (u - J->u0) / J->fx, py = Z[1][1] * (v - J->v0) / J->fy;
                double qx = Z[a][b] * (u + du - J->u0) / J->fx, qy = Z[a][b] * (v + dv - J->v0) / J->fy;
                cand = ((qx - px) * nx + (qy - py) * ny) / dz;
            } else {
                /* Algebraic form: dx = (dz (u-u0) + Z_j du)/fx, dy likewise, so
                 * c = [(u-u0) gu + (v-v0) gv + Z_j (du gu + dv gv)/dz] * k,
                 * k = 1 (depth form) or 1/f (disparity form). */
                double A = (u - J->u0) * gu + (v - J->v0) * gv;
                double R = Z[a][b] * (du * gu + dv * gv) / dz;
                cand = disparity ? (A + R) / J->fx : (A + R);
            }
            c[m++] = cand;
            if (J->cands) J->cands[slot * HW + idx] = cand;
        }

    if (m == 0) { /* reading R6: every valid neighbour at the centre's depth */
        n0[idx] = 0.0; n1[idx] = 0.0; n2[idx] = -1.0;
        return;
    }
    /* Phi: mean or median (reading R5). */
    double phi;
    if (J->phi == OR_MEAN) {
        double acc = 0;
        for (int k = 0; k < m; ++k) acc += c[k];
        phi = acc / m;
    } else {
        qsort(c, m, sizeof(double), cmp_double);
        phi = (m & 1) ? c[m / 2] : 0.5 * (c[m / 2 - 1] + c[m / 2]);
    }
    double nz = -phi;
    if (J->nprime) {
        J->nprime[idx] = nx; J->nprime[HW + idx] = ny; J->nprime[2 * HW + idx] = nz;
    }
    double len = sqrt(nx * nx + ny * ny + nz * nz);
    n0[idx] = -nx / len; /* reading R7 */
    n1[idx] = -ny / len;
    n2[idx] = -nz / len;
}

static void run_rows(const job_t *J, int y0, int y1)
{
    for (int v = y0; v < y1; ++v)
        for (int u = 0; u < J->W; ++u) pixel(J, u, v);
}

static int check_args(const void *in, int64_t pitch, int H, int W, int type, int grad, int phi,
                      int form, double fx, double fy, double tc, double disp_scale)
{
    if (!in || H < 1 || W < 1) return OR_BAD_ARG;
    if (type != OR_DEPTH_F32 && type != OR_DEPTH_F16 && type != OR_DISP_U16 && type != OR_DISP_F32 &&
        type != OR_DEPTH_F64)
        return OR_BAD_ARG;
    if (grad < 0 || grad > OR_PREWITT5 || phi < 0 || phi > 1 || form < 0 || form > 1) return OR_BAD_ARG;
    if (!(fx > 0) || !(fy > 0)) return OR_BAD_ARG;
    int esz = type == OR_DEPTH_F64 ? 8 : (type == OR_DEPTH_F32 || type == OR_DISP_F32) ? 4 : 2;
    if (pitch < (int64_t)W * esz) return OR_BAD_ARG;
    if (type == OR_DISP_U16 || type == OR_DISP_F32) {
        if (fx != fy || !(tc > 0)) return OR_BAD_ARG;
        if (type == OR_DISP_U16 && !(disp_scale > 0)) return OR_BAD_ARG;
    }
    return OR_OK;
}

/*
 * Normals of one frame.  `normals` receives 3 planes of H*W doubles (x, y, z),
 * `mask` H*W bytes.  `cands` (8*H*W, neighbour raster order) and `nprime`
 * (3*H*W) are optional diagnostics, NULL to skip.
 */
int tfn_oracle_normals_weighted(const void *in, int64_t pitch, int H, int W, int type, double disp_scale,
                                double fx, double fy, double u0, double v0, double tc, int grad,
                                const double *weights, int phi, int form, double *normals, uint8_t *mask,
                                double *cands, double *nprime)
{
    int st = check_args(in, pitch, H, W, type, grad, phi, form, fx, fy, tc, disp_scale);
    if (st || !normals || !mask) return st ? st : OR_BAD_ARG;
    const int nw = grad == OR_WEIGHTED ? 3 : grad == OR_SEP5 ? 5 : 0;
    if (nw) {
        if (!weights) return OR_BAD_ARG;
        for (int k = 0; k < nw; ++k)
            if (!isfinite(weights[k])) return OR_BAD_ARG;
        if (grad == OR_WEIGHTED && weights[0] == 0 && weights[1] == 0 && weights[2] == 0) return OR_BAD_ARG;
        /* OR_SEP5: the profiles must measure a derivative (reading R15) */
        if (grad == OR_SEP5 && (weights[0] + 2 * weights[1] == 0 || weights[2] + 2 * weights[3] + 2 * weights[4] == 0))
            return OR_BAD_ARG;
    }
    job_t J = {in, pitch, H, W, type, grad, phi, form, disp_scale, fx, fy, u0, v0, tc, {0, 0, 0, 0, 0},
               normals, mask, cands, nprime};
    for (int k = 0; k < nw; ++k) J.cw[k] = weights[k];
    run_rows(&J, 0, H);
    return OR_OK;
}

int tfn_oracle_normals(const void *in, int64_t pitch, int H, int W, int type, double disp_scale,
                       double fx, double fy, double u0, double v0, double tc, int grad, int phi,
                       int form, double *normals, uint8_t *mask, double *cands, double *nprime)
{
    if (grad == OR_WEIGHTED || grad == OR_SEP5) return OR_BAD_ARG; /* need weights: tfn_oracle_normals_weighted */
    return tfn_oracle_normals_weighted(in, pitch, H, W, type, disp_scale, fx, fy, u0, v0, tc, grad, NULL, phi, form,
                                       normals, mask, cands, nprime);
}

typedef struct {
    job_t *jobs;
    int n, next;
    pthread_mutex_t lock;
} pool_t;

static void *worker(void *arg)
{
    pool_t *P = (pool_t *)arg;
    for (;;) {
        pthread_mutex_lock(&P->lock);
        int k = P->next++;
        pthread_mutex_unlock(&P->lock);
        if (k >= P->n) return NULL;
        run_rows(&P->jobs[k], 0, P->jobs[k].H);
    }
}

/*
 * Normals of n same-shaped frames stored back to back (frame stride =
 * H * pitch bytes; outputs frame-major), spread over `threads` threads, one
 * frame at a time per thread.
 */
int tfn_oracle_normals_batch(const void *in, int64_t pitch, int n, int H, int W, int type,
                             double disp_scale, double fx, double fy, double u0, double v0,
                             double tc, int grad, int phi, int form, double *normals,
                             uint8_t *mask, int threads)
{
    int st = check_args(in, pitch, H, W, type, grad, phi, form, fx, fy, tc, disp_scale);
    if (st || !normals || !mask || n < 0 || grad == OR_WEIGHTED || grad == OR_SEP5) return st ? st : OR_BAD_ARG;
    if (threads < 1) threads = 1;
    job_t *jobs = (job_t *)calloc(n > 0 ? n : 1, sizeof(job_t));
    if (!jobs) return OR_BAD_ARG;
    const int64_t HW = (int64_t)H * W;
    for (int k = 0; k < n; ++k) {
        job_t J = {(const char *)in + (int64_t)k * H * pitch, pitch, H, W, type, grad, phi, form,
                   disp_scale, fx, fy, u0, v0, tc, {0, 0, 0, 0, 0}, normals + 3 * HW * k, mask + HW * k, NULL, NULL};
        jobs[k] = J;
    }
    pool_t P = {jobs, n, 0, PTHREAD_MUTEX_INITIALIZER};
    if (threads == 1) {
        worker(&P);
    } else {
        pthread_t *t = (pthread_t *)calloc(threads, sizeof(pthread_t));
        int started = 0;
        for (int i = 0; i < threads; ++i)
            if (pthread_create(&t[i], NULL, worker, &P) == 0) ++started;
        if (started == 0) worker(&P);
        for (int i = 0; i < started; ++i) pthread_join(t[i], NULL);
        free(t);
    }
    free(jobs);
    return OR_OK;
}

/*
 * Back-projected point cloud of one frame, every valid sample (Sec. III, Eq.
 * intrinsic matrix: p = (Z (u - u0)/fx, Z (v - v0)/fy, Z); disparity input:
 * Z = f t_c / d, Eq. z_d, with f = fx = fy).  `points` receives 3 planes of
 * H*W doubles (X, Y, Z); holes (reading R1) give (0, 0, 0).
 */
int tfn_oracle_points(const void *in, int64_t pitch, int H, int W, int type, double disp_scale, double fx,
                      double fy, double u0, double v0, double tc, double *points)
{
    int st = check_args(in, pitch, H, W, type, OR_FD, OR_MEAN, OR_LITERAL, fx, fy, tc, disp_scale);
    if (st || !points) return st ? st : OR_BAD_ARG;
    const int disparity = (type == OR_DISP_U16 || type == OR_DISP_F32);
    const int64_t HW = (int64_t)H * W;
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            const int64_t idx = (int64_t)v * W + u;
            const double s = read_sample(in, pitch, type, disp_scale, u, v);
            const int ok = type == OR_DISP_U16 ? s > 0 : is_valid(s);
            double X = 0, Y = 0, Z = 0;
            if (ok) {
                Z = disparity ? fx * tc / s : s;
                X = Z * (u - u0) / fx;
                Y = Z * (v - v0) / fy;
            }
            points[idx] = X;
            points[HW + idx] = Y;
            points[2 * HW + idx] = Z;
        }
    return OR_OK;
}

/* Angle in degrees between two 3-vectors, atan2(|a x b|, a.b) (Sec. IV-A, Eq.
 * ea_ep defines psi = arccos of the normalised dot product; atan2 gives the
 * same angle without the loss of accuracy of arccos near 0). */
double tfn_oracle_angle_deg(const double a[3], const double b[3])
{
    double cx = a[1] * b[2] - a[2] * b[1];
    double cy = a[2] * b[0] - a[0] * b[2];
    double cz = a[0] * b[1] - a[1] * b[0];
    double d = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
    return atan2(sqrt(cx * cx + cy * cy + cz * cz), d) * (180.0 / M_PI);
}
