/*
 * tfn_scenes.c -- seeded synthetic range images (the stand-in for the paper's
 * rendered 480x640 datasets, which are not available).
 *
 * Holds no arithmetic of the normal estimator: it ray-casts planes and
 * spheres through a pinhole camera, adds depth noise and holes, and can
 * quantise to stereo disparity.  Both the oracle-side tests and the CUDA-side
 * tests/bench draw their inputs from here.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded through
 * splitmix64 (Steele, Lea & Flood, 2014); normal deviates by the Box-Muller
 * transform (1958).  All three are written here from their published
 * definitions, so a seed gives the same bits on every machine.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t *x)
{
    uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t next_u64(rng_t *r)
{
    uint64_t *s = r->s;
    uint64_t out = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return out;
}

static void seed_rng(rng_t *r, uint64_t seed)
{
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

/* uniform in [0, 1) with 53 random bits */
static double uni(rng_t *r) { return (double)(next_u64(r) >> 11) * (1.0 / 9007199254740992.0); }
static double uni_ab(rng_t *r, double a, double b) { return a + (b - a) * uni(r); }

static double gauss(rng_t *r)
{
    double u1 = uni(r), u2 = uni(r);
    if (u1 < 1e-300) u1 = 1e-300;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* Scene recipe.  Depth beyond [zmin, zmax] becomes a hole (0). */
typedef struct {
    int H, W;
    double fx, fy, u0, v0;
    double zmin, zmax;           /* kept depth range */
    int n_planes, n_spheres;
    double plane_z0, plane_z1;   /* anchor depth range of the planes */
    double max_tilt_deg;         /* plane tilt from the optical axis */
    double sphere_z0, sphere_z1; /* centre depth range */
    double radius0, radius1;
    double noise_k;              /* sigma = noise_k * Z^2 */
    double hole_frac;            /* iid zero-depth fraction */
} recipe_t;

typedef struct { double n[3], P[3]; } plane_t;
typedef struct { double C[3], r; } sphere_t;

/*
 * One frame.  depth: H*W floats (0 = hole).  Optional outputs (NULL to skip):
 * depth64: the exact ray-cast depth before noise, FP64 (0 = no hit in range);
 * prim: primitive index per pixel (-1 none; planes 0.., spheres n_planes..);
 * gt: 3 planes of H*W floats, the analytic unit normal facing the camera.
 */
static void render(const recipe_t *R, uint64_t seed, float *depth, double *depth64, int32_t *prim,
                   float *gt)
{
    rng_t rng;
    seed_rng(&rng, seed);
    plane_t pl[16];
    sphere_t sp[16];
    int np = R->n_planes < 16 ? R->n_planes : 16, ns = R->n_spheres < 16 ? R->n_spheres : 16;
    for (int k = 0; k < np; ++k) {
        double pu = uni_ab(&rng, 0, R->W), pv = uni_ab(&rng, 0, R->H);
        double z = uni_ab(&rng, R->plane_z0, R->plane_z1);
        double th = uni_ab(&rng, 0, R->max_tilt_deg) * (3.141592653589793 / 180.0);
        double ph = uni_ab(&rng, 0, 6.283185307179586);
        plane_t *p = &pl[k];
        p->P[0] = (pu - R->u0) / R->fx * z;
        p->P[1] = (pv - R->v0) / R->fy * z;
        p->P[2] = z;
        p->n[0] = sin(th) * cos(ph);
        p->n[1] = sin(th) * sin(ph);
        p->n[2] = -cos(th);
        double s = p->n[0] * p->P[0] + p->n[1] * p->P[1] + p->n[2] * p->P[2];
        if (s > 0)
            for (int c = 0; c < 3; ++c) p->n[c] = -p->n[c]; /* face the camera */
    }
    for (int k = 0; k < ns; ++k) {
        double pu = uni_ab(&rng, 0, R->W), pv = uni_ab(&rng, 0, R->H);
        double z = uni_ab(&rng, R->sphere_z0, R->sphere_z1);
        sphere_t *s = &sp[k];
        s->C[0] = (pu - R->u0) / R->fx * z;
        s->C[1] = (pv - R->v0) / R->fy * z;
        s->C[2] = z;
        s->r = uni_ab(&rng, R->radius0, R->radius1);
    }
    const int64_t HW = (int64_t)R->H * R->W;
    for (int v = 0; v < R->H; ++v)
        for (int u = 0; u < R->W; ++u) {
            double d[3] = {(u - R->u0) / R->fx, (v - R->v0) / R->fy, 1.0};
            double best = INFINITY;
            int who = -1;
            for (int k = 0; k < np; ++k) {
                const plane_t *p = &pl[k];
                double den = p->n[0] * d[0] + p->n[1] * d[1] + p->n[2] * d[2];
                if (den == 0) continue;
                double t = (p->n[0] * p->P[0] + p->n[1] * p->P[1] + p->n[2] * p->P[2]) / den;
                if (t > 0 && t < best) { best = t; who = k; }
            }
            for (int k = 0; k < ns; ++k) {
                const sphere_t *s = &sp[k];
                double a = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                double b = -2 * (d[0] * s->C[0] + d[1] * s->C[1] + d[2] * s->C[2]);
                double c = s->C[0] * s->C[0] + s->C[1] * s->C[1] + s->C[2] * s->C[2] - s->r * s->r;
                double disc = b * b - 4 * a * c;
                if (disc < 0) continue;
                double t = (-b - sqrt(disc)) / (2 * a);
                if (t > 0 && t < best) { best = t; who = np + k; }
            }
            int64_t i = (int64_t)v * R->W + u;
            int hit = who >= 0 && best >= R->zmin && best <= R->zmax;
            if (depth64) depth64[i] = hit ? best : 0.0;
            depth[i] = hit ? (float)best : 0.0f;
            if (prim) prim[i] = hit ? who : -1;
            if (gt) {
                double n[3] = {0, 0, 0};
                if (hit && who < np) {
                    for (int c = 0; c < 3; ++c) n[c] = pl[who].n[c];
                } else if (hit) {
                    const sphere_t *s = &sp[who - np];
                    for (int c = 0; c < 3; ++c) n[c] = (best * d[c] - s->C[c]) / s->r;
                }
                for (int c = 0; c < 3; ++c) gt[c * HW + i] = (float)n[c];
            }
        }
    if (R->noise_k > 0)
        for (int64_t i = 0; i < HW; ++i) {
            double g = gauss(&rng);
            if (depth[i] > 0) {
                double z = depth[i];
                depth[i] = (float)(z + R->noise_k * z * z * g);
            }
        }
    if (R->hole_frac > 0)
        for (int64_t i = 0; i < HW; ++i)
            if (uni(&rng) < R->hole_frac) depth[i] = 0.0f;
}

typedef struct {
    const recipe_t *R;
    uint64_t seed0;
    int n, next;
    float *depth;
    int32_t *prim;
    float *gt;
    pthread_mutex_t lock;
} batch_t;

static void *batch_worker(void *arg)
{
    batch_t *B = (batch_t *)arg;
    const int64_t HW = (int64_t)B->R->H * B->R->W;
    for (;;) {
        pthread_mutex_lock(&B->lock);
        int k = B->next++;
        pthread_mutex_unlock(&B->lock);
        if (k >= B->n) return NULL;
        render(B->R, B->seed0 + (uint64_t)k, B->depth + HW * k, NULL, B->prim ? B->prim + HW * k : NULL,
               B->gt ? B->gt + 3 * HW * k : NULL);
    }
}

int tfn_scene_recipe_size(void) { return (int)sizeof(recipe_t); }

/* One frame (see render()). */
int tfn_scene_render(const recipe_t *R, uint64_t seed, float *depth, double *depth64, int32_t *prim,
                     float *gt)
{
    if (!R || !depth || R->H < 1 || R->W < 1) return 1;
    render(R, seed, depth, depth64, prim, gt);
    return 0;
}

/* n frames, frame k seeded with seed0 + k, rendered on `threads` threads. */
int tfn_scene_render_batch(const recipe_t *R, uint64_t seed0, int n, float *depth, int32_t *prim,
                           float *gt, int threads)
{
    if (!R || !depth || n < 0 || R->H < 1 || R->W < 1) return 1;
    batch_t B = {R, seed0, n, 0, depth, prim, gt, PTHREAD_MUTEX_INITIALIZER};
    if (threads < 1) threads = 1;
    pthread_t t[64];
    if (threads > 64) threads = 64;
    int started = 0;
    for (int i = 0; i < threads; ++i)
        if (pthread_create(&t[i], NULL, batch_worker, &B) == 0) ++started;
    if (started == 0) batch_worker(&B);
    for (int i = 0; i < started; ++i) pthread_join(t[i], NULL);
    return 0;
}

/*
 * Stereo disparity of a depth image (Sec. III, Eq. z_d: Z = f t_c / d),
 * quantised to unsigned 16-bit fixed point with `frac_bits` fractional bits,
 * rounded to nearest, clamped to [1, 65535]; holes stay 0.  Then a
 * `hole_frac` share of pixels is zeroed iid, drawn from `seed`.
 */
int tfn_scene_disparity_u16(const float *depth, int64_t n, double f_tc, int frac_bits,
                            double hole_frac, uint64_t seed, uint16_t *out)
{
    if (!depth || !out || n < 0 || !(f_tc > 0)) return 1;
    double scale = ldexp(1.0, frac_bits);
    for (int64_t i = 0; i < n; ++i) {
        double z = depth[i];
        if (!(z > 0)) { out[i] = 0; continue; }
        double q = floor(f_tc / z * scale + 0.5);
        if (q < 1) q = 1;
        if (q > 65535) q = 65535;
        out[i] = (uint16_t)q;
    }
    if (hole_frac > 0) {
        rng_t rng;
        seed_rng(&rng, seed);
        for (int64_t i = 0; i < n; ++i)
            if (uni(&rng) < hole_frac) out[i] = 0;
    }
    return 0;
}
