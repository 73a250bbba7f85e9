// tfn_api.cu -- host side of the C ABI declared in include/tfn.h.
//
// Validates requests, builds per-frame descriptors and TMA tensor maps in a
// ring of scratch slots, launches the persistent kernel, and implements the
// pipelined host-buffer path.  No C++ exception leaves this file.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/tfn.h"
#include "tfn_ctx.h"
#include "tfn_internal.h"

namespace tfn {
KernelFn kernels_depth_f32(int grad, int phi, int cfg, bool noref);
KernelFn kernels_depth_f16(int grad, int phi, int cfg, bool noref);
KernelFn kernels_disp_u16(int grad, int phi, int cfg, bool noref);
KernelFn kernels_disp_f32(int grad, int phi, int cfg, bool noref);
KernelFn kernels_depth_f32_fdmean(int cfg);
KernelFn kernels_depth_f16_fdmean(int cfg);
KernelFn kernels_disp_u16_fdmean(int cfg);
KernelFn kernels_disp_f32_fdmean(int cfg);
KernelFn refiners_depth_f32(int grad, int phi);
KernelFn refiners_depth_f16(int grad, int phi);
KernelFn refiners_disp_u16(int grad, int phi);
KernelFn refiners_disp_f32(int grad, int phi);

KernelFn kernel_for(int kind, int grad, int phi, int cfg, bool noref)
{
    if (grad_is_sep5(grad)) grad = GRAD_SEP5;  // the named 5x5 filters are weight presets
    if (grad == GRAD_FD && phi == PHI_MEAN && !noref) {  // (their own translation units)
        switch (kind) {
        case KIND_DEPTH_F32: return kernels_depth_f32_fdmean(cfg);
        case KIND_DEPTH_F16: return kernels_depth_f16_fdmean(cfg);
        case KIND_DISP_U16: return kernels_disp_u16_fdmean(cfg);
        case KIND_DISP_F32: return kernels_disp_f32_fdmean(cfg);
        }
        return nullptr;
    }
    switch (kind) {
    case KIND_DEPTH_F32: return kernels_depth_f32(grad, phi, cfg, noref);
    case KIND_DEPTH_F16: return kernels_depth_f16(grad, phi, cfg, noref);
    case KIND_DISP_U16: return kernels_disp_u16(grad, phi, cfg, noref);
    case KIND_DISP_F32: return kernels_disp_f32(grad, phi, cfg, noref);
    }
    return nullptr;
}

KernelFn refiner_for(int kind, int grad, int phi)
{
    if (grad_is_sep5(grad)) grad = GRAD_SEP5;
    switch (kind) {
    case KIND_DEPTH_F32: return refiners_depth_f32(grad, phi);
    case KIND_DEPTH_F16: return refiners_depth_f16(grad, phi);
    case KIND_DISP_U16: return refiners_disp_u16(grad, phi);
    case KIND_DISP_F32: return refiners_disp_f32(grad, phi);
    }
    return nullptr;
}
}  // namespace tfn

using namespace tfn;

namespace tfn {

thread_local char g_cuda_err[256] = "";

bool cuda_ok(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return true;
    snprintf(g_cuda_err, sizeof g_cuda_err, "%s: %s", what, cudaGetErrorString(e));
    return false;
}

}  // namespace tfn

namespace {

#define TFN_CUDA(call)                                   \
    do {                                                 \
        if (!cuda_ok((call), #call)) return TFN_ERR_CUDA; \
    } while (0)

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

bool load_encode()
{
    std::call_once(g_encode_once, [] {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    });
    return g_encode != nullptr;
}

}  // namespace


namespace tfn {

tfn_status ctx_alloc(tfn_ctx *c, void **p, size_t bytes)
{
    if (c->budget && c->used + bytes > c->budget) return TFN_ERR_OUT_OF_MEMORY;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return TFN_ERR_OUT_OF_MEMORY;
    }
    if (!cuda_ok(e, "cudaMalloc")) return TFN_ERR_CUDA;
    c->used += bytes;
    return TFN_OK;
}

void ctx_free(tfn_ctx *c, void *&p, size_t bytes)
{
    if (p) {
        cudaFree(p);
        c->used -= bytes;
        p = nullptr;
    }
}


bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }
bool mult16(int64_t x) { return (x & 15) == 0; }

int out_elem_bytes(int fmt)
{
    return fmt == OUT_F32 || fmt == OUT_OCT16 ? 4 : (fmt == OUT_F16 || fmt == OUT_BF16) ? 2 : 8;
}

tfn_status validate_method(const tfn_method *m)
{
    if (!m) return TFN_ERR_INVALID_ARG;
    if (m->estimator != TFN_EST_3F2N && m->estimator != TFN_EST_PLANEPCA) return TFN_ERR_INVALID_ARG;
    if (m->grad < 0 || m->grad > GRAD_PREWITT5 || m->phi < 0 || m->phi >= PHI_COUNT || m->output < 0 ||
        m->output > OUT_OCT16 || (m->flags & ~(TFN_FLAG_REFINE_ALL | TFN_FLAG_TEST_WAIT_TIMEOUT | TFN_FLAG_FULL_BOUND)))
        return TFN_ERR_INVALID_ARG;
    if (m->grad == GRAD_WEIGHTED) {
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(m->weights[k])) return TFN_ERR_INVALID_ARG;
        if (m->weights[0] == 0.f && m->weights[1] == 0.f && m->weights[2] == 0.f) return TFN_ERR_INVALID_ARG;
    }
    if (m->grad == GRAD_SEP5) {
        // (d1 d2 s0 s1 s2): the profiles must measure a derivative, so neither
        // d1 + 2 d2 nor s0 + 2 s1 + 2 s2 may vanish (computed in double: exact)
        const float *w = m->weights;
        for (int k = 0; k < 5; ++k)
            if (!std::isfinite(w[k])) return TFN_ERR_INVALID_ARG;
        if ((double)w[0] + 2.0 * w[1] == 0.0 || (double)w[2] + 2.0 * w[3] + 2.0 * w[4] == 0.0)
            return TFN_ERR_INVALID_ARG;
    }
    return TFN_OK;
}

bool finite_in(float x, float lo, float hi) { return std::isfinite(x) && x >= lo && x <= hi; }

// `host` relaxes nothing but the meaning of the pointers (host vs device).
tfn_status validate_frame(const tfn_frame *f, int out_fmt)
{
    if (!f || !f->input || !f->normals || !f->mask) return TFN_ERR_INVALID_ARG;
    if (f->height < 1 || f->width < 1 || f->height > 32768 || f->width > 32768) return TFN_ERR_INVALID_ARG;
    if (f->input_type < 0 || f->input_type >= KIND_COUNT) return TFN_ERR_INVALID_ARG;
    const tfn_camera &c = f->cam;
    if (!finite_in(c.fx, 1.0f / 256, 16777216.f) || !finite_in(c.fy, 1.0f / 256, 16777216.f) ||
        !finite_in(c.u0, -16777216.f, 16777216.f) || !finite_in(c.v0, -16777216.f, 16777216.f))
        return TFN_ERR_INVALID_ARG;
    const bool disp = f->input_type == KIND_DISP_U16 || f->input_type == KIND_DISP_F32;
    if (disp) {
        if (!(c.baseline > 0) || !std::isfinite(c.baseline)) return TFN_ERR_INVALID_ARG;
        if (f->input_type == KIND_DISP_U16 && !(f->disp_scale > 0 && std::isfinite(f->disp_scale)))
            return TFN_ERR_INVALID_ARG;
        if (c.fx != c.fy) return TFN_ERR_UNSUPPORTED;
    }
    const int64_t es = kind_elem_size(f->input_type);
    const int64_t ob = out_elem_bytes(out_fmt);
    if (f->input_pitch < f->width * es || f->normals_pitch < f->width * ob || f->mask_pitch < f->width)
        return TFN_ERR_INVALID_ARG;
    const bool planar = out_fmt <= OUT_BF16;
    if (planar && f->normals_plane_stride < f->normals_pitch * (int64_t)f->height) return TFN_ERR_INVALID_ARG;
    if (!aligned16(f->input) || !aligned16(f->normals) || !aligned16(f->mask) || !mult16(f->input_pitch) ||
        !mult16(f->normals_pitch) || !mult16(f->mask_pitch) || (planar && !mult16(f->normals_plane_stride)))
        return TFN_ERR_MISALIGNED;
    if (f->points) {
        if (f->points_pitch < (int64_t)f->width * 4 || f->points_plane_stride < f->points_pitch * (int64_t)f->height)
            return TFN_ERR_INVALID_ARG;
        if (!aligned16(f->points) || !mult16(f->points_pitch) || !mult16(f->points_plane_stride))
            return TFN_ERR_MISALIGNED;
    }
    return TFN_OK;
}

// Per-pixel refinement threshold: a pixel is recomputed in double-float when
// its FP32 error bound, fixed u + K1 u bound/|n'|, could exceed 3/4 of the
// 1e-3 degree budget (u = 2^-24); the kernel compares bound with thr |n'|.
//
// Mean: bound = sum_p |num_p| (|rho_j| + |rho_-j|) over the four pairs of
// opposite neighbours (j, -j) with numerators G_u, G_v, G_u + G_v, G_u - G_v;
// median: the larger |middle candidate|, K1 = 11.  cA bounds |A|/|n'|, A =
// (u-u0) G_u + (v-v0) G_v, |n'| >= |(fx G_u, fy G_v)|.  fixed = 6 + 4 cA +
// 32/min(fx, fy) covers the roundings of A, n' and the normalisation.
//
// Compensated gradients (h + l to about u^2; every filter but FD on depth
// with the mean): K1 = 23 covers the per-edge reciprocal, rho, numerator,
// product and accumulation roundings.
//
// One-pass FD gradients on depth with the mean (kFdOnePassMean), worst case
// to first order in u: the edge reciprocal r = d rcp(d^2 + eps) is within
// 4u of 1/d (square, reciprocal within one ulp, product; eps below 2^-32 of
// d^2), 5u if the difference d itself rounds; rho = s r within 6u; a pair's
// rho_j - rho_-j within 7u of |rho_j| + |rho_-j|; the gradients within 5u, so
// num_p * (rho_j - rho_-j) within 12u |num_p| (|rho_j| + |rho_-j|) for the axis
// pairs and 8u of that plus 5u (|G_u| + |G_v|) (|rho_j| + |rho_-j|) for the
// diagonal ones; the four-term FMA chain adds 4u sum_p |num_p| (...).  That is
// 16u bound + 5u (|G_u| + |G_v|) (diagonal magnitudes): K1 = 17, and the
// kernel adds 0.3 (|G_u| + |G_v|) (>= 5/17) to the diagonal weights.  The
// gradients' 5u also reach (nx', ny') and A: 5 + 5 sqrt(2) cA more in fixed.
float refine_threshold(const tfn_frame &f, int grad, int phi)
{
    const double u = std::ldexp(1.0, -24);
    const double tol_part = 0.75 * 1e-3 * M_PI / 180.0;
    const double mu = std::max(std::fabs(0.0 - f.cam.u0), std::fabs(f.width - 1.0 - f.cam.u0));
    const double mv = std::max(std::fabs(0.0 - f.cam.v0), std::fabs(f.height - 1.0 - f.cam.v0));
    const double cA = std::sqrt((mu / f.cam.fx) * (mu / f.cam.fx) + (mv / f.cam.fy) * (mv / f.cam.fy));
    const bool depth = f.input_type == KIND_DEPTH_F32 || f.input_type == KIND_DEPTH_F16;
    const bool one_pass = kFdOnePassMean && grad == GRAD_FD && phi == PHI_MEAN && depth;
    const double fixed = (6.0 + 4.0 * cA + 32.0 / std::min(f.cam.fx, f.cam.fy) +
                          (one_pass ? 5.0 + 5.0 * std::sqrt(2.0) * cA : 0.0)) * u;
    const double k1 = phi == PHI_MEAN ? (one_pass ? 17.0 : 23.0) : 11.0;
    const double t = (tol_part - fixed) / (k1 * u);
    return t > 0 ? (float)t : 0.f;
}

// Whether no pixel of these frames can be flagged for refinement, so that
// the launch may run the NOREF kernel (no error bound, no refinement test,
// no refinement kernel; the same result bits).  Only FP16 depth with the FD
// filter qualifies, by the spacing of binary16: two distinct samples a < b
// differ by at least one ulp of a, which is at least 2^-11 a (2^-10 a for
// subnormal a), so |rho_j| = Z_j / |Z_j - Z_i| <= 2^11 + 1 for every kept
// neighbour (Z_j the smaller: <= 2^11; the larger: 1 + Z_i / (Z_j - Z_i)).
// With g = |G_u| + |G_v|, every weight of the bound is at most 1.3 g (mean:
// |G_u|, |G_v|, |G_u +- G_v| + 0.3 g) or g (median), so bound <= 1.3 g m rho_max
// (mean, over its m kept neighbours) or g rho_max (median: one candidate),
// while |n'| >= m min(fx, fy) g / sqrt(2) (the mean's n' is scaled by m) or
// min(fx, fy) g / sqrt(2): bound / |n'| <= c rho_max / min(fx, fy), c = 1.3
// sqrt(2) or sqrt(2), whatever the depths.  A frame qualifies when that is
// below its threshold (with a margin for the FP32 roundings of rho, m and
// |n'|, all within a few u); at the usual 480x640 intrinsics it is 7.8
// against 11.7 (mean) and 6.0 against 19.1 (median).
bool refinement_idle(const tfn_frame *frames, int n, const tfn_method &m)
{
    if (method_grad(m) != GRAD_FD || (m.flags & (TFN_FLAG_REFINE_ALL | TFN_FLAG_FULL_BOUND))) return false;
    const int phi = method_phi(m);
    const double rho_max = 2049.0;
    const double c = (phi == PHI_MEAN ? 1.3 : 1.0) * std::sqrt(2.0);
    for (int i = 0; i < n; ++i) {
        const tfn_frame &f = frames[i];
        if (f.input_type != KIND_DEPTH_F16) return false;
        const double ratio = c * rho_max / std::min(f.cam.fx, f.cam.fy) * (1.0 + 1e-3);
        if (!(ratio < (double)refine_threshold(f, GRAD_FD, phi))) return false;
    }
    return n > 0;
}

tfn_status encode_map(CUtensorMap *map, const tfn_frame &f, int cfg)
{
    if (!load_encode()) {
        snprintf(g_cuda_err, sizeof g_cuda_err, "cuTensorMapEncodeTiled unavailable");
        return TFN_ERR_CUDA;
    }
    const int kind = f.input_type;
    CUtensorMapDataType dt = kind == KIND_DEPTH_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                             : kind == KIND_DISP_U16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                                                     : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    cuuint64_t dims[2] = {(cuuint64_t)f.width, (cuuint64_t)f.height};
    cuuint64_t strides[1] = {(cuuint64_t)f.input_pitch};
    cuuint32_t box[2] = {(cuuint32_t)box_w(kind, cfg), (cuuint32_t)box_h(cfg)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, dt, 2, const_cast<void *>(f.input), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        snprintf(g_cuda_err, sizeof g_cuda_err, "cuTensorMapEncodeTiled failed (%d)", (int)r);
        return TFN_ERR_CUDA;
    }
    return TFN_OK;
}

// Fills the device descriptor of one frame for tile shape `cfg`.
FrameDesc describe_frame(const tfn_frame &f, int cfg, const tfn_method &m, int tile_begin)
{
    const int tw = kCfgs[cfg].tw;
    FrameDesc fd;
    memset(&fd, 0, sizeof fd);
    fd.out = (char *)f.normals;
    fd.out_pitch = f.normals_pitch;
    fd.out_plane = f.normals_plane_stride;
    fd.mask = f.mask;
    fd.mask_pitch = f.mask_pitch;
    fd.in = f.input;
    fd.in_pitch = f.input_pitch;
    fd.pts = (char *)f.points;
    fd.pts_pitch = f.points ? f.points_pitch : 0;
    fd.pts_plane = f.points ? f.points_plane_stride : 0;
    // Z = f t_c / d with d = raw * disp_scale for 16-bit disparity (Eq. z_d)
    if (f.input_type == KIND_DISP_U16)
        fd.ztc = (float)((double)f.cam.fx * f.cam.baseline / f.disp_scale);
    else if (f.input_type == KIND_DISP_F32)
        fd.ztc = (float)((double)f.cam.fx * f.cam.baseline);
    fd.H = f.height;
    fd.W = f.width;
    fd.tiles_x = (f.width + tw - 1) / tw;
    fd.tile_begin = tile_begin;
    fd.fx = f.cam.fx;
    fd.fy = f.cam.fy;
    fd.u0 = f.cam.u0;
    fd.v0 = f.cam.v0;
    fd.thr = refine_threshold(f, m.grad, m.phi);
    fd.kind = f.input_type;
    return fd;
}

int frame_tiles(const tfn_frame &f, int cfg)
{
    const int tw = kCfgs[cfg].tw, th = kCfgs[cfg].th;
    return ((f.width + tw - 1) / tw) * ((f.height + th - 1) / th);
}

// The launch (kernel, grid, arguments, and the refinement kernel that
// follows it, if any) for frames of one input kind whose descriptors and
// tensor maps are already in device memory.  spec.grid == 0: nothing to run.
tfn_status make_launch(int kind, const tfn_method &m, int cfg, bool noref, const FrameDesc *d_frames,
                       const CUtensorMap *d_maps, uint32_t *d_status, void *d_refine, int refine_cap, int nframes,
                       int total_tiles, int num_sms, LaunchSpec *spec)
{
    const int grad = method_grad(m);
    LaunchSpec &L = *spec;
    L.fn = kernel_for(kind, grad, method_phi(m), cfg, noref);
    if (!L.fn) return TFN_ERR_UNSUPPORTED;
    L.threads = cfg_threads(cfg, grad);
    L.smem = smem_bytes(kind, cfg, grad);
    if (!cuda_ok(cudaFuncSetAttribute((const void *)L.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem),
                 "cudaFuncSetAttribute"))
        return TFN_ERR_CUDA;
    int per_sm = 0;
    if (!cuda_ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)L.fn, L.threads, L.smem),
                 "cudaOccupancyMaxActiveBlocksPerMultiprocessor"))
        return TFN_ERR_CUDA;
    if (per_sm < 1) per_sm = 1;
    // one warp per work item at a time: no more CTAs than items / warps per CTA
    const int nw = cta_warps(cfg, grad);
    L.grid = std::max(0, std::min((total_tiles + nw - 1) / nw, per_sm * num_sms));
    // the refinement kernel of this method (none for PlanePCA, which never flags a pixel)
    L.rf = nullptr;
    if (grad != GRAD_PLANEPCA && !noref && !refines_in_kernel(cfg, grad, method_phi(m)) &&
        !(L.rf = refiner_for(kind, grad, method_phi(m))))
        return TFN_ERR_UNSUPPORTED;
    // its grid: the flagged pixels (about one per thousand on noisy frames),
    // as many threads as fit on the GPU at once: each refines its pixels one
    // after another, so a list that fits in one round costs one pixel's latency
    int rf_per_sm = 1;
    if (L.rf && !cuda_ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rf_per_sm, (const void *)L.rf, kRefineThreads, 0),
                         "cudaOccupancyMaxActiveBlocksPerMultiprocessor(refine)"))
        return TFN_ERR_CUDA;
    L.rf_grid = std::max(1, rf_per_sm) * num_sms;
    L.d_refine = d_refine;
    LaunchArgs &a = L.args;
    a.frames = d_frames;
    a.maps = d_maps;
    a.status = d_status;
    a.rcount = (unsigned long long *)d_refine;
    a.rlist = (unsigned long long *)((char *)d_refine + 128);
    a.rcap = refine_cap;
    a.nframes = nframes;
    a.total_tiles = total_tiles;
    a.out_fmt = m.output;
    a.flags = m.flags;
    for (int k = 0; k < 5; ++k) a.w[k] = m.grad == GRAD_WEIGHTED && k < 3 ? m.weights[k] : 0.f;
    if (grad_is_sep5(m.grad)) sep5_weights(m.grad, m.weights, a.w);
    a.pad[0] = a.pad[1] = 0;
    return TFN_OK;
}

// Enqueues a launch made by make_launch.
tfn_status enqueue_launch(LaunchSpec &L, cudaStream_t stream)
{
    if (L.grid < 1) return TFN_OK;
    void *params[] = {&L.args};
    if (!cuda_ok(cudaLaunchKernel((const void *)L.fn, dim3(L.grid), dim3(L.threads), params, L.smem, stream),
                 "cudaLaunchKernel"))
        return TFN_ERR_CUDA;
    if (!L.rf) return TFN_OK;
    // the refinement kernel as a programmatic dependent launch: scheduled
    // while normals_kernel's last blocks run, it waits on the device for that
    // grid's completion (griddepcontrol.wait) instead of starting after it
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(L.rf_grid);
    lc.blockDim = dim3(kRefineThreads);
    lc.dynamicSmemBytes = 0;
    lc.stream = stream;
    lc.attrs = attr;
    lc.numAttrs = 1;
    if (!cuda_ok(cudaLaunchKernelExC(&lc, (const void *)L.rf, params), "cudaLaunchKernelEx(refine)")) {
        cudaMemsetAsync(L.d_refine, 0, 128, stream);  // (what the refinement kernel would have zeroed)
        return TFN_ERR_CUDA;
    }
    return TFN_OK;
}

tfn_status launch_normals(int kind, const tfn_method &m, int cfg, bool noref, const FrameDesc *d_frames,
                          const CUtensorMap *d_maps, uint32_t *d_status, void *d_refine, int refine_cap, int nframes,
                          int total_tiles, int num_sms, cudaStream_t stream)
{
    LaunchSpec L;
    tfn_status st = make_launch(kind, m, cfg, noref, d_frames, d_maps, d_status, d_refine, refine_cap, nframes,
                                total_tiles, num_sms, &L);
    if (st) return st;
    return enqueue_launch(L, stream);
}

}  // namespace tfn

namespace {

void append_key(std::vector<unsigned char> &k, const void *p, size_t n)
{
    const unsigned char *b = (const unsigned char *)p;
    k.insert(k.end(), b, b + n);
}

void frame_key(std::vector<unsigned char> &k, const tfn_frame &f)
{
    append_key(k, &f.input, sizeof f.input);
    append_key(k, &f.input_pitch, sizeof f.input_pitch);
    append_key(k, &f.height, sizeof f.height);
    append_key(k, &f.width, sizeof f.width);
    append_key(k, &f.input_type, sizeof f.input_type);
    append_key(k, &f.disp_scale, sizeof f.disp_scale);
    append_key(k, &f.cam, sizeof f.cam);
    append_key(k, &f.normals, sizeof f.normals);
    append_key(k, &f.normals_pitch, sizeof f.normals_pitch);
    append_key(k, &f.normals_plane_stride, sizeof f.normals_plane_stride);
    append_key(k, &f.mask, sizeof f.mask);
    append_key(k, &f.mask_pitch, sizeof f.mask_pitch);
    append_key(k, &f.points, sizeof f.points);
    append_key(k, &f.points_pitch, sizeof f.points_pitch);
    append_key(k, &f.points_plane_stride, sizeof f.points_plane_stride);
}

}  // namespace

namespace tfn {

// A slot: cap frame descriptors, cap tensor maps (128-byte aligned), then the
// launch's refinement list (128-byte aligned).
size_t slot_bytes(int cap)
{
    return (size_t)cap * sizeof(FrameDesc) + 128 + (size_t)cap * sizeof(CUtensorMap) + 128 + kRefineListBytes;
}

FrameDesc *slot_descs(void *base) { return (FrameDesc *)base; }
CUtensorMap *slot_maps(void *base, int cap)
{
    uintptr_t p = (uintptr_t)base + (size_t)cap * sizeof(FrameDesc);
    return (CUtensorMap *)((p + 127) & ~(uintptr_t)127);
}
void *slot_refine(void *base, int cap)
{
    uintptr_t p = (uintptr_t)(slot_maps(base, cap) + cap);
    return (void *)((p + 127) & ~(uintptr_t)127);
}

}  // namespace tfn

namespace {

tfn_status slot_reserve(tfn_ctx *c, Slot &s, int n)
{
    if (s.cap >= n) return TFN_OK;
    if (s.done) TFN_CUDA(cudaEventSynchronize(s.done));
    int cap = std::max(n, std::max(8, s.cap * 2));
    ctx_free(c, s.dev, s.bytes);
    if (s.host) cudaFreeHost(s.host);
    s.host = nullptr;
    s.cap = 0;
    s.has_key = false;
    size_t bytes = slot_bytes(cap);
    tfn_status st = ctx_alloc(c, &s.dev, bytes);
    if (st) return st;
    if (!cuda_ok(cudaMemset(slot_refine(s.dev, cap), 0, 128), "cudaMemset(refinement list)")) {
        ctx_free(c, s.dev, bytes);
        return TFN_ERR_CUDA;
    }
    if (!cuda_ok(cudaMallocHost(&s.host, bytes), "cudaMallocHost")) {
        ctx_free(c, s.dev, bytes);
        return TFN_ERR_CUDA;
    }
    s.bytes = bytes;
    s.cap = cap;
    return TFN_OK;
}



// One launch over frames[0..n) (all of one input kind).
tfn_status launch_group(tfn_ctx *c, const tfn_frame *frames, int n, const tfn_method &m, cudaStream_t stream,
                        uint32_t *status)
{
    const int kind = frames[0].input_type;
    const int cfg = choose_cfg(c, frames, n, m);
    std::vector<unsigned char> key;
    key.reserve(16 + (size_t)n * 96);
    append_key(key, &m, sizeof m);
    append_key(key, &cfg, sizeof cfg);
    for (int i = 0; i < n; ++i) frame_key(key, frames[i]);

    int si = -1;
    if (c->last_slot >= 0 && c->slots[c->last_slot].has_key && c->slots[c->last_slot].key == key) si = c->last_slot;
    int total = 0;
    for (int i = 0; i < n; ++i) total += frame_tiles(frames[i], cfg);
    if (si < 0) {
        si = c->next_slot;
        c->next_slot = (c->next_slot + 1) % kSlots;
        Slot &s = c->slots[si];
        if (s.done) TFN_CUDA(cudaEventSynchronize(s.done));  // the previous launch from this slot is finished
        tfn_status st = slot_reserve(c, s, n);
        if (st) return st;
        FrameDesc *d = slot_descs(s.host);
        CUtensorMap *maps = slot_maps(s.host, s.cap);
        int tb = 0;
        for (int i = 0; i < n; ++i) {
            const tfn_frame &f = frames[i];
            d[i] = describe_frame(f, cfg, m, tb);
            tb += frame_tiles(f, cfg);
            st = encode_map(&maps[i], f, cfg);
            if (st) return st;
        }
        const size_t off_maps = (uintptr_t)slot_maps(s.host, s.cap) - (uintptr_t)s.host;
        TFN_CUDA(cudaMemcpyAsync(s.dev, s.host, (size_t)n * sizeof(FrameDesc), cudaMemcpyHostToDevice, stream));
        TFN_CUDA(cudaMemcpyAsync((char *)s.dev + off_maps, (char *)s.host + off_maps, (size_t)n * sizeof(CUtensorMap),
                                 cudaMemcpyHostToDevice, stream));
        s.key.swap(key);
        s.has_key = true;
    }
    Slot &s = c->slots[si];
    c->last_slot = si;
    if (!s.done) TFN_CUDA(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));

    tfn_status lst = launch_normals(kind, m, cfg, refinement_idle(frames, n, m), slot_descs(s.dev), slot_maps(s.dev, s.cap),
                                    status ? status : c->status, slot_refine(s.dev, s.cap), kRefineCap, n, total,
                                    c->num_sms, stream);
    if (lst) return lst;
    TFN_CUDA(cudaEventRecord(s.done, stream));
    return TFN_OK;
}

}  // namespace

namespace tfn {

tfn_status run_batch(tfn_ctx *c, const tfn_frame *frames, int n, const tfn_method &m, cudaStream_t stream,
                     uint32_t *status)
{
    // frames of one input kind go to one launch; keep the caller's order
    int i = 0;
    while (i < n) {
        int j = i + 1;
        while (j < n && frames[j].input_type == frames[i].input_type) ++j;
        tfn_status st = launch_group(c, frames + i, j - i, m, stream, status);
        if (st) return st;
        i = j;
    }
    return TFN_OK;
}

}  // namespace tfn

namespace {

// Queues the copies of one direction on one stream, merging a copy into the
// previous one when both of its ends start exactly where the previous one's
// full extent ends.  A batch of same-size frames laid out back to back on
// both sides then costs one large copy per direction and chunk instead of one
// per frame and plane, which is what bounds the host path otherwise (each
// call costs microseconds of CPU).  The padding after the last row of the
// last merged copy is left out, so no copy reads or writes past a buffer.
// When the destination is the caller's memory (`exact_rows`), only rows
// without padding merge: a pitched view's padding may belong to other data.
struct CopyQueue {
    cudaMemcpyKind kind;
    cudaStream_t stream;
    bool exact_rows;
    char *dst = nullptr;
    const char *src = nullptr;
    size_t extent = 0, trim = 0;
    bool ok = true;

    CopyQueue(cudaMemcpyKind k, cudaStream_t s, bool exact) : kind(k), stream(s), exact_rows(exact) {}

    // rows x width bytes, at dpitch / spitch bytes per row
    void add(void *d, size_t dpitch, const void *sp, size_t spitch, size_t width, size_t rows)
    {
        if (!ok || rows == 0 || width == 0) return;
        if (dpitch != spitch || (exact_rows && dpitch != width)) {  // a 2D copy of its own
            flush();
            ok = cuda_ok(cudaMemcpy2DAsync(d, dpitch, sp, spitch, width, rows, kind, stream), "cudaMemcpy2DAsync");
            return;
        }
        const size_t ext = dpitch * rows;
        if (extent && (char *)d == dst + extent && (const char *)sp == src + extent) {
            extent += ext;
        } else {
            flush();
            dst = (char *)d;
            src = (const char *)sp;
            extent = ext;
        }
        trim = dpitch - width;
    }
    void flush()
    {
        if (extent && ok) ok = cuda_ok(cudaMemcpyAsync(dst, src, extent - trim, kind, stream), "cudaMemcpyAsync");
        extent = 0;
    }
};

}  // namespace

extern "C" {

const char *tfn_status_string(tfn_status s)
{
    switch (s) {
    case TFN_OK: return "ok";
    case TFN_ERR_INVALID_ARG: return "invalid argument";
    case TFN_ERR_UNSUPPORTED: return "unsupported combination";
    case TFN_ERR_MISALIGNED: return "pointer or pitch not a multiple of 16 bytes";
    case TFN_ERR_OUT_OF_MEMORY: return "out of memory (context budget or device)";
    case TFN_ERR_CUDA: return "CUDA error";
    case TFN_ERR_TIMEOUT: return "timed out";
    case TFN_ERR_CANCELLED: return "cancelled";
    case TFN_ERR_BUSY: return "busy";
    case TFN_ERR_DEVICE: return "a kernel reported a failed bounded wait";
    case TFN_ERR_IO: return "file could not be opened, read or written";
    }
    return "unknown status";
}

const char *tfn_version(void) { return "tfn 0.1 (sm_103a)"; }

const char *tfn_last_cuda_error(void) { return g_cuda_err; }

tfn_status tfn_create(tfn_ctx **out, int device, size_t budget)
{
    if (!out) return TFN_ERR_INVALID_ARG;
    *out = nullptr;
    if (device < 0 && !cuda_ok(cudaGetDevice(&device), "cudaGetDevice")) return TFN_ERR_CUDA;
    int ndev = 0;
    if (!cuda_ok(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount")) return TFN_ERR_CUDA;
    if (device >= ndev) return TFN_ERR_INVALID_ARG;
    DeviceGuard g(device);
    if (!g.ok) return TFN_ERR_CUDA;
    tfn_ctx *c = new (std::nothrow) tfn_ctx();
    if (!c) return TFN_ERR_OUT_OF_MEMORY;
    c->device = device;
    c->budget = budget;
    if (!cuda_ok(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device), "cudaDeviceGetAttribute")) {
        delete c;
        return TFN_ERR_CUDA;
    }
    tfn_status st = ctx_alloc(c, (void **)&c->status, 256);
    if (st || !cuda_ok(cudaMemset(c->status, 0, 256), "cudaMemset") ||
        !cuda_ok(cudaMallocHost((void **)&c->status_host, sizeof(uint32_t)), "cudaMallocHost")) {
        tfn_destroy(c);
        return st ? st : TFN_ERR_CUDA;
    }
    *out = c;
    return TFN_OK;
}

tfn_status tfn_destroy(tfn_ctx *c)
{
    if (!c) return TFN_OK;
    DeviceGuard g(c->device);
    for (Slot &s : c->slots) {
        if (s.done) {
            cudaEventSynchronize(s.done);
            cudaEventDestroy(s.done);
        }
        ctx_free(c, s.dev, s.bytes);
        if (s.host) cudaFreeHost(s.host);
    }
    for (Stage &s : c->stages) {
        if (s.stream) {
            cudaStreamSynchronize(s.stream);
            cudaStreamDestroy(s.stream);
        }
        ctx_free(c, s.in, s.in_bytes);
        ctx_free(c, s.out, s.out_bytes);
        ctx_free(c, s.mask, s.mask_bytes);
        ctx_free(c, s.pts, s.pts_bytes);
    }
    void *st = c->status;
    ctx_free(c, st, 256);
    if (c->status_host) cudaFreeHost(c->status_host);
    delete c;
    return TFN_OK;
}

tfn_status tfn_normals(tfn_ctx *c, const tfn_frame *frame, const tfn_method *m, tfn_stream stream)
{
    return tfn_normals_batch(c, frame, 1, m, stream);
}

tfn_status tfn_normals_batch(tfn_ctx *c, const tfn_frame *frames, int n, const tfn_method *m, tfn_stream stream)
{
    if (!c || n < 0 || (n > 0 && !frames)) return TFN_ERR_INVALID_ARG;
    tfn_status st = validate_method(m);
    if (st) return st;
    for (int i = 0; i < n; ++i)
        if ((st = validate_frame(&frames[i], m->output))) return st;
    if (n == 0) return TFN_OK;
    DeviceGuard g(c->device);
    if (!g.ok) return TFN_ERR_CUDA;
    return run_batch(c, frames, n, *m, (cudaStream_t)stream);
}

tfn_status tfn_normals_batch_host(tfn_ctx *c, const tfn_frame *frames, int n, const tfn_method *m, tfn_stream stream)
{
    if (!c || n < 0 || (n > 0 && !frames)) return TFN_ERR_INVALID_ARG;
    tfn_status st = validate_method(m);
    if (st) return st;
    for (int i = 0; i < n; ++i) {
        const tfn_frame &f = frames[i];
        if (!f.input || !f.normals || !f.mask || f.height < 1 || f.width < 1 || f.height > 32768 || f.width > 32768 ||
            f.input_type < 0 || f.input_type >= KIND_COUNT)
            return TFN_ERR_INVALID_ARG;
        if (f.points && (f.points_pitch < (int64_t)f.width * 4 || f.points_plane_stride < f.points_pitch * f.height))
            return TFN_ERR_INVALID_ARG;
    }
    if (n == 0) return TFN_OK;
    DeviceGuard g(c->device);
    if (!g.ok) return TFN_ERR_CUDA;
    const int fmt = m->output;
    const bool planar = fmt <= OUT_BF16;
    const int ob = out_elem_bytes(fmt);
    // Device rows use the host's pitch when it suits the kernel (a multiple of
    // 16 bytes), so that host and device layouts match and copies merge.
    auto dev_pitch = [](int64_t host_pitch, size_t row_bytes) -> size_t {
        const size_t a = (row_bytes + 15) & ~(size_t)15;
        return (host_pitch > 0 && (host_pitch & 15) == 0 && (size_t)host_pitch >= a && (size_t)host_pitch <= 4 * a)
                   ? (size_t)host_pitch
                   : a;
    };
    size_t max_in = 0, max_out = 0, max_mask = 0, max_pts = 0;
    for (int i = 0; i < n; ++i) {
        const tfn_frame &f = frames[i];
        const size_t ip = dev_pitch(f.input_pitch, (size_t)f.width * kind_elem_size(f.input_type));
        const size_t op = dev_pitch(f.normals_pitch, (size_t)f.width * ob);
        const size_t mp = dev_pitch(f.mask_pitch, (size_t)f.width);
        max_in = std::max(max_in, ip * f.height);
        max_out = std::max(max_out, op * f.height * (planar ? 3 : 1));
        max_mask = std::max(max_mask, mp * f.height);
        if (f.points) max_pts = std::max(max_pts, dev_pitch(f.points_pitch, (size_t)f.width * 4) * f.height * 3);
    }
    // Chunks of about 1/16 of the batch's input (8 to 64 MB, at least one frame): the first
    // chunk's upload and kernel run before any download can start, so smaller chunks start the
    // downloads (the larger direction) sooner; the three stages keep both directions busy after.
    const size_t chunk_bytes = std::min<size_t>(64u << 20, std::max<size_t>(8u << 20, max_in * (size_t)n / 16));
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)n, chunk_bytes / std::max<size_t>(max_in, 1)));
    const int nst = 3;
    for (int k = 0; k < nst; ++k) {
        Stage &s = c->stages[k];
        if (!s.stream) TFN_CUDA(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking));
        const size_t need_in = max_in * chunk, need_out = max_out * chunk, need_mask = max_mask * chunk;
        const size_t need_pts = max_pts * chunk;
        if (s.in_bytes < need_in || s.out_bytes < need_out || s.mask_bytes < need_mask || s.pts_bytes < need_pts) {
            TFN_CUDA(cudaStreamSynchronize(s.stream));
            ctx_free(c, s.in, s.in_bytes);
            ctx_free(c, s.out, s.out_bytes);
            ctx_free(c, s.mask, s.mask_bytes);
            ctx_free(c, s.pts, s.pts_bytes);
            s.in_bytes = s.out_bytes = s.mask_bytes = s.pts_bytes = 0;
            if ((st = ctx_alloc(c, &s.in, need_in)) || (st = ctx_alloc(c, &s.out, need_out)) ||
                (st = ctx_alloc(c, &s.mask, need_mask)) || (need_pts && (st = ctx_alloc(c, &s.pts, need_pts))))
                return st;
            s.in_bytes = need_in;
            s.out_bytes = need_out;
            s.mask_bytes = need_mask;
            s.pts_bytes = need_pts;
            for (Slot &sl : c->slots) sl.has_key = false;  // device pointers changed
        }
    }
    cudaEvent_t start;
    TFN_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    cuda_ok(cudaEventRecord(start, (cudaStream_t)stream), "cudaEventRecord");
    for (int k = 0; k < nst; ++k) cuda_ok(cudaStreamWaitEvent(c->stages[k].stream, start, 0), "cudaStreamWaitEvent");
    cudaEventDestroy(start);
    std::vector<tfn_frame> dframes;
    for (int base = 0, ci = 0; base < n && st == TFN_OK; base += chunk, ++ci) {
        Stage &s = c->stages[ci % nst];
        const int cnt = std::min(chunk, n - base);
        dframes.resize(cnt);
        CopyQueue h2d(cudaMemcpyHostToDevice, s.stream, false);
        for (int i = 0; i < cnt; ++i) {
            const tfn_frame &f = frames[base + i];
            tfn_frame d = f;
            const size_t row_in = (size_t)f.width * kind_elem_size(f.input_type);
            const size_t ip = dev_pitch(f.input_pitch, row_in);
            const size_t op = dev_pitch(f.normals_pitch, (size_t)f.width * ob);
            const size_t mp = dev_pitch(f.mask_pitch, (size_t)f.width);
            d.input = (char *)s.in + max_in * i;
            d.input_pitch = ip;
            d.normals = (char *)s.out + max_out * i;
            d.normals_pitch = op;
            d.normals_plane_stride = op * f.height;
            d.mask = (uint8_t *)s.mask + max_mask * i;
            d.mask_pitch = mp;
            if (f.points) {
                const size_t pp = dev_pitch(f.points_pitch, (size_t)f.width * 4);
                d.points = (char *)s.pts + max_pts * i;
                d.points_pitch = pp;
                d.points_plane_stride = pp * f.height;
            }
            if ((st = validate_frame(&d, fmt))) break;
            h2d.add((void *)d.input, ip, f.input, f.input_pitch, row_in, f.height);
            dframes[i] = d;
        }
        h2d.flush();
        if (!st && !h2d.ok) st = TFN_ERR_CUDA;
        if (st) break;
        if ((st = run_batch(c, dframes.data(), cnt, *m, s.stream))) break;
        CopyQueue d2h(cudaMemcpyDeviceToHost, s.stream, true), d2h_mask(cudaMemcpyDeviceToHost, s.stream, true);
        CopyQueue d2h_pts(cudaMemcpyDeviceToHost, s.stream, true);
        for (int i = 0; i < cnt; ++i) {
            const tfn_frame &f = frames[base + i];
            const tfn_frame &d = dframes[i];
            for (int p = 0; p < (planar ? 3 : 1); ++p)
                d2h.add((char *)f.normals + p * f.normals_plane_stride, f.normals_pitch,
                        (char *)d.normals + p * d.normals_plane_stride, d.normals_pitch, (size_t)f.width * ob,
                        f.height);
            d2h_mask.add(f.mask, f.mask_pitch, d.mask, d.mask_pitch, f.width, f.height);
            if (f.points)
                for (int p = 0; p < 3; ++p)
                    d2h_pts.add((char *)f.points + p * f.points_plane_stride, f.points_pitch,
                                (char *)d.points + p * d.points_plane_stride, d.points_pitch, (size_t)f.width * 4,
                                f.height);
        }
        d2h.flush();
        d2h_mask.flush();
        d2h_pts.flush();
        if (!d2h.ok || !d2h_mask.ok || !d2h_pts.ok) st = TFN_ERR_CUDA;
    }
    for (int k = 0; k < nst; ++k)
        if (!cuda_ok(cudaStreamSynchronize(c->stages[k].stream), "cudaStreamSynchronize") && st == TFN_OK)
            st = TFN_ERR_CUDA;
    return st;
}

tfn_status tfn_plan_create(tfn_ctx *c, const tfn_frame *frames, int n, const tfn_method *m, tfn_plan **out)
{
    if (!out) return TFN_ERR_INVALID_ARG;
    *out = nullptr;
    if (!c || n < 1 || !frames) return TFN_ERR_INVALID_ARG;
    tfn_status st = validate_method(m);
    if (st) return st;
    for (int i = 0; i < n; ++i)
        if ((st = validate_frame(&frames[i], m->output))) return st;
    DeviceGuard g(c->device);
    if (!g.ok) return TFN_ERR_CUDA;
    tfn_plan *p = new (std::nothrow) tfn_plan();
    if (!p) return TFN_ERR_OUT_OF_MEMORY;
    p->ctx = c;
    p->n = n;
    p->bytes = slot_bytes(n);
    if ((st = ctx_alloc(c, &p->dev, p->bytes))) {
        delete p;
        return st;
    }
    std::vector<unsigned char> host(p->bytes + 128);
    void *hbase = (void *)(((uintptr_t)host.data() + 127) & ~(uintptr_t)127);
    FrameDesc *d = slot_descs(hbase);
    CUtensorMap *maps = slot_maps(hbase, n);
    // one launch per run of frames of the same input kind, each with its shape
    std::vector<int> run_cfg(n);
    for (int i = 0; i < n;) {
        int j = i + 1;
        while (j < n && frames[j].input_type == frames[i].input_type) ++j;
        const int cfg = choose_cfg(c, frames + i, j - i, *m);
        for (int k = i; k < j; ++k) run_cfg[k] = cfg;
        i = j;
    }
    for (int i = 0, tb = 0; i < n; ++i) {
        if (i > 0 && frames[i].input_type != frames[i - 1].input_type) tb = 0;
        const int cfg = run_cfg[i];
        d[i] = describe_frame(frames[i], cfg, *m, tb);
        tb += frame_tiles(frames[i], cfg);
        if ((st = encode_map(&maps[i], frames[i], cfg))) break;
    }
    cudaStream_t cs = nullptr;
    if (st == TFN_OK && !cuda_ok(cudaMemcpy(p->dev, hbase, p->bytes, cudaMemcpyHostToDevice), "cudaMemcpy"))
        st = TFN_ERR_CUDA;
    if (st == TFN_OK && !cuda_ok(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cudaStreamCreate"))
        st = TFN_ERR_CUDA;
    // capture one launch per run of frames of the same input kind
    if (st == TFN_OK && cuda_ok(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture")) {
        tfn_status lst = TFN_OK;
        for (int i = 0; i < n && lst == TFN_OK;) {
            int j = i + 1;
            while (j < n && frames[j].input_type == frames[i].input_type) ++j;
            const int cfg = run_cfg[i];
            int total = 0;
            for (int k = i; k < j; ++k) total += frame_tiles(frames[k], cfg);
            lst = launch_normals(frames[i].input_type, *m, cfg, refinement_idle(frames + i, j - i, *m),
                                 slot_descs(p->dev) + i, slot_maps(p->dev, n) + i, c->status, slot_refine(p->dev, n),
                                 kRefineCap, j - i, total, c->num_sms, cs);
            i = j;
        }
        if (!cuda_ok(cudaStreamEndCapture(cs, &p->graph), "cudaStreamEndCapture") && lst == TFN_OK) lst = TFN_ERR_CUDA;
        st = lst;
        if (st == TFN_OK && !cuda_ok(cudaGraphInstantiate(&p->exec, p->graph, 0), "cudaGraphInstantiate"))
            st = TFN_ERR_CUDA;
    } else if (st == TFN_OK) {
        st = TFN_ERR_CUDA;
    }
    if (cs) cudaStreamDestroy(cs);
    if (st) {
        tfn_plan_destroy(p);
        return st;
    }
    *out = p;
    return TFN_OK;
}

tfn_status tfn_plan_launch(tfn_plan *p, tfn_stream stream)
{
    if (!p || !p->exec) return TFN_ERR_INVALID_ARG;
    DeviceGuard g(p->ctx->device);
    if (!g.ok) return TFN_ERR_CUDA;
    TFN_CUDA(cudaGraphLaunch(p->exec, (cudaStream_t)stream));
    return TFN_OK;
}

tfn_status tfn_plan_kernels(const tfn_plan *p, int32_t *count)
{
    if (!p || !p->graph || !count) return TFN_ERR_INVALID_ARG;
    size_t nn = 0;
    TFN_CUDA(cudaGraphGetNodes(p->graph, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) TFN_CUDA(cudaGraphGetNodes(p->graph, nodes.data(), &nn));
    int32_t k = 0;
    for (size_t i = 0; i < nn; ++i) {
        cudaGraphNodeType t;
        TFN_CUDA(cudaGraphNodeGetType(nodes[i], &t));
        k += t == cudaGraphNodeTypeKernel;
    }
    *count = k;
    return TFN_OK;
}

tfn_status tfn_plan_kernel_name(const tfn_plan *p, int32_t index, const char **name)
{
    if (!p || !p->graph || !name || index < 0) return TFN_ERR_INVALID_ARG;
    size_t nn = 0;
    TFN_CUDA(cudaGraphGetNodes(p->graph, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) TFN_CUDA(cudaGraphGetNodes(p->graph, nodes.data(), &nn));
    int32_t k = 0;
    for (size_t i = 0; i < nn; ++i) {
        cudaGraphNodeType t;
        TFN_CUDA(cudaGraphNodeGetType(nodes[i], &t));
        if (t != cudaGraphNodeTypeKernel) continue;
        if (k++ != index) continue;
        cudaKernelNodeParams kp;
        TFN_CUDA(cudaGraphKernelNodeGetParams(nodes[i], &kp));
        const char *nm = nullptr;
        TFN_CUDA(cudaFuncGetName(&nm, kp.func));
        if (!nm) return TFN_ERR_CUDA;
        *name = nm;
        return TFN_OK;
    }
    return TFN_ERR_INVALID_ARG;
}

tfn_status tfn_plan_destroy(tfn_plan *p)
{
    if (!p) return TFN_OK;
    DeviceGuard g(p->ctx->device);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->dev) {
        cudaDeviceSynchronize();  // a replay may still read the descriptors
        ctx_free(p->ctx, p->dev, p->bytes);
    }
    delete p;
    return TFN_OK;
}

int tfn_tile_shape_count(void) { return kNumCfg; }

tfn_status tfn_tile_shape_info(int index, int *tile_w, int *tile_h, int *rows_per_thread)
{
    if (index < 0 || index >= kNumCfg) return TFN_ERR_INVALID_ARG;
    if (tile_w) *tile_w = kCfgs[index].tw;
    if (tile_h) *tile_h = kCfgs[index].th;
    if (rows_per_thread) *rows_per_thread = kCfgs[index].pr;
    return TFN_OK;
}

tfn_status tfn_tile_shape_warps(int index, int *warps_3x3, int *warps_other)
{
    if (index < 0 || index >= kNumCfg) return TFN_ERR_INVALID_ARG;
    if (warps_3x3) *warps_3x3 = kCfgs[index].warps3;
    if (warps_other) *warps_other = kCfgs[index].warps5;
    return TFN_OK;
}

tfn_status tfn_set_tile_shape(tfn_ctx *c, int index)
{
    if (!c || index < -1 || index >= kNumCfg) return TFN_ERR_INVALID_ARG;
    c->forced_cfg = index;
    c->last_slot = -1;  // descriptors depend on the tile shape
    return TFN_OK;
}

tfn_status tfn_refined_pixels(tfn_ctx *c, uint64_t *count, tfn_stream stream)
{
    if (!c || !count) return TFN_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok) return TFN_ERR_CUDA;
    TFN_CUDA(cudaMemcpyAsync(c->status_host, c->status + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                             (cudaStream_t)stream));
    TFN_CUDA(cudaMemsetAsync(c->status + 1, 0, sizeof(uint32_t), (cudaStream_t)stream));
    TFN_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    *count = *c->status_host;
    return TFN_OK;
}

tfn_status tfn_device_status(tfn_ctx *c, uint32_t *bits, tfn_stream stream)
{
    if (!c || !bits) return TFN_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok) return TFN_ERR_CUDA;
    TFN_CUDA(cudaMemcpyAsync(c->status_host, c->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    TFN_CUDA(cudaMemsetAsync(c->status, 0, sizeof(uint32_t), (cudaStream_t)stream));
    TFN_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    *bits = *c->status_host;
    return TFN_OK;
}

}  // extern "C"
