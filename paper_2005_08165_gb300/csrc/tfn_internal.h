// tfn_internal.h -- types shared by the host side (tfn_api.cu) and the kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tfn {

enum Kind { KIND_DEPTH_F32 = 0, KIND_DEPTH_F16 = 1, KIND_DISP_U16 = 2, KIND_DISP_F32 = 3, KIND_COUNT = 4 };
// GRAD_FD5 .. GRAD_PREWITT5 are GRAD_SEP5 with fixed weights (sep5_weights);
// GRAD_PLANEPCA stands for the PlanePCA estimator (tfn_method.estimator), a
// kernel with no gradient filter and no Phi.  The kernels are compiled for
// GRAD_FD .. GRAD_SEP5 and GRAD_PLANEPCA (with PHI_MEAN).
enum Grad {
    GRAD_FD = 0,
    GRAD_SOBEL = 1,
    GRAD_SCHARR = 2,
    GRAD_PREWITT = 3,
    GRAD_WEIGHTED = 4,
    GRAD_SEP5 = 5,
    GRAD_FD5 = 6,
    GRAD_SOBEL5 = 7,
    GRAD_PREWITT5 = 8,
    GRAD_PLANEPCA = 9,
    GRAD_COUNT = 10
};
enum Phi { PHI_MEAN = 0, PHI_MEDIAN = 1, PHI_COUNT = 2 };
enum OutFmt { OUT_F32 = 0, OUT_F16 = 1, OUT_BF16 = 2, OUT_F16X4 = 3, OUT_BF16X4 = 4, OUT_OCT16 = 5 };

// The FD gradients of the mean on depth: compensated quotients (false), or
// one-pass quotients within 5u whose error the mean's bound carries (true).
// The one-pass form saves arithmetic and flags about three times as many
// pixels for the double-float pass on noisy frames.
constexpr bool kFdOnePassMean = true;

// Device status bits written by kernels.
enum : uint32_t { DEVERR_TMA_WAIT = 1u };

// Per-frame descriptor in device memory (one per frame of a launch).
struct alignas(16) FrameDesc {
    char *out;           // normals: plane c at out + c * out_plane
    int64_t out_pitch;   // bytes
    int64_t out_plane;   // bytes
    uint8_t *mask;
    int64_t mask_pitch;  // bytes
    const void *in;      // the input image (read again only for the rare refined pixels)
    int64_t in_pitch;    // bytes
    int32_t H, W;
    int32_t tiles_x;     // work items per row band of this frame
    int32_t tile_begin;  // global index of this frame's first work item
    float fx, fy, u0, v0;
    float thr;           // refinement threshold (see refine_threshold in tfn_api.cu)
    int32_t kind;        // Kind of this frame (a launch holds frames of one kind)
    char *pts;           // optional point cloud: plane c at pts + c * pts_plane (nullptr: none)
    int64_t pts_pitch;   // bytes
    int64_t pts_plane;   // bytes
    float ztc;           // disparity input: Z = ztc / raw sample (f t_c / disp_scale)
    int32_t pad;
};
static_assert(sizeof(FrameDesc) == 128, "FrameDesc layout");

// Kernel arguments (passed by value as a __grid_constant__).
struct LaunchArgs {
    const FrameDesc *frames;
    const CUtensorMap *maps;  // one 2D tiled map per frame, 64-byte aligned
    uint32_t *status;         // [0]: DEVERR_* bits, [1]: refined-pixel count
    unsigned long long *rlist;   // pixels to refine: frame index << 32 | y << 16 | x
    unsigned long long *rcount;  // entries appended (may exceed rcap); then the refinement kernel's block counter
    int32_t rcap;                // capacity of rlist
    int32_t nframes;
    int32_t total_tiles;
    int32_t out_fmt;
    int32_t flags;
    float w[5];               // GRAD_WEIGHTED: row weights (w0 w1 w2); GRAD_SEP5: (d1 d2 s0 s1 s2)
    int32_t pad[2];
};

// The refinement list of one launch: a 128-byte header (the entry count,
// then the refinement kernel's finished-block counter; both zero between
// launches: zeroed at allocation, and again by the refinement kernel's last
// block), then its entries.  Every launch owns one: context slots and plans
// hold kRefineCap entries (2 MB, about 3 per thousand pixels of a 256-frame
// 480x640 batch), the allocation-free scratch kNoallocRefineCap.  A launch
// that flags more pixels than its list holds still refines them all (the
// refinement kernel then scans the masks).
constexpr int kRefineCap = 262144;
constexpr int kNoallocRefineCap = 65536;
constexpr size_t refine_list_bytes(int cap) { return 128 + (size_t)cap * 8; }
constexpr size_t kRefineListBytes = refine_list_bytes(kRefineCap);
constexpr int kRefineThreads = 128;

// Work-item shapes the kernels are compiled for.  An item is a band of tw =
// 128 pixel columns (32 lanes x 4) by th rows of one frame, computed by one
// warp that rolls down its rows (pr = th rows per lane); the rows stream
// through a ring of nst shared-memory stages of cr rows each (th + 2 rows per
// item: one above, one below; th + 4 for the 5x5 filters, the last chunk of
// an item then partly unused), per warp; a CTA has `warps3` warps for the
// 3x3 filters and `warps5` for the 5x5 filters and PlanePCA.  Shapes 4 and 5 repeat the heights of shapes 1 and 2
// with other CTA widths, so that the autotuner chooses the threads per CTA
// as well as the item height.
struct TileCfg {
    int tw, th, pr, cr, nst, warps5, warps3;
};
constexpr int kNumCfg = 6;
constexpr TileCfg kCfgs[kNumCfg] = {{128, 18, 18, 5, 3, 4, 2}, {128, 30, 30, 8, 3, 4, 2}, {128, 12, 12, 7, 3, 4, 2},
                                    {128, 6, 6, 4, 2, 4, 2},   {128, 30, 30, 8, 3, 2, 4}, {128, 12, 12, 7, 3, 2, 1}};
// the default shape for launches with few items (short items spread one frame over many warps)
constexpr int kSmallCfg = 3;
// Whether the (shape) kernel refines its flagged pixels itself, at the end of
// each item, rather than listing them for the refinement kernel: the
// short-item shape of small launches, where a second launch would cost more
// than the refinement.
constexpr bool refines_in_place(int c) { return c == kSmallCfg; }
// Whether the (shape, filter, Phi) kernel refines its flagged pixels itself
// through a per-warp queue, 32 pixels at a time, rather than listing them for
// the refinement kernel: the FD mean in the other shapes.  Its flagged pixels
// are rare (about 2 per 128 x 30 item on noisy frames), so a warp drains its
// queue about once in a launch, where a second kernel costs a launch, its
// latency-bound reads and its fixed time (256 x 480x640 frames: 0.341 ->
// 0.334 ms a pass).  The FD median flags almost nothing and keeps the list
// (its refinement kernel finds it empty); the smoothed 3x3 filters and the
// 5x5 ones keep it too, as their shared memory already holds as many CTAs per
// SM as it can.
constexpr bool refines_by_queue(int c, int grad, int phi)
{
    return c != kSmallCfg && grad == GRAD_FD && phi == PHI_MEAN;
}
constexpr bool refines_in_kernel(int c, int grad, int phi) { return refines_in_place(c) || refines_by_queue(c, grad, phi); }
// the default shape otherwise: the tallest items (the least halo per row) measured fastest for every
// filter on 256 x 480x640 frames (FD mean 0.9%, Sobel 4.5%, the 5x5 filters 13% faster than 18 rows)
constexpr int kDefaultCfg = 1;

// The 3x3 filters (FD, Sobel, Scharr, Prewitt, the weighted family) run the
// pixel-pair row step (row_step2) with the row carry in shared memory; the
// 5x5 filters and PlanePCA run the scalar one.
constexpr bool grad_is_pair(int grad) { return grad >= GRAD_FD && grad <= GRAD_WEIGHTED; }
// Warps per CTA of the (shape, filter) kernel.  The 3x3 kernels (128
// registers) run 2-warp CTAs in the default shapes, 8 of them per SM, whose
// finer grain scheduled better than 4 x 4 warps (`warps3`); the 5x5 filters
// and PlanePCA 4-warp CTAs (`warps5`).
constexpr int cta_warps(int c, int grad) { return grad_is_pair(grad) ? kCfgs[c].warps3 : kCfgs[c].warps5; }
// CTAs per SM that the 3x3 kernels are compiled for (their register bound).
constexpr int ctas3_per_sm(int c) { return 16 / cta_warps(c, GRAD_FD); }
inline int cfg_threads(int c, int grad) { return 32 * cta_warps(c, grad); }
inline int kind_elem_size(int kind) { return (kind == KIND_DEPTH_F32 || kind == KIND_DISP_F32) ? 4 : 2; }
// Halo columns loaded on each side so that the TMA box starts on a 16-byte boundary.
inline int kind_padx(int kind) { return 16 / kind_elem_size(kind); }
inline int box_w(int kind, int c) { return kCfgs[c].tw + 2 * kind_padx(kind); }
inline int box_h(int c) { return kCfgs[c].cr; }
inline size_t stage_bytes(int kind, int c) { return (size_t)box_w(kind, c) * box_h(c) * kind_elem_size(kind); }
inline size_t stage_stride(int kind, int c) { return (stage_bytes(kind, c) + 127) & ~(size_t)127; }
// GRAD_SEP5 keeps each lane's row derivatives and smoothings of the last 5
// sample rows in shared memory: 5 rows x 4 float4 per lane.
constexpr size_t kSep5RingBytes = 5 * 4 * 32 * 16;
constexpr bool grad_is_sep5(int grad) { return grad >= GRAD_SEP5 && grad <= GRAD_PREWITT5; }
// Stages of a warp's TMA ring.  The 5x5 filters keep 2: with their 10 KB
// derivative ring a third stage makes shared memory the occupancy limit
// (2 CTAs = 8 warps per SM instead of the 12 their registers allow), and a
// chunk of 8 rows takes far longer to compute than one copy takes to land.
// The 3x3 kernels keep 2 as well: with their carry buffer (below) 3 stages
// would make shared memory the occupancy limit.
constexpr int cfg_nst(int c, int grad)
{
    return (grad_is_sep5(grad) || grad_is_pair(grad)) && kCfgs[c].nst > 2 ? 2 : kCfgs[c].nst;
}
// The 3x3 kernels keep each lane's carry from one row to the next (the rho of
// the up, up-left and up-right neighbours and their count, 8 floats per
// pixel pair) in shared memory rather than in registers: 2 pairs x 2 x 16
// bytes per lane.
constexpr size_t kCarry3Bytes = 2 * 2 * 32 * 16;
// The smoothed 3x3 filters also keep each sample row's horizontal tap
// differences (w[c+1] - w[c-1] as h + l at the lane's 4 columns) for the three
// output rows that use them: a ring of 3 rows x 2 pairs x 16 bytes per lane.
constexpr size_t kDRingBytes = 3 * 2 * 32 * 16;
// Shared memory per warp for the row carry (and the ring) of the 3x3 kernels.
constexpr size_t carry_bytes(int grad)
{
    return grad_is_pair(grad) ? kCarry3Bytes + (grad != GRAD_FD ? kDRingBytes : 0) : 0;
}
inline size_t smem_bytes(int kind, int c, int grad)
{
    return (size_t)cta_warps(c, grad) * (cfg_nst(c, grad) * stage_stride(kind, c) + (grad_is_sep5(grad) ? kSep5RingBytes : 0) +
                                         carry_bytes(grad)) +
           128;
}
// The profiles (d1 d2 s0 s1 s2) of a 5x5 filter: the named members' fixed
// ones, else the caller's.
inline void sep5_weights(int grad, const float *given, float w[5])
{
    static const float fd5[5] = {8.f, -1.f, 1.f, 0.f, 0.f}, sobel5[5] = {2.f, 1.f, 6.f, 4.f, 1.f},
                       prewitt5[5] = {1.f, 2.f, 1.f, 1.f, 1.f};
    const float *src = grad == GRAD_FD5 ? fd5 : grad == GRAD_SOBEL5 ? sobel5 : grad == GRAD_PREWITT5 ? prewitt5 : given;
    for (int k = 0; k < 5; ++k) w[k] = src[k];
}

// Kernel entry points, one per (kind, grad, phi, cfg), and the NOREF forms
// (noref: FP16 depth with FD only, else nullptr); defined in tfn_k_*.cu.
typedef void (*KernelFn)(LaunchArgs);
KernelFn kernel_for(int kind, int grad, int phi, int cfg, bool noref = false);
// The refinement kernel of (kind, grad, phi); nullptr for PlanePCA.
KernelFn refiner_for(int kind, int grad, int phi);

}  // namespace tfn

#include "../../include/tfn.h"

namespace tfn {

// The kernel a method runs: its filter (GRAD_PLANEPCA for the PlanePCA
// estimator) and Phi (PHI_MEAN for PlanePCA).
inline int method_grad(const tfn_method &m) { return m.estimator == TFN_EST_PLANEPCA ? (int)GRAD_PLANEPCA : m.grad; }
inline int method_phi(const tfn_method &m) { return m.estimator == TFN_EST_PLANEPCA ? (int)PHI_MEAN : m.phi; }

// Host helpers shared by the entry points (tfn_api.cu).
bool cuda_ok(cudaError_t e, const char *what);
tfn_status validate_method(const tfn_method *m);
tfn_status validate_frame(const tfn_frame *f, int out_fmt);
float refine_threshold(const tfn_frame &f, int grad, int phi);
tfn_status encode_map(CUtensorMap *map, const tfn_frame &f, int cfg);
FrameDesc describe_frame(const tfn_frame &f, int cfg, const tfn_method &m, int tile_begin);
int frame_tiles(const tfn_frame &f, int cfg);
// One launch of the kernel for frames of one input kind, and of the
// refinement kernel after it (rf, or none).
struct LaunchSpec {
    KernelFn fn = nullptr, rf = nullptr;
    int grid = 0, threads = 0, rf_grid = 0;
    size_t smem = 0;
    void *d_refine = nullptr;
    LaunchArgs args;
};
// d_refine: the launch's refinement list (refine_list_bytes(refine_cap), 128-byte aligned).
// noref: run the NOREF kernel (refinement_idle holds for the launch's frames).
tfn_status make_launch(int kind, const tfn_method &m, int cfg, bool noref, const FrameDesc *d_frames,
                       const CUtensorMap *d_maps, uint32_t *d_status, void *d_refine, int refine_cap, int nframes,
                       int total_tiles, int num_sms, LaunchSpec *spec);
tfn_status enqueue_launch(LaunchSpec &spec, cudaStream_t stream);
tfn_status launch_normals(int kind, const tfn_method &m, int cfg, bool noref, const FrameDesc *d_frames,
                          const CUtensorMap *d_maps, uint32_t *d_status, void *d_refine, int refine_cap, int nframes,
                          int total_tiles, int num_sms, cudaStream_t stream);
// Whether the FP16 depth frames' sample spacing proves that no pixel can be
// flagged for refinement (FD filter only; see its definition).
bool refinement_idle(const tfn_frame *frames, int n, const tfn_method &m);

}  // namespace tfn
