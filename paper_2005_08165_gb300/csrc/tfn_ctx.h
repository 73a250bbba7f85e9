// tfn_ctx.h -- the context and plan objects behind the opaque handles of the
// C ABI, shared by the host-side translation units (tfn_api.cu, tfn_tune.cu,
// tfn_server.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include "tfn_internal.h"

namespace tfn {

constexpr int kSlots = 4;
constexpr int kOutCount = OUT_BF16X4 + 1;

// One scratch slot: descriptors + tensor maps for one launch.
struct Slot {
    void *dev = nullptr;   // FrameDesc[cap] then CUtensorMap[cap]
    void *host = nullptr;  // pinned mirror
    int cap = 0;
    size_t bytes = 0;
    cudaEvent_t done = nullptr;  // recorded after the launch that used it
    std::vector<unsigned char> key;
    bool has_key = false;
};

// Staging of the host-buffer path: one set per pipeline stream.
struct Stage {
    cudaStream_t stream = nullptr;
    void *in = nullptr, *out = nullptr, *mask = nullptr, *pts = nullptr;
    size_t in_bytes = 0, out_bytes = 0, mask_bytes = 0, pts_bytes = 0;
};

}  // namespace tfn

struct tfn_ctx {
    int device = 0;
    int num_sms = 0;
    size_t budget = 0, used = 0;
    uint32_t *status = nullptr;
    uint32_t *status_host = nullptr;
    tfn::Slot slots[tfn::kSlots];
    int next_slot = 0, last_slot = -1;
    // tile shape: forced >= 0 (tfn_set_tile_shape), else the tune table's
    // entry for (input kind, gradient, phi, output), else kDefaultCfg (or
    // kSmallCfg for a small launch)
    int forced_cfg = -1;
    signed char tuned[tfn::KIND_COUNT][tfn::GRAD_COUNT][tfn::PHI_COUNT][tfn::kOutCount];
    float tuned_ms[tfn::KIND_COUNT][tfn::GRAD_COUNT][tfn::PHI_COUNT][tfn::kOutCount];
    tfn::Stage stages[3];
    tfn_ctx()
    {
        for (auto &a : tuned)
            for (auto &b : a)
                for (auto &c : b)
                    for (auto &d : c) d = -1;
        for (auto &a : tuned_ms)
            for (auto &b : a)
                for (auto &c : b)
                    for (auto &d : c) d = 0.f;
    }
};

struct tfn_plan {
    tfn_ctx *ctx = nullptr;
    void *dev = nullptr;  // FrameDesc[n] then CUtensorMap[n]
    size_t bytes = 0;
    int n = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace tfn {

struct DeviceGuard {  // switches to the context's device for the call's duration
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cuda_ok(cudaSetDevice(dev), "cudaSetDevice");
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// The layout of a descriptor slot (context slots, plans, server pipelines):
// FrameDesc[cap], then CUtensorMap[cap] (128-byte aligned), then the launch's
// refinement list (kRefineListBytes, 128-byte aligned).
size_t slot_bytes(int cap);
FrameDesc *slot_descs(void *base);
CUtensorMap *slot_maps(void *base, int cap);
void *slot_refine(void *base, int cap);

// Device allocations counted against the context's budget.
tfn_status ctx_alloc(tfn_ctx *c, void **p, size_t bytes);
void ctx_free(tfn_ctx *c, void *&p, size_t bytes);

// True when a launch over frames[0..n) would have fewer than two 18-row work
// items (shape 0) per resident warp (one or a few small frames).
inline bool small_launch(const tfn_frame *frames, int n, int num_sms)
{
    long long items = 0;
    for (int i = 0; i < n; ++i) items += frame_tiles(frames[i], 0);
    return items < (long long)num_sms * 32;
}

// Tile shape for a launch over frames[0..n) (one input kind) with method m:
// forced (tfn_set_tile_shape), else the tune table's, else the short-item
// shape for a small launch, else kDefaultCfg.
inline int choose_cfg(const tfn_ctx *c, const tfn_frame *frames, int n, const tfn_method &m)
{
    if (c->forced_cfg >= 0) return c->forced_cfg;
    const int t = c->tuned[frames[0].input_type][method_grad(m)][method_phi(m)][m.output];
    if (t >= 0) return t;
    return small_launch(frames, n, c->num_sms) ? kSmallCfg : kDefaultCfg;
}

// Enqueues the estimator over frames[0..n) (device pointers, already
// validated) on `stream`: one persistent launch per run of frames of one
// input kind.  The kernels report to `status` (2 words: failed-wait bits,
// refined pixels), the context's status word when null.
tfn_status run_batch(tfn_ctx *c, const tfn_frame *frames, int n, const tfn_method &m, cudaStream_t stream,
                     uint32_t *status = nullptr);

}  // namespace tfn
