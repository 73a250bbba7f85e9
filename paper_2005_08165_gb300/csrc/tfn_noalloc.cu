// tfn_noalloc.cu -- tfn_normals_noalloc: the normal estimator without any
// device allocation, for callers that must not allocate.
//
// Who needs it: code that runs under a fixed device-memory plan -- a host
// framework or plugin interface that owns every device byte and forbids its
// extensions to call cudaMalloc, or a latency-critical loop where cudaMalloc
// / cudaFree could synchronise the device and stall other streams.  Such a
// caller cannot create a tfn_ctx (a context allocates its scratch), so this
// entry point keeps the scratch the kernels need -- per-frame descriptors,
// TMA tensor maps, the status word and the refinement list -- in one
// file-scope __device__ array of fixed size instead.
//
// The array is a device symbol: in host code its name is only a host-side
// stand-in, so the first call on each device (with that device current)
// looks up its device address with cudaGetSymbolAddress and caches it.
// Every call shares the one array and overwrites what the previous call left
// there; calls whose GPU work overlaps (different streams, or work still
// running from a previous call on another stream) race on it.
#include <cstring>
#include <mutex>

#include "../../include/tfn.h"
#include "tfn_ctx.h"
#include "tfn_internal.h"

namespace {

using namespace tfn;

constexpr int kMax = TFN_NOALLOC_MAX_FRAMES;
constexpr int kMaxDevices = 64;

// Layout of the scratch array (also used for the host-side staging copy).
struct alignas(256) Scratch {
    CUtensorMap maps[kMax];  // 128 bytes each, 64-byte aligned
    FrameDesc desc[kMax];
    uint32_t status[64];
    alignas(128) unsigned char refine[refine_list_bytes(kNoallocRefineCap)];  // the refinement list (runs of a call take turns)
};
// The host-side staging of a call: what is copied into the scratch.
struct Staging {
    CUtensorMap maps[kMax];
    FrameDesc desc[kMax];
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(Scratch)];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// Device address of the scratch array and the SM count for the current device.
tfn_status device_setup(int dev, Scratch **addr, int *sms)
{
    if (dev < 0 || dev >= kMaxDevices) return TFN_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (!cuda_ok(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress")) return TFN_ERR_CUDA;
        int n = 0;
        if (!cuda_ok(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute"))
            return TFN_ERR_CUDA;
        g_addr[dev] = p;
        g_sms[dev] = n;
    }
    *addr = (Scratch *)g_addr[dev];
    *sms = g_sms[dev];
    return TFN_OK;
}

}  // namespace

extern "C" tfn_status tfn_normals_noalloc(const tfn_frame *frames, int n, const tfn_method *method, tfn_stream stream)
{
    if (n < 0 || (n > 0 && !frames)) return TFN_ERR_INVALID_ARG;
    if (n > kMax) return TFN_ERR_INVALID_ARG;  // the fixed scratch holds at most kMax frames
    tfn_status st = validate_method(method);
    if (st) return st;
    for (int i = 0; i < n; ++i)
        if ((st = validate_frame(&frames[i], method->output))) return st;
    if (n == 0) return TFN_OK;
    // The copies below read the thread-local staging when the stream runs
    // them.  A stream that records its work instead of running it would read
    // the staging later, after other calls have overwritten it: such a stream
    // gets TFN_ERR_UNSUPPORTED and nothing is enqueued.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (!cuda_ok(cudaStreamIsCapturing((cudaStream_t)stream, &cap), "cudaStreamIsCapturing")) return TFN_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return TFN_ERR_UNSUPPORTED;
    int dev = 0;
    if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice")) return TFN_ERR_CUDA;
    Scratch *d = nullptr;
    int sms = 0;
    if ((st = device_setup(dev, &d, &sms))) return st;

    // Descriptors and tensor maps are built in thread-local host storage (no
    // allocation) and copied into the device array on the caller's stream.
    // A copy from pageable memory returns once its source has been consumed
    // (the runtime may first wait for the work already queued on the stream
    // to stage it), so the staging is free for the next call once this one
    // returns.
    thread_local Staging h;
    // one launch per run of frames of one input kind; a small run takes the short-item shape
    int run_cfg[kMax];
    for (int i = 0; i < n;) {
        int j = i + 1;
        while (j < n && frames[j].input_type == frames[i].input_type) ++j;
        const int cfg = small_launch(frames + i, j - i, sms) ? kSmallCfg : kDefaultCfg;
        for (int k = i; k < j; ++k) run_cfg[k] = cfg;
        i = j;
    }
    int tb = 0;
    for (int i = 0; i < n; ++i) {
        if (i > 0 && frames[i].input_type != frames[i - 1].input_type)
            tb = 0;  // a new launch (input kind) starts its own tile queue
        h.desc[i] = describe_frame(frames[i], run_cfg[i], *method, tb);
        tb += frame_tiles(frames[i], run_cfg[i]);
        if ((st = encode_map(&h.maps[i], frames[i], run_cfg[i]))) return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (!cuda_ok(cudaMemcpyAsync(d->maps, h.maps, (size_t)n * sizeof(CUtensorMap), cudaMemcpyHostToDevice, s),
                 "cudaMemcpyAsync") ||
        !cuda_ok(cudaMemcpyAsync(d->desc, h.desc, (size_t)n * sizeof(FrameDesc), cudaMemcpyHostToDevice, s),
                 "cudaMemcpyAsync") ||
        !cuda_ok(cudaMemsetAsync(d->status, 0, sizeof d->status, s), "cudaMemsetAsync") ||
        // the list's count and the refinement kernel's block counter start at
        // zero whatever an earlier (possibly overlapping) call left there
        !cuda_ok(cudaMemsetAsync(d->refine, 0, 128, s), "cudaMemsetAsync"))
        return TFN_ERR_CUDA;
    // one launch per run of frames of the same input kind
    for (int i = 0; i < n;) {
        int j = i + 1;
        while (j < n && frames[j].input_type == frames[i].input_type) ++j;
        int total = 0;
        for (int k = i; k < j; ++k) total += frame_tiles(frames[k], run_cfg[i]);
        st = launch_normals(frames[i].input_type, *method, run_cfg[i], refinement_idle(frames + i, j - i, *method),
                            d->desc + i, d->maps + i, d->status, d->refine, kNoallocRefineCap, j - i, total, sms, s);
        if (st) return st;
        i = j;
    }
    return TFN_OK;
}
