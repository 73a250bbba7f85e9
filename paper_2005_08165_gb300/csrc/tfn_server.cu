// tfn_server.cu -- the serving form: a thread-safe request server with
// continuous batching and memory-budget admission.
//
// Clients submit single frames (any size, input type and intrinsics; one
// method per server) from any thread and get a ticket; tfn_wait blocks, with a
// limit, until that frame's normals are in the client's buffers.  Inside, two
// threads run the pipeline:
//
//   launcher: waits until requests are queued and a pipeline is free, admits
//             requests from the front of the queue while the batch stays within
//             max_batch_frames and its staging bytes fit in one block of the
//             ring arena (host-buffer requests are staged through device
//             memory; device-buffer requests need none), then enqueues on that
//             pipeline's stream: host-to-device copies, one persistent kernel
//             launch per input type over the whole batch (the same launch path
//             as tfn_normals_batch), device-to-host copies, an event;
//   retirer:  waits for the oldest batch in flight, checks its kernels' status
//             word (one per pipeline, zeroed per batch), completes the batch's
//             requests (status, latency), releases its arena block and
//             wakes the waiters and the launcher.
//
// Requests that arrive while batches are in flight queue up and form the next
// batch as soon as a pipeline frees up (continuous batching); with
// max_delay_us > 0 the launcher also holds a partial batch for up to that long
// while the device is busy.  Every pixel's result is independent of which
// other frames share its launch, so a request gets the same bits alone and in
// any mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/tfn.h"
#include "tfn_ctx.h"
#include "tfn_internal.h"
#include "tfn_sched.h"

using namespace tfn;

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kMaxPipes = 4;
constexpr size_t kLatencyWindow = 65536;

size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }
size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

int out_bytes_per_elem(int fmt)
{
    return fmt == OUT_F32 || fmt == OUT_OCT16 ? 4 : (fmt == OUT_F16 || fmt == OUT_BF16) ? 2 : 8;
}

// Device staging layout of one host-buffer request: input, normals, mask.
struct StageLayout {
    size_t in_pitch, out_pitch, mask_pitch, pts_pitch;
    size_t in_off, out_off, mask_off, pts_off, bytes;
    int planes;
};

StageLayout stage_layout(const tfn_frame &f, int fmt)
{
    StageLayout L;
    const int ob = out_bytes_per_elem(fmt);
    L.planes = fmt <= OUT_BF16 ? 3 : 1;
    L.in_pitch = al16((size_t)f.width * kind_elem_size(f.input_type));
    L.out_pitch = al16((size_t)f.width * ob);
    L.mask_pitch = al16((size_t)f.width);
    L.in_off = 0;
    L.out_off = al256(L.in_pitch * f.height);
    L.mask_off = L.out_off + al256(L.out_pitch * f.height * L.planes);
    L.pts_pitch = al16((size_t)f.width * 4);
    L.pts_off = L.mask_off + al256(L.mask_pitch * f.height);
    L.bytes = L.pts_off + (f.points ? al256(L.pts_pitch * f.height * 3) : 0);
    return L;
}

struct Request {
    uint64_t ticket;
    tfn_frame frame;  // as submitted
    bool host;
    bool test_wait;      // TFN_REQ_TEST_WAIT_TIMEOUT
    size_t stage_bytes;  // 0 for device-buffer requests
    Clock::time_point t_submit;
};

struct Result {
    bool done = false;
    tfn_status status = TFN_OK;
};

struct Batch {
    int pipe;
    bool has_block;
    bool captured = false;  // its kernels were captured into a new graph (not replayed from one)
    std::vector<Request> reqs;
    tfn_status launch_status = TFN_OK;  // failure while enqueueing
};

// The descriptors of one launch (one input kind) of a pipeline's batches:
// a descriptor slot (slot_bytes) and its pinned host mirror.
struct GroupBuf {
    void *dev = nullptr, *host = nullptr;
    int cap = 0;
};

// A batch's kernels as a CUDA graph: the status word's reset, then per
// launch (input kind) normals_kernel and its refinement kernel, if any.
// Captured once per key (the method's flags, then per launch its kind, tile
// shape, whether it runs the NOREF kernel and whether it refines in a second
// kernel: together they fix the kernels); replayed with each kernel node's
// grid and arguments updated to the batch.
struct GraphEntry {
    std::vector<int> key;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaGraphNode_t> fn_node, rf_node;  // per launch
};
constexpr size_t kMaxGraphs = 64;  // per pipeline, least recently used first out

struct Pipe {
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;  // the stream graphs are captured on
    cudaEvent_t done = nullptr;
    cudaEvent_t k_start = nullptr, k_end = nullptr;  // (timing) around the batch's kernels
    uint32_t *status_dev = nullptr;   // the status word of this pipeline's kernels, zeroed per batch
    uint32_t *status_host = nullptr;  // its pinned copy after the batch
    GroupBuf groups[KIND_COUNT];
    std::vector<GraphEntry> graphs;
    bool busy = false;
};

}  // namespace

struct tfn_server {
    tfn_ctx *ctx = nullptr;  // the server's own context (the launcher thread uses it alone)
    tfn_method method;
    size_t max_batch = 256, max_queue = 65536;
    int max_delay_us = 0;
    int npipes = 2;
    bool use_graphs = true;
    cudaEvent_t t0_event = nullptr;  // the zero of the device timeline of the batches (timing)
    float last_kernel_end_ms = -1.f;  // (retirer) when the previous batch's kernels ended
    Pipe pipes[kMaxPipes];
    void *arena_base = nullptr;
    size_t arena_bytes = 0;
    RingArena arena;

    std::mutex mu;
    std::condition_variable cv_launch;  // launcher: queue or resources changed
    std::condition_variable cv_retire;  // retirer: a batch was launched
    std::condition_variable cv_done;    // waiters: a request completed
    std::deque<Request> queue;
    std::deque<Batch> inflight;
    std::unordered_map<uint64_t, Result> results;
    uint64_t next_ticket = 1;
    bool stopping = false, launcher_done = false;
    std::thread launcher, retirer;

    // statistics (under mu)
    uint64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, rejected = 0, batches = 0, batch_frames = 0;
    uint64_t pixels = 0;
    uint64_t graph_launches = 0, graph_captures = 0, max_inflight = 0, admitted_busy = 0, device_overlaps = 0;
    Clock::time_point t0;
    std::vector<float> lat_us;  // ring of the last kLatencyWindow latencies
    size_t lat_next = 0;
    int inflight_reqs = 0;
};

namespace {

void complete_locked(tfn_server *s, const Request &r, tfn_status st, Clock::time_point now)
{
    auto it = s->results.find(r.ticket);
    if (it != s->results.end()) {
        it->second.done = true;
        it->second.status = st;
    }
    if (st == TFN_OK) {
        ++s->completed;
        s->pixels += (uint64_t)r.frame.height * r.frame.width;
        const float us = std::chrono::duration<float, std::micro>(now - r.t_submit).count();
        if (s->lat_us.size() < kLatencyWindow)
            s->lat_us.push_back(us);
        else
            s->lat_us[s->lat_next] = us;
        s->lat_next = (s->lat_next + 1) % kLatencyWindow;
    } else if (st == TFN_ERR_CANCELLED) {
        ++s->cancelled;
    } else {
        ++s->failed;
    }
}

void destroy_graph(GraphEntry &e)
{
    if (e.exec) cudaGraphExecDestroy(e.exec);
    if (e.graph) cudaGraphDestroy(e.graph);
    e.exec = nullptr;
    e.graph = nullptr;
}

// Enqueues a batch's kernels (frames of any input kinds, device pointers)
// on the pipeline's stream from one of its graphs: the frames grouped by
// input kind, one launch each, the descriptors in the pipeline's own slots.
tfn_status enqueue_kernels_graph(tfn_server *s, Pipe &p, const std::vector<tfn_frame> &dev, const tfn_method &m,
                                 bool *captured)
{
    tfn_ctx *c = s->ctx;
    std::vector<LaunchSpec> specs;
    std::vector<int> key{m.flags};
    std::vector<tfn_frame> fr;
    for (int kind = 0; kind < KIND_COUNT; ++kind) {
        fr.clear();
        for (const tfn_frame &f : dev)
            if (f.input_type == kind) fr.push_back(f);
        if (fr.empty()) continue;
        const int n = (int)fr.size();
        const int cfg = choose_cfg(c, fr.data(), n, m);
        GroupBuf &g = p.groups[kind];
        if (g.cap < n) {
            // (the pipeline is idle: its previous batch has retired)
            const int cap = std::max(n, std::max(8, 2 * g.cap));
            if (g.dev) cudaFree(g.dev);
            if (g.host) cudaFreeHost(g.host);
            g.dev = g.host = nullptr;
            g.cap = 0;
            if (!cuda_ok(cudaMalloc(&g.dev, slot_bytes(cap)), "cudaMalloc(descriptors)") ||
                !cuda_ok(cudaMemset(slot_refine(g.dev, cap), 0, 128), "cudaMemset(refinement list)") ||
                !cuda_ok(cudaMallocHost(&g.host, slot_bytes(cap)), "cudaMallocHost(descriptors)"))
                return TFN_ERR_CUDA;
            g.cap = cap;
        }
        FrameDesc *d = slot_descs(g.host);
        CUtensorMap *maps = slot_maps(g.host, g.cap);
        int tiles = 0;
        for (int i = 0; i < n; ++i) {
            d[i] = describe_frame(fr[i], cfg, m, tiles);
            tiles += frame_tiles(fr[i], cfg);
            tfn_status st = encode_map(&maps[i], fr[i], cfg);
            if (st) return st;
        }
        const size_t off_maps = (uintptr_t)maps - (uintptr_t)g.host;
        if (!cuda_ok(cudaMemcpyAsync(g.dev, g.host, (size_t)n * sizeof(FrameDesc), cudaMemcpyHostToDevice, p.stream),
                     "cudaMemcpyAsync(descriptors)") ||
            !cuda_ok(cudaMemcpyAsync((char *)g.dev + off_maps, maps, (size_t)n * sizeof(CUtensorMap),
                                     cudaMemcpyHostToDevice, p.stream),
                     "cudaMemcpyAsync(tensor maps)"))
            return TFN_ERR_CUDA;
        LaunchSpec L;
        const bool noref = refinement_idle(fr.data(), n, m);
        tfn_status st = make_launch(kind, m, cfg, noref, slot_descs(g.dev), slot_maps(g.dev, g.cap), p.status_dev,
                                    slot_refine(g.dev, g.cap), kRefineCap, n, tiles, c->num_sms, &L);
        if (st) return st;
        if (L.grid < 1) continue;
        specs.push_back(L);
        key.insert(key.end(), {kind, cfg, noref, L.rf != nullptr});
    }
    // the graphs are kept in order of use: a hit moves to the back, a capture
    // past the limit evicts the front (the least recently used)
    GraphEntry *ge = nullptr;
    for (size_t i = 0; i < p.graphs.size(); ++i)
        if (p.graphs[i].key == key) {
            std::rotate(p.graphs.begin() + i, p.graphs.begin() + i + 1, p.graphs.end());
            ge = &p.graphs.back();
            break;
        }
    *captured = ge == nullptr;
    if (ge) {
        for (size_t i = 0; i < specs.size(); ++i) {
            LaunchSpec &L = specs[i];
            void *params[] = {&L.args};
            cudaKernelNodeParams kp = {};
            kp.func = (void *)L.fn;
            kp.gridDim = dim3(L.grid);
            kp.blockDim = dim3(L.threads);
            kp.sharedMemBytes = (unsigned)L.smem;
            kp.kernelParams = params;
            if (!cuda_ok(cudaGraphExecKernelNodeSetParams(ge->exec, ge->fn_node[i], &kp), "cudaGraphExecKernelNodeSetParams"))
                return TFN_ERR_CUDA;
            if (L.rf) {
                kp.func = (void *)L.rf;
                kp.gridDim = dim3(L.rf_grid);
                kp.blockDim = dim3(kRefineThreads);
                kp.sharedMemBytes = 0;
                if (!cuda_ok(cudaGraphExecKernelNodeSetParams(ge->exec, ge->rf_node[i], &kp),
                             "cudaGraphExecKernelNodeSetParams(refine)"))
                    return TFN_ERR_CUDA;
            }
        }
    } else {
        if (p.graphs.size() >= kMaxGraphs) {  // (the least recently used goes)
            destroy_graph(p.graphs.front());
            p.graphs.erase(p.graphs.begin());
        }
        GraphEntry e;
        e.key = key;
        if (!cuda_ok(cudaStreamBeginCapture(p.capture, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture"))
            return TFN_ERR_CUDA;
        tfn_status st = cuda_ok(cudaMemsetAsync(p.status_dev, 0, 2 * sizeof(uint32_t), p.capture), "cudaMemsetAsync")
                            ? TFN_OK
                            : TFN_ERR_CUDA;
        for (size_t i = 0; i < specs.size() && st == TFN_OK; ++i) st = enqueue_launch(specs[i], p.capture);
        if (!cuda_ok(cudaStreamEndCapture(p.capture, &e.graph), "cudaStreamEndCapture") && st == TFN_OK) st = TFN_ERR_CUDA;
        if (st == TFN_OK && !cuda_ok(cudaGraphInstantiate(&e.exec, e.graph, 0), "cudaGraphInstantiate")) st = TFN_ERR_CUDA;
        // the kernel nodes of each launch, found by their functions (a batch's
        // launches are of distinct input kinds, so their functions differ)
        size_t nn = 0;
        if (st == TFN_OK && !cuda_ok(cudaGraphGetNodes(e.graph, nullptr, &nn), "cudaGraphGetNodes")) st = TFN_ERR_CUDA;
        std::vector<cudaGraphNode_t> nodes(nn);
        if (st == TFN_OK && nn && !cuda_ok(cudaGraphGetNodes(e.graph, nodes.data(), &nn), "cudaGraphGetNodes"))
            st = TFN_ERR_CUDA;
        e.fn_node.assign(specs.size(), nullptr);
        e.rf_node.assign(specs.size(), nullptr);
        for (size_t k = 0; k < nn && st == TFN_OK; ++k) {
            cudaGraphNodeType t;
            if (!cuda_ok(cudaGraphNodeGetType(nodes[k], &t), "cudaGraphNodeGetType")) st = TFN_ERR_CUDA;
            if (st || t != cudaGraphNodeTypeKernel) continue;
            cudaKernelNodeParams kp;
            if (!cuda_ok(cudaGraphKernelNodeGetParams(nodes[k], &kp), "cudaGraphKernelNodeGetParams")) st = TFN_ERR_CUDA;
            for (size_t i = 0; i < specs.size() && st == TFN_OK; ++i) {
                if (kp.func == (void *)specs[i].fn) e.fn_node[i] = nodes[k];
                if (specs[i].rf && kp.func == (void *)specs[i].rf) e.rf_node[i] = nodes[k];
            }
        }
        for (size_t i = 0; i < specs.size() && st == TFN_OK; ++i)
            if (!e.fn_node[i] || (specs[i].rf && !e.rf_node[i])) st = TFN_ERR_CUDA;
        if (st) {
            destroy_graph(e);
            return st;
        }
        p.graphs.push_back(e);
        ge = &p.graphs.back();
    }
    if (!cuda_ok(cudaGraphLaunch(ge->exec, p.stream), "cudaGraphLaunch")) return TFN_ERR_CUDA;
    return TFN_OK;
}

// Enqueues one batch on its pipeline's stream (launcher thread, no lock held).
tfn_status enqueue_batch(tfn_server *s, Batch &b, size_t block_off)
{
    Pipe &p = s->pipes[b.pipe];
    const int fmt = s->method.output;
    const int ob = out_bytes_per_elem(fmt);
    std::vector<tfn_frame> dev(b.reqs.size());
    size_t off = block_off;
    for (size_t i = 0; i < b.reqs.size(); ++i) {
        const Request &r = b.reqs[i];
        if (!r.host) {
            dev[i] = r.frame;
            continue;
        }
        const tfn_frame &f = r.frame;
        const StageLayout L = stage_layout(f, fmt);
        char *base = (char *)s->arena_base + off;
        off += r.stage_bytes;
        tfn_frame d = f;
        d.input = base + L.in_off;
        d.input_pitch = (int64_t)L.in_pitch;
        d.normals = base + L.out_off;
        d.normals_pitch = (int64_t)L.out_pitch;
        d.normals_plane_stride = (int64_t)(L.out_pitch * f.height);
        d.mask = (uint8_t *)(base + L.mask_off);
        d.mask_pitch = (int64_t)L.mask_pitch;
        if (f.points) {
            d.points = base + L.pts_off;
            d.points_pitch = (int64_t)L.pts_pitch;
            d.points_plane_stride = (int64_t)(L.pts_pitch * f.height);
        }
        dev[i] = d;
        if (!cuda_ok(cudaMemcpy2DAsync((void *)d.input, L.in_pitch, f.input, (size_t)f.input_pitch,
                                       (size_t)f.width * kind_elem_size(f.input_type), f.height, cudaMemcpyHostToDevice,
                                       p.stream),
                     "cudaMemcpy2DAsync(H2D)"))
            return TFN_ERR_CUDA;
    }
    tfn_method m = s->method;
    for (const Request &r : b.reqs)
        if (r.test_wait) m.flags |= TFN_FLAG_TEST_WAIT_TIMEOUT;
    if (!cuda_ok(cudaEventRecord(p.k_start, p.stream), "cudaEventRecord")) return TFN_ERR_CUDA;
    // each batch reports only its own kernels' failed waits (the graphs reset
    // the pipeline's status word themselves)
    tfn_status st;
    if (s->use_graphs) {
        st = enqueue_kernels_graph(s, p, dev, m, &b.captured);
    } else {
        st = cuda_ok(cudaMemsetAsync(p.status_dev, 0, 2 * sizeof(uint32_t), p.stream), "cudaMemsetAsync(status)")
                 ? run_batch(s->ctx, dev.data(), (int)dev.size(), m, p.stream, p.status_dev)
                 : TFN_ERR_CUDA;
    }
    if (st) return st;
    if (!cuda_ok(cudaEventRecord(p.k_end, p.stream), "cudaEventRecord")) return TFN_ERR_CUDA;
    for (size_t i = 0; i < b.reqs.size(); ++i) {
        const Request &r = b.reqs[i];
        if (!r.host) continue;
        const tfn_frame &f = r.frame, &d = dev[i];
        const int planes = fmt <= OUT_BF16 ? 3 : 1;
        for (int q = 0; q < planes; ++q)
            if (!cuda_ok(cudaMemcpy2DAsync((char *)f.normals + q * f.normals_plane_stride, (size_t)f.normals_pitch,
                                           (const char *)d.normals + q * d.normals_plane_stride,
                                           (size_t)d.normals_pitch, (size_t)f.width * ob, f.height,
                                           cudaMemcpyDeviceToHost, p.stream),
                         "cudaMemcpy2DAsync(D2H)"))
                return TFN_ERR_CUDA;
        if (!cuda_ok(cudaMemcpy2DAsync(f.mask, (size_t)f.mask_pitch, d.mask, (size_t)d.mask_pitch, f.width, f.height,
                                       cudaMemcpyDeviceToHost, p.stream),
                     "cudaMemcpy2DAsync(D2H)"))
            return TFN_ERR_CUDA;
        if (f.points)
            for (int q = 0; q < 3; ++q)
                if (!cuda_ok(cudaMemcpy2DAsync((char *)f.points + q * f.points_plane_stride, (size_t)f.points_pitch,
                                               (const char *)d.points + q * d.points_plane_stride,
                                               (size_t)d.points_pitch, (size_t)f.width * 4, f.height,
                                               cudaMemcpyDeviceToHost, p.stream),
                             "cudaMemcpy2DAsync(D2H)"))
                    return TFN_ERR_CUDA;
    }
    if (!cuda_ok(cudaMemcpyAsync(p.status_host, p.status_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, p.stream),
                 "cudaMemcpyAsync(status)") ||
        !cuda_ok(cudaEventRecord(p.done, p.stream), "cudaEventRecord"))
        return TFN_ERR_CUDA;
    return TFN_OK;
}

void launcher_main(tfn_server *s)
{
    DeviceGuard g(s->ctx->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        int pipe = -1;
        for (;;) {
            if (s->stopping) break;
            pipe = -1;
            for (int k = 0; k < s->npipes; ++k)
                if (!s->pipes[k].busy) {
                    pipe = k;
                    break;
                }
            if (pipe >= 0 && !s->queue.empty()) {
                // optional batching delay: hold a partial batch while the device is busy
                bool any_busy = false;
                for (int k = 0; k < s->npipes; ++k) any_busy |= s->pipes[k].busy;
                if (s->max_delay_us > 0 && any_busy && s->queue.size() < s->max_batch) {
                    const auto deadline = s->queue.front().t_submit + std::chrono::microseconds(s->max_delay_us);
                    if (Clock::now() < deadline) {
                        s->cv_launch.wait_until(lk, deadline);
                        continue;
                    }
                }
                size_t bytes = 0;
                const size_t k = admit_count(s->queue, s->max_batch, s->arena.largest_fit(),
                                             [](const Request &r) { return r.stage_bytes; }, &bytes);
                if (k > 0) break;
            }
            s->cv_launch.wait(lk);
        }
        if (s->stopping) break;
        // admit
        size_t bytes = 0;
        const size_t k = admit_count(s->queue, s->max_batch, s->arena.largest_fit(),
                                     [](const Request &r) { return r.stage_bytes; }, &bytes);
        if (!s->inflight.empty()) s->admitted_busy += k;  // admitted while an earlier batch is on the GPU
        Batch b;
        b.pipe = pipe;
        b.reqs.assign(s->queue.begin(), s->queue.begin() + k);
        s->queue.erase(s->queue.begin(), s->queue.begin() + k);
        size_t off = 0;
        b.has_block = bytes > 0;
        if (b.has_block) off = s->arena.alloc(bytes);  // fits: admit_count checked largest_fit
        s->pipes[pipe].busy = true;
        s->inflight_reqs += (int)k;
        ++s->batches;
        s->batch_frames += k;
        lk.unlock();
        b.launch_status = enqueue_batch(s, b, off);
        if (b.launch_status != TFN_OK) {
            // let the stream drain what was enqueued before the failure, so the
            // retirer can release the block safely
            cudaEventRecord(s->pipes[pipe].done, s->pipes[pipe].stream);
        }
        lk.lock();
        if (b.launch_status == TFN_OK && s->use_graphs) ++s->graph_launches;
        if (b.captured) ++s->graph_captures;
        s->inflight.push_back(std::move(b));
        s->max_inflight = std::max<uint64_t>(s->max_inflight, s->inflight.size());
        s->cv_retire.notify_one();
    }
    // cancel what was never admitted
    const auto now = Clock::now();
    for (const Request &r : s->queue) complete_locked(s, r, TFN_ERR_CANCELLED, now);
    s->queue.clear();
    s->launcher_done = true;
    s->cv_retire.notify_one();
    s->cv_done.notify_all();
}

void retirer_main(tfn_server *s)
{
    DeviceGuard g(s->ctx->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv_retire.wait(lk, [s] { return !s->inflight.empty() || s->launcher_done; });
        if (s->inflight.empty()) break;  // launcher finished and nothing in flight
        const int pipe = s->inflight.front().pipe;
        const bool launched = s->inflight.front().launch_status == TFN_OK;
        Pipe &p = s->pipes[pipe];
        lk.unlock();
        tfn_status st = cuda_ok(cudaEventSynchronize(p.done), "cudaEventSynchronize") ? TFN_OK : TFN_ERR_CUDA;
        const auto now = Clock::now();
        // when this batch's kernels ran on the device, against the previous batch's
        float t_start = 0.f, t_end = 0.f;
        const bool timed = st == TFN_OK && launched &&
                           cudaEventElapsedTime(&t_start, s->t0_event, p.k_start) == cudaSuccess &&
                           cudaEventElapsedTime(&t_end, s->t0_event, p.k_end) == cudaSuccess;
        if (!timed) cudaGetLastError();
        lk.lock();
        if (timed) {
            if (s->last_kernel_end_ms >= 0.f && t_start < s->last_kernel_end_ms) ++s->device_overlaps;
            s->last_kernel_end_ms = std::max(s->last_kernel_end_ms, t_end);
        }
        Batch b = std::move(s->inflight.front());
        s->inflight.pop_front();
        if (st == TFN_OK) st = b.launch_status;
        if (st == TFN_OK && *p.status_host != 0) st = TFN_ERR_DEVICE;  // a kernel gave up a bounded wait
        for (const Request &r : b.reqs) complete_locked(s, r, st, now);
        if (b.has_block) s->arena.free_oldest();
        p.busy = false;
        s->inflight_reqs -= (int)b.reqs.size();
        s->cv_done.notify_all();
        s->cv_launch.notify_one();
    }
}

void destroy_resources(tfn_server *s)
{
    for (Pipe &p : s->pipes) {
        if (p.stream) {
            cudaStreamSynchronize(p.stream);
            cudaStreamDestroy(p.stream);
        }
        if (p.done) cudaEventDestroy(p.done);
        if (p.status_host) cudaFreeHost(p.status_host);
        if (p.status_dev) cudaFree(p.status_dev);
        for (GraphEntry &e : p.graphs) destroy_graph(e);
        for (GroupBuf &g : p.groups) {
            if (g.dev) cudaFree(g.dev);
            if (g.host) cudaFreeHost(g.host);
        }
        if (p.capture) cudaStreamDestroy(p.capture);
        if (p.k_start) cudaEventDestroy(p.k_start);
        if (p.k_end) cudaEventDestroy(p.k_end);
    }
    if (s->t0_event) cudaEventDestroy(s->t0_event);
    if (s->arena_base) cudaFree(s->arena_base);
    if (s->ctx) tfn_destroy(s->ctx);
}

// Geometry, type and intrinsics of a host-buffer request, checked on a
// stand-in frame with the staging pointers and pitches it would get.
tfn_status validate_host_request(const tfn_frame &f, int fmt)
{
    if (!f.input || !f.normals || !f.mask) return TFN_ERR_INVALID_ARG;
    if (f.height < 1 || f.width < 1 || f.height > 32768 || f.width > 32768 || f.input_type < 0 ||
        f.input_type >= KIND_COUNT)
        return TFN_ERR_INVALID_ARG;
    const int ob = out_bytes_per_elem(fmt);
    if (f.input_pitch < (int64_t)f.width * kind_elem_size(f.input_type) || f.normals_pitch < (int64_t)f.width * ob ||
        f.mask_pitch < f.width)
        return TFN_ERR_INVALID_ARG;
    if (fmt <= OUT_BF16 && f.normals_plane_stride < f.normals_pitch * (int64_t)f.height) return TFN_ERR_INVALID_ARG;
    if (f.points && (f.points_pitch < (int64_t)f.width * 4 || f.points_plane_stride < f.points_pitch * f.height))
        return TFN_ERR_INVALID_ARG;
    const StageLayout L = stage_layout(f, fmt);
    tfn_frame d = f;
    d.input = (const void *)(uintptr_t)256;
    d.input_pitch = (int64_t)L.in_pitch;
    d.normals = (void *)(uintptr_t)256;
    d.normals_pitch = (int64_t)L.out_pitch;
    d.normals_plane_stride = (int64_t)(L.out_pitch * f.height);
    d.mask = (uint8_t *)(uintptr_t)256;
    d.mask_pitch = (int64_t)L.mask_pitch;
    if (f.points) {
        d.points = (void *)(uintptr_t)256;
        d.points_pitch = (int64_t)L.pts_pitch;
        d.points_plane_stride = (int64_t)(L.pts_pitch * f.height);
    }
    return validate_frame(&d, fmt);
}

}  // namespace

extern "C" {

tfn_status tfn_server_create(tfn_ctx *ctx, const tfn_server_opts *o, tfn_server **out)
{
    if (!out) return TFN_ERR_INVALID_ARG;
    *out = nullptr;
    if (!ctx || !o) return TFN_ERR_INVALID_ARG;
    tfn_status st = validate_method(&o->method);
    if (st) return st;
    if (o->max_batch_frames < 0 || o->max_queue < 0 || o->max_delay_us < 0 || o->pipelines < 0 ||
        o->pipelines > kMaxPipes)
        return TFN_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return TFN_ERR_CUDA;
    tfn_server *s = new (std::nothrow) tfn_server();
    if (!s) return TFN_ERR_OUT_OF_MEMORY;
    s->method = o->method;
    s->max_batch = o->max_batch_frames ? (size_t)o->max_batch_frames : 256;
    s->max_queue = o->max_queue ? (size_t)o->max_queue : 65536;
    s->max_delay_us = o->max_delay_us;
    s->npipes = o->pipelines ? o->pipelines : 2;
    if (o->flags & ~TFN_SERVER_NO_GRAPHS) {
        delete s;
        return TFN_ERR_INVALID_ARG;
    }
    s->use_graphs = !(o->flags & TFN_SERVER_NO_GRAPHS);
    s->arena_bytes = o->mem_budget_bytes ? o->mem_budget_bytes : ((size_t)1 << 30);
    if ((st = tfn_create(&s->ctx, ctx->device, 0))) {
        delete s;
        return st;
    }
    // the server inherits the caller's tune table and forced shape
    memcpy(s->ctx->tuned, ctx->tuned, sizeof ctx->tuned);
    memcpy(s->ctx->tuned_ms, ctx->tuned_ms, sizeof ctx->tuned_ms);
    s->ctx->forced_cfg = ctx->forced_cfg;
    cudaError_t e = cudaMalloc(&s->arena_base, s->arena_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        s->arena_base = nullptr;
        destroy_resources(s);
        delete s;
        return e == cudaErrorMemoryAllocation ? TFN_ERR_OUT_OF_MEMORY : TFN_ERR_CUDA;
    }
    s->arena = RingArena(s->arena_bytes, 256);
    for (int k = 0; k < s->npipes; ++k) {
        Pipe &p = s->pipes[k];
        if (!cuda_ok(cudaStreamCreateWithFlags(&p.stream, cudaStreamNonBlocking), "cudaStreamCreate") ||
            !cuda_ok(cudaEventCreateWithFlags(&p.done, cudaEventDisableTiming), "cudaEventCreate") ||
            !cuda_ok(cudaMallocHost((void **)&p.status_host, sizeof(uint32_t)), "cudaMallocHost") ||
            !cuda_ok(cudaMalloc((void **)&p.status_dev, 256), "cudaMalloc(status)") ||
            !cuda_ok(cudaMemset(p.status_dev, 0, 256), "cudaMemset(status)") ||
            !cuda_ok(cudaStreamCreateWithFlags(&p.capture, cudaStreamNonBlocking), "cudaStreamCreate") ||
            !cuda_ok(cudaEventCreate(&p.k_start), "cudaEventCreate") ||
            !cuda_ok(cudaEventCreate(&p.k_end), "cudaEventCreate")) {
            destroy_resources(s);
            delete s;
            return TFN_ERR_CUDA;
        }
        *p.status_host = 0;
    }
    if (!cuda_ok(cudaEventCreate(&s->t0_event), "cudaEventCreate") ||
        !cuda_ok(cudaEventRecord(s->t0_event, s->pipes[0].stream), "cudaEventRecord") ||
        !cuda_ok(cudaEventSynchronize(s->t0_event), "cudaEventSynchronize")) {
        destroy_resources(s);
        delete s;
        return TFN_ERR_CUDA;
    }
    s->t0 = Clock::now();
    s->lat_us.reserve(kLatencyWindow);
    try {
        s->launcher = std::thread(launcher_main, s);
        s->retirer = std::thread(retirer_main, s);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stopping = true;
        }
        s->cv_launch.notify_all();
        if (s->launcher.joinable()) s->launcher.join();
        if (s->retirer.joinable()) s->retirer.join();
        destroy_resources(s);
        delete s;
        return TFN_ERR_OUT_OF_MEMORY;
    }
    *out = s;
    return TFN_OK;
}

tfn_status tfn_submit(tfn_server *s, const tfn_frame *frame, int flags, uint64_t *ticket)
{
    if (!s || !frame || !ticket || (flags & ~(TFN_REQ_HOST | TFN_REQ_TEST_WAIT_TIMEOUT))) return TFN_ERR_INVALID_ARG;
    const bool host = flags & TFN_REQ_HOST;
    tfn_status st = host ? validate_host_request(*frame, s->method.output) : validate_frame(frame, s->method.output);
    if (st) return st;
    Request r;
    r.frame = *frame;
    r.host = host;
    r.test_wait = flags & TFN_REQ_TEST_WAIT_TIMEOUT;
    r.stage_bytes = host ? s->arena.round(stage_layout(*frame, s->method.output).bytes) : 0;
    if (r.stage_bytes > s->arena.capacity()) return TFN_ERR_OUT_OF_MEMORY;  // could never be admitted
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return TFN_ERR_CANCELLED;
    if (s->queue.size() >= s->max_queue) {
        ++s->rejected;
        return TFN_ERR_BUSY;
    }
    r.ticket = s->next_ticket++;
    r.t_submit = Clock::now();
    s->results.emplace(r.ticket, Result());
    s->queue.push_back(r);
    ++s->submitted;
    *ticket = r.ticket;
    s->cv_launch.notify_one();
    return TFN_OK;
}

tfn_status tfn_wait(tfn_server *s, uint64_t ticket, int32_t timeout_ms, tfn_status *result)
{
    if (!s || !result || timeout_ms < 0) return TFN_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return TFN_ERR_INVALID_ARG;  // unknown, or already waited for
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
    while (!it->second.done) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !it->second.done)
            return TFN_ERR_TIMEOUT;
        it = s->results.find(ticket);
        if (it == s->results.end()) return TFN_ERR_INVALID_ARG;  // consumed by a concurrent waiter
    }
    *result = it->second.status;
    s->results.erase(it);
    return TFN_OK;
}

tfn_status tfn_server_stats(tfn_server *s, tfn_serving_stats *o, int reset)
{
    if (!s || !o) return TFN_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    memset(o, 0, sizeof *o);
    o->submitted = s->submitted;
    o->completed = s->completed;
    o->failed = s->failed;
    o->cancelled = s->cancelled;
    o->rejected = s->rejected;
    o->batches = s->batches;
    o->pixels = s->pixels;
    const auto now = Clock::now();
    o->elapsed_s = std::chrono::duration<double>(now - s->t0).count();
    o->frames_per_s = o->elapsed_s > 0 ? (double)s->completed / o->elapsed_s : 0.0;
    o->mean_batch_frames = s->batches ? (double)s->batch_frames / (double)s->batches : 0.0;
    if (!s->lat_us.empty()) {
        std::vector<float> v(s->lat_us);
        auto at = [&v](double q) {
            const size_t i = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
            std::nth_element(v.begin(), v.begin() + i, v.end());
            return (double)v[i];
        };
        o->latency_p50_us = at(0.50);
        o->latency_p99_us = at(0.99);
        o->latency_max_us = *std::max_element(v.begin(), v.end());
        o->latency_samples = v.size();
    }
    o->queued = (int32_t)s->queue.size();
    o->in_flight = s->inflight_reqs;
    o->staging_bytes_in_use = s->arena.in_use();
    o->staging_bytes_capacity = s->arena.capacity();
    o->graph_launches = s->graph_launches;
    o->max_batches_in_flight = s->max_inflight;
    o->admitted_while_busy = s->admitted_busy;
    o->device_overlaps = s->device_overlaps;
    o->graph_captures = s->graph_captures;
    if (reset) {
        s->submitted = s->completed = s->failed = s->cancelled = s->rejected = s->batches = s->batch_frames = 0;
        s->graph_launches = s->graph_captures = s->max_inflight = s->admitted_busy = s->device_overlaps = 0;
        s->pixels = 0;
        s->t0 = now;
        s->lat_us.clear();
        s->lat_next = 0;
    }
    return TFN_OK;
}

tfn_status tfn_server_destroy(tfn_server *s)
{
    if (!s) return TFN_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_launch.notify_all();
    if (s->launcher.joinable()) s->launcher.join();
    if (s->retirer.joinable()) s->retirer.join();
    DeviceGuard g(s->ctx->device);
    destroy_resources(s);
    delete s;
    return TFN_OK;
}

}  // extern "C"
