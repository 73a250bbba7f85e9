// tfn_tune.cu -- tile-shape autotuner and its persistent cache.
//
// Every compiled tile shape (item height and CTA width) computes the same
// bits (the kernels' per-pixel arithmetic does not depend on the shape), so
// the choice is purely one of speed.  tfn_autotune times each shape on a
// batch the caller provides and
// records the fastest in the context's table under (input kind, gradient,
// phi, output); later launches of that combination use it.  The table can be
// written to a text file and read back on a later run on the same kind of
// device:
//
//   tfn-tune 2
//   device <name with spaces as '_'> sms <SM count> cc <major>.<minor>
//   entry <input> <grad> <phi> <output> <tile_w> <tile_h> <rows_per_thread> <warps_3x3> <warps_other> <ms>
//
// Shapes are stored by geometry (item size and CTA widths), not by index, so
// that a cache stays valid across builds that compile a different list of
// shapes (entries whose shape is not compiled are skipped).  Version 1 files
// (no CTA widths) load as the shapes of the default widths.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/tfn.h"
#include "tfn_ctx.h"
#include "tfn_internal.h"

using namespace tfn;

namespace {

std::string device_line(int dev)
{
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return std::string();
    std::string name(p.name);
    for (char &ch : name)
        if (ch == ' ' || ch == '\t' || ch == '\n') ch = '_';
    char buf[320];
    snprintf(buf, sizeof buf, "device %s sms %d cc %d.%d", name.c_str(), p.multiProcessorCount, p.major, p.minor);
    return buf;
}

// (version 1 entries give no widths: the default ones, 2 warps for the 3x3 filters and 4 for the others)
int shape_index(int tw, int th, int pr, int w3 = 2, int w5 = 4)
{
    for (int k = 0; k < kNumCfg; ++k)
        if (kCfgs[k].tw == tw && kCfgs[k].th == th && kCfgs[k].pr == pr && kCfgs[k].warps3 == w3 &&
            kCfgs[k].warps5 == w5)
            return k;
    return -1;
}

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

}  // namespace

extern "C" {

tfn_status tfn_autotune(tfn_ctx *c, const tfn_frame *frames, int n, const tfn_method *m, int reps,
                        tfn_stream stream, int *best, float *ms_per_shape)
{
    if (!c || n < 1 || !frames || reps < 1 || reps > 10000) return TFN_ERR_INVALID_ARG;
    tfn_status st = validate_method(m);
    if (st) return st;
    for (int i = 0; i < n; ++i)
        if ((st = validate_frame(&frames[i], m->output))) return st;
    DeviceGuard g(c->device);
    if (!g.ok) return TFN_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    EventPair ev;
    if (!cuda_ok(cudaEventCreate(&ev.a), "cudaEventCreate") || !cuda_ok(cudaEventCreate(&ev.b), "cudaEventCreate"))
        return TFN_ERR_CUDA;
    const int saved = c->forced_cfg;
    float ms[kNumCfg];
    for (int k = 0; k < kNumCfg && st == TFN_OK; ++k) {
        c->forced_cfg = k;
        // one untimed run uploads this shape's descriptors and warms the caches
        if ((st = run_batch(c, frames, n, *m, s))) break;
        if (!cuda_ok(cudaEventRecord(ev.a, s), "cudaEventRecord")) st = TFN_ERR_CUDA;
        for (int r = 0; r < reps && st == TFN_OK; ++r) st = run_batch(c, frames, n, *m, s);
        if (st) break;
        if (!cuda_ok(cudaEventRecord(ev.b, s), "cudaEventRecord") || !cuda_ok(cudaEventSynchronize(ev.b), "cudaEventSynchronize") ||
            !cuda_ok(cudaEventElapsedTime(&ms[k], ev.a, ev.b), "cudaEventElapsedTime"))
            st = TFN_ERR_CUDA;
        ms[k] /= reps;
    }
    c->forced_cfg = saved;
    if (st) return st;
    int b = 0;
    for (int k = 1; k < kNumCfg; ++k)
        if (ms[k] < ms[b]) b = k;
    for (int i = 0; i < n; ++i) {
        const int kind = frames[i].input_type;
        c->tuned[kind][method_grad(*m)][method_phi(*m)][m->output] = (signed char)b;
        c->tuned_ms[kind][method_grad(*m)][method_phi(*m)][m->output] = ms[b];
    }
    c->last_slot = -1;
    if (best) *best = b;
    if (ms_per_shape)
        for (int k = 0; k < kNumCfg; ++k) ms_per_shape[k] = ms[k];
    return TFN_OK;
}

tfn_status tfn_tuned_shape(tfn_ctx *c, int input_type, const tfn_method *m, int *index)
{
    if (!c || !index || input_type < 0 || input_type >= KIND_COUNT) return TFN_ERR_INVALID_ARG;
    tfn_status st = validate_method(m);
    if (st) return st;
    *index = c->tuned[input_type][method_grad(*m)][method_phi(*m)][m->output];
    return TFN_OK;
}

tfn_status tfn_tune_cache_save(tfn_ctx *c, const char *path)
{
    if (!c || !path) return TFN_ERR_INVALID_ARG;
    const std::string dl = device_line(c->device);
    if (dl.empty()) return TFN_ERR_CUDA;
    FILE *f = fopen(path, "w");
    if (!f) return TFN_ERR_IO;
    bool ok = fprintf(f, "tfn-tune 2\n%s\n", dl.c_str()) > 0;
    for (int k = 0; k < KIND_COUNT; ++k)
        for (int gi = 0; gi < GRAD_COUNT; ++gi)
            for (int p = 0; p < PHI_COUNT; ++p)
                for (int o = 0; o < kOutCount; ++o) {
                    const int t = c->tuned[k][gi][p][o];
                    if (t < 0) continue;
                    ok = ok && fprintf(f, "entry %d %d %d %d %d %d %d %d %d %.6f\n", k, gi, p, o, kCfgs[t].tw,
                                       kCfgs[t].th, kCfgs[t].pr, kCfgs[t].warps3, kCfgs[t].warps5,
                                       (double)c->tuned_ms[k][gi][p][o]) > 0;
                }
    ok = (fclose(f) == 0) && ok;
    return ok ? TFN_OK : TFN_ERR_IO;
}

tfn_status tfn_tune_cache_load(tfn_ctx *c, const char *path)
{
    if (!c || !path) return TFN_ERR_INVALID_ARG;
    FILE *f = fopen(path, "r");
    if (!f) return TFN_ERR_IO;
    std::vector<std::string> lines;
    char buf[512];
    while (fgets(buf, sizeof buf, f)) {
        size_t len = strlen(buf);
        if (len == sizeof buf - 1 && buf[len - 1] != '\n') {  // over-long line: not a cache file
            fclose(f);
            return TFN_ERR_INVALID_ARG;
        }
        while (len && (buf[len - 1] == '\n' || buf[len - 1] == '\r')) buf[--len] = 0;
        lines.emplace_back(buf);
    }
    const bool read_ok = !ferror(f);
    fclose(f);
    if (!read_ok) return TFN_ERR_IO;
    if (lines.size() < 2 || (lines[0] != "tfn-tune 1" && lines[0] != "tfn-tune 2")) return TFN_ERR_INVALID_ARG;
    const bool v2 = lines[0] == "tfn-tune 2";
    const std::string dl = device_line(c->device);
    if (dl.empty()) return TFN_ERR_CUDA;
    if (lines[1].compare(0, 7, "device ") != 0) return TFN_ERR_INVALID_ARG;
    if (lines[1] != dl) return TFN_ERR_UNSUPPORTED;  // tuned on another kind of device
    // parse everything before changing the table: a malformed file loads nothing
    struct E {
        int k, g, p, o, shape;
        float ms;
    };
    std::vector<E> es;
    for (size_t i = 2; i < lines.size(); ++i) {
        if (lines[i].empty()) continue;
        int k, gi, p, o, tw, th, pr, w3 = 2, w5 = 4, used = 0;
        float ms;
        const bool parsed =
            v2 ? sscanf(lines[i].c_str(), "entry %d %d %d %d %d %d %d %d %d %f%n", &k, &gi, &p, &o, &tw, &th, &pr, &w3,
                        &w5, &ms, &used) == 10
               : sscanf(lines[i].c_str(), "entry %d %d %d %d %d %d %d %f%n", &k, &gi, &p, &o, &tw, &th, &pr, &ms,
                        &used) == 8;
        if (!parsed || (size_t)used != lines[i].size()) return TFN_ERR_INVALID_ARG;
        if (k < 0 || k >= KIND_COUNT || gi < 0 || gi >= GRAD_COUNT || p < 0 || p >= PHI_COUNT || o < 0 ||
            o >= kOutCount || !(ms >= 0.f))
            return TFN_ERR_INVALID_ARG;
        const int shape = shape_index(tw, th, pr, w3, w5);
        if (shape >= 0) es.push_back({k, gi, p, o, shape, ms});
    }
    for (const E &e : es) {
        c->tuned[e.k][e.g][e.p][e.o] = (signed char)e.shape;
        c->tuned_ms[e.k][e.g][e.p][e.o] = e.ms;
    }
    c->last_slot = -1;
    return TFN_OK;
}

}  // extern "C"
