// Batched regularisation of many independent scatterplots (the panels of a
// scatterplot matrix) and the band-height autotuner.
//
// Each panel has its own context (resolution, buffers) and runs as one branch
// of one CUDA graph (a fork from the capture stream to one stream per branch
// and a join back), so that the phases of different panels overlap.  With
// DC_OPT_BATCHED_LAUNCHES the panels of one resolution instead form a
// class whose every step is one launch over all its panels (the kernels take
// a table of the panels' buffers and index it with blockIdx.y); the results
// are bit-identical, but at 120 panels of 256^2..1024^2 the per-panel
// branches measured faster (10.3 ms against 11.4 ms for 6 iterations): each
// panel's launches already fill the GPU, and the class launches serialise
// what the branches overlap.  Classes that cannot take the batched launches
// (grids from 2048^2, kept sample order) always run per panel.  The graph is
// cached per (sample pointers, sizes, iterations, metrics).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <mutex>
#include <tuple>
#include <vector>

#include "dc_internal.cuh"

using namespace dc;

struct dc_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap_stream = nullptr;
    dc_params base{};
    std::vector<dc_ctx *> ctx;
    std::vector<uint32_t> log2;
    std::vector<int64_t> cap;
    std::vector<cudaStream_t> branch;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    bool batched = false;  // batched launches per resolution class (DC_OPT_BATCHED_LAUNCHES)
    struct Entry {
        std::vector<const void *> pos;
        std::vector<int64_t> n;
        int iters = 0;
        int metrics = 0;
        cudaGraphExec_t exec = nullptr;
        std::vector<void *> tables;  // device PanelDesc arrays of the batched classes
    };
    std::vector<Entry> graphs;
};

namespace {

dc_status bfail(dc_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return st;
}

#define DC_BCUDA(call)                                                                            \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return bfail(DC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

struct Guard {
    int prev = -1;
    bool changed = false;
    explicit Guard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
    }
    ~Guard()
    {
        if (changed) cudaSetDevice(prev);
    }
};

// Autotuned settings, per GPU model (name and SM count, so that a cache file
// carries over to other runs and devices of the same model), resolution,
// radius, carry mode, sample order, floor(log2 n) and whether the launch
// options were searched: -> (band rows, options).
using TuneKey = std::tuple<std::string, int, int, int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune_cache;

std::string gpu_model(int device, int *sms)
{
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        cudaGetLastError();
        *sms = 0;
        return "unknown";
    }
    *sms = prop.multiProcessorCount;
    std::string name = prop.name;
    for (auto &ch : name)
        if (ch == ' ' || ch == '\t') ch = '_';
    return name;
}

int n_bucket(int64_t n) { return n > 0 ? (int)std::floor(std::log2((double)n)) : 0; }

void drop_entry(dc_batch::Entry &e)
{
    if (e.exec) cudaGraphExecDestroy(e.exec);
    for (void *t : e.tables) cudaFree(t);
    e.exec = nullptr;
    e.tables.clear();
}

void drop_graphs(dc_batch *b)
{
    for (auto &e : b->graphs) drop_entry(e);
    b->graphs.clear();
}

// Can a class of panels (same context settings) take the batched launches?
bool batchable(const dc_ctx *c)
{
    return c->p.keep_order == 0 && c->g.N >= 32 && c->g.N < 2048 && (c->mode == MODE_FLOAT || c->mode == MODE_COUNT);
}

// The iteration sequence of enqueue_regularize for P same-resolution panels
// at once (tab: their device PanelDesc array; c0: one of their contexts).
cudaError_t enqueue_class(const dc_ctx *c0, cudaStream_t s, const PanelDesc *tab, int P, int64_t max_n, int iters,
                          int metrics)
{
    const int lg = c0->g.log2N;
    cudaError_t e = launch_zero_batched(s, tab, P, lg, 0, metrics ? 3 * iters : 0);
    if (e == cudaSuccess) e = launch_splat_rank_batched(s, tab, P, max_n, lg);
    if (e == cudaSuccess) e = launch_reorder_batched(s, tab, P, max_n, lg);
    int cur = 0;
    for (int it = 0; it < iters && e == cudaSuccess; ++it) {
        const int nxt = cur ^ 1;
        const bool need_next = (it + 1 < iters) || metrics;
        if (c0->mode == MODE_FLOAT) e = launch_smooth_batched(s, tab, P, lg, c0->w, cur, need_next);
        if (e == cudaSuccess) e = launch_band_batched(s, c0->g, c0->mode, c0->p.carry_mode, tab, P, cur, need_next);
        if (e == cudaSuccess)
            e = launch_advect_batched(s, tab, P, max_n, lg, c0->p.pixel_center, c0->p.clamp_positions,
                                      need_next ? nxt : -1, true);
        if (e == cudaSuccess && metrics) e = launch_quality_batched(s, tab, P, lg, nxt, it);
        if (need_next) cur = nxt;
    }
    if (e == cudaSuccess) e = launch_back_batched(s, tab, P, max_n);
    return e;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

// Times regularize(iters) on a copy of the samples for every band height
// 1, 2, 4, .. 64 with at most 1024 bands and the automatic height, and, with
// search_options, for each of the launch sequences (default, separate
// smoothing in float mode, one cooperative band launch below 2048^2); keeps
// the fastest (median of five runs after two warm-ups).
dc_status tune(const dc_params *params, int device, void *cuda_stream, const float *pos_xy, int64_t n, int32_t iters,
               bool search_options, int *best_rows, int *best_opts, float *best_ms_out)
{
    if (!params) return bfail(DC_ERR_INVALID_ARG, "null params");
    if (n <= 0 || !pos_xy || (reinterpret_cast<uintptr_t>(pos_xy) & 7)) return bfail(DC_ERR_INVALID_ARG, "samples");
    if (iters < 1) return bfail(DC_ERR_INVALID_ARG, "iters = %d", iters);
    if (params->log2_res < 4 || params->log2_res > 13) return bfail(DC_ERR_NOT_POW2, "log2_res");
    const int N = 1 << params->log2_res;
    const int r = params->kernel_r < 0 ? (N / 128 < 2 ? 2 : N / 128) : params->kernel_r;
    int sms = 0;
    const std::string model = gpu_model(device, &sms);
    const TuneKey key{model, sms, (int)params->log2_res, r, (int)params->carry_mode, (int)params->keep_order,
                      n_bucket(n), search_options ? 1 : 0};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *best_rows = it->second.first;
            *best_opts = it->second.second;
            if (best_ms_out) *best_ms_out = -1.f;
            return DC_OK;
        }
    }
    Guard guard(device);
    float *tmp = nullptr;
    if (cudaMalloc(&tmp, sizeof(float) * 2 * (size_t)n) != cudaSuccess) {
        cudaGetLastError();
        return bfail(DC_ERR_OOM, "autotune staging");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = 0, best_o = params->options;
    float best_ms = 0.f;
    dc_status st = DC_OK;
    const int base_opts = params->options & ~(DC_OPT_FUSED_BANDS | DC_OPT_SEPARATE_SMOOTH);
    std::vector<int> opt_set{search_options ? base_opts : params->options};
    if (search_options) {
        if (r > 0) opt_set.push_back(base_opts | DC_OPT_SEPARATE_SMOOTH);
        if (N < 2048) opt_set.push_back(base_opts | DC_OPT_FUSED_BANDS);
    }
    // powers of two, then the automatic height (one band per SM)
    const int T_auto = make_band_geom(params->log2_res, 0, device_sms()).T;
    for (int opts : opt_set) {
        for (int Tk = 1; Tk <= 128 && st == DC_OK; Tk *= 2) {
            const int T = Tk <= 64 ? Tk : T_auto;
            if (Tk > 64 && (T_auto & (T_auto - 1)) == 0) continue;  // already timed
            if (T > N || (N + T - 1) / T > 1024) continue;
            dc_params p = *params;
            p.band_rows = T;
            p.options = opts;
            dc_ctx *c = nullptr;
            if ((st = declutter_create(&p, device, cuda_stream, &c)) != DC_OK) break;
            float ms[5];
            for (int rep = -2; rep < 5 && st == DC_OK; ++rep) {
                if (cudaMemcpyAsync(tmp, pos_xy, sizeof(float) * 2 * (size_t)n, cudaMemcpyDeviceToDevice,
                                    c->stream) != cudaSuccess) {
                    st = bfail(DC_ERR_CUDA, "autotune copy");
                    break;
                }
                cudaEventRecord(e0, c->stream);
                st = regularize(c, tmp, n, iters, nullptr);
                cudaEventRecord(e1, c->stream);
                if (st == DC_OK && cudaEventSynchronize(e1) != cudaSuccess) st = bfail(DC_ERR_CUDA, "autotune sync");
                if (st == DC_OK && rep >= 0) cudaEventElapsedTime(&ms[rep], e0, e1);
            }
            declutter_destroy(c);
            if (st != DC_OK) break;
            std::sort(ms, ms + 5);
            if (!best || ms[2] < best_ms) {
                best = T;
                best_o = opts;
                best_ms = ms[2];
            }
        }
        if (st != DC_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(tmp);
    if (st != DC_OK) return st;
    if (!best) return bfail(DC_ERR_INVALID_ARG, "no band height fits");
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = {best, best_o};
    }
    *best_rows = best;
    *best_opts = best_o;
    if (best_ms_out) *best_ms_out = best_ms;
    return DC_OK;
}

constexpr const char *kTuneHeader = "declutter-autotune 1";

}  // namespace

extern "C" {

dc_status declutter_autotune_band_rows(const dc_params *params, int device, void *cuda_stream, const float *pos_xy,
                                       int64_t n, int32_t iters, int32_t *best_out, float *best_ms_out)
{
    if (!best_out) return bfail(DC_ERR_INVALID_ARG, "null best_out");
    int rows = 0, opts = 0;
    if (dc_status st = tune(params, device, cuda_stream, pos_xy, n, iters, false, &rows, &opts, best_ms_out)) return st;
    *best_out = rows;
    return DC_OK;
}

dc_status declutter_autotune(const dc_params *params, int device, void *cuda_stream, const float *pos_xy, int64_t n,
                             int32_t iters, dc_params *best_out, float *best_ms_out)
{
    if (!best_out) return bfail(DC_ERR_INVALID_ARG, "null best_out");
    int rows = 0, opts = 0;
    if (dc_status st = tune(params, device, cuda_stream, pos_xy, n, iters, true, &rows, &opts, best_ms_out)) return st;
    *best_out = *params;
    best_out->band_rows = rows;
    best_out->options = opts;
    return DC_OK;
}

dc_status declutter_autotune_save(const char *path)
{
    if (!path) return bfail(DC_ERR_INVALID_ARG, "null path");
    FILE *f = std::fopen(path, "w");
    if (!f) return bfail(DC_ERR_INVALID_ARG, "cannot write %s", path);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    std::fprintf(f, "%s\n", kTuneHeader);
    for (const auto &kv : g_tune_cache) {
        const auto &k = kv.first;
        std::fprintf(f, "%s %d %d %d %d %d %d %d %d %d\n", std::get<0>(k).c_str(), std::get<1>(k), std::get<2>(k),
                     std::get<3>(k), std::get<4>(k), std::get<5>(k), std::get<6>(k), std::get<7>(k), kv.second.first,
                     kv.second.second);
    }
    const bool ok = std::fclose(f) == 0;
    return ok ? DC_OK : bfail(DC_ERR_INVALID_ARG, "write error on %s", path);
}

dc_status declutter_autotune_load(const char *path)
{
    if (!path) return bfail(DC_ERR_INVALID_ARG, "null path");
    FILE *f = std::fopen(path, "r");
    if (!f) return bfail(DC_ERR_INVALID_ARG, "cannot read %s", path);
    char line[512];
    std::vector<std::pair<TuneKey, std::pair<int, int>>> got;
    bool ok = std::fgets(line, sizeof(line), f) && std::strncmp(line, kTuneHeader, std::strlen(kTuneHeader)) == 0;
    while (ok && std::fgets(line, sizeof(line), f)) {
        char name[256];
        int v[10];
        if (std::sscanf(line, "%255s %d %d %d %d %d %d %d %d %d", name, &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6],
                        &v[7], &v[8]) != 10 ||
            v[7] < 1 || v[7] > 64 || v[1] < 4 || v[1] > 13) {
            ok = false;
            break;
        }
        got.push_back({TuneKey{name, v[0], v[1], v[2], v[3], v[4], v[5], v[6]}, {v[7], v[8]}});
    }
    std::fclose(f);
    if (!ok) return bfail(DC_ERR_INVALID_ARG, "%s is not a declutter autotune cache", path);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto &e : got) g_tune_cache[e.first] = e.second;
    return DC_OK;
}

dc_status declutter_autotune_clear(void)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache.clear();
    return DC_OK;
}

dc_status declutter_batch_create(const dc_params *base, const uint32_t *log2_res, const int64_t *max_samples,
                                 int32_t n_panels, int device, void *cuda_stream, dc_batch **out)
{
    if (!base || !log2_res || !max_samples || !out) return bfail(DC_ERR_INVALID_ARG, "null argument");
    if (n_panels < 1 || n_panels > 4096) return bfail(DC_ERR_INVALID_ARG, "n_panels = %d", n_panels);
    *out = nullptr;
    Guard guard(device);
    dc_batch *b = new dc_batch();
    b->device = device;
    b->base = *base;
    b->batched = (base->options & DC_OPT_BATCHED_LAUNCHES) != 0;
    auto bail = [&](dc_status st) {
        declutter_batch_destroy(b);
        return st;
    };
    if (cuda_stream) {
        b->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreate(&b->stream) != cudaSuccess) return bail(bfail(DC_ERR_CUDA, "cudaStreamCreate"));
        b->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
        return bail(bfail(DC_ERR_CUDA, "stream or event creation"));
    for (int p = 0; p < n_panels; ++p) {
        if (max_samples[p] < 0 || max_samples[p] >= (int64_t(1) << 32))
            return bail(bfail(DC_ERR_INVALID_ARG, "max_samples[%d]", p));
        dc_params pp = *base;
        pp.log2_res = log2_res[p];
        dc_ctx *c = nullptr;
        if (dc_status st = declutter_create(&pp, device, b->stream, &c)) return bail(st);
        // panels run as concurrent graph branches: no cooperative launches,
        // whose CTAs must all be resident at once; and the smoothing as its
        // own launch (the fused kernel's wide CTAs, 3/4 of them idle during
        // the aggregate, measured slower when panels overlap: 11.5 ms
        // against 10.2 ms for 120 panels, the same bits)
        c->fused = false;
        c->smooth_agg = false;
        b->ctx.push_back(c);
        b->log2.push_back(log2_res[p]);
        b->cap.push_back(max_samples[p]);
        cudaStream_t br = nullptr;
        cudaEvent_t ev = nullptr;
        if (cudaStreamCreateWithFlags(&br, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
            return bail(bfail(DC_ERR_CUDA, "branch stream"));
        b->branch.push_back(br);
        b->join.push_back(ev);
        if (dc_status st = prepare_regularize(c, max_samples[p], 1, 0)) return bail(st);
    }
    *out = b;
    return DC_OK;
}

dc_status declutter_batch_destroy(dc_batch *b)
{
    if (!b) return DC_OK;
    Guard guard(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    for (auto *c : b->ctx) declutter_destroy(c);
    for (auto s : b->branch) cudaStreamDestroy(s);
    for (auto e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return DC_OK;
}

dc_status declutter_batch_autotune(dc_batch *b, float *const *pos_xy, const int64_t *n, int32_t iters,
                                   int32_t *band_rows_out)
{
    if (!b || !pos_xy || !n) return bfail(DC_ERR_INVALID_ARG, "null argument");
    Guard guard(b->device);
    const int P = (int)b->ctx.size();
    // one representative per resolution: the panel with the most samples
    std::map<uint32_t, int> rep;
    for (int p = 0; p < P; ++p) {
        auto it = rep.find(b->log2[p]);
        if (it == rep.end() || n[p] > n[it->second]) rep[b->log2[p]] = p;
    }
    std::map<uint32_t, int> best;
    for (auto &kv : rep) {
        dc_params pp = b->base;
        pp.log2_res = kv.first;
        int32_t T = 0;
        if (dc_status st = declutter_autotune_band_rows(&pp, b->device, b->stream, pos_xy[kv.second], n[kv.second],
                                                        iters, &T, nullptr))
            return st;
        best[kv.first] = T;
    }
    drop_graphs(b);
    for (int p = 0; p < P; ++p) {
        const int T = best[b->log2[p]];
        if (b->ctx[p]->g.T != T) {
            dc_params pp = b->base;
            pp.log2_res = b->log2[p];
            pp.band_rows = T;
            dc_ctx *c = nullptr;
            if (dc_status st = declutter_create(&pp, b->device, b->stream, &c)) return st;
            c->fused = false;  // as in declutter_batch_create
            c->smooth_agg = false;
            if (dc_status st = prepare_regularize(c, b->cap[p], 1, 0)) {
                declutter_destroy(c);
                return st;
            }
            declutter_destroy(b->ctx[p]);
            b->ctx[p] = c;
        }
        if (band_rows_out) band_rows_out[p] = T;
    }
    return DC_OK;
}

dc_status declutter_batch_regularize(dc_batch *b, float *const *pos_xy, const int64_t *n, int32_t iters,
                                     double *uniformity_out)
{
    if (!b || !pos_xy || !n) return bfail(DC_ERR_INVALID_ARG, "null argument");
    if (iters < 0) return bfail(DC_ERR_INVALID_ARG, "iters = %d", iters);
    if (iters == 0) return DC_OK;
    Guard guard(b->device);
    const int P = (int)b->ctx.size();
    const int metrics = uniformity_out ? 1 : 0;
    bool moved = false;
    for (int p = 0; p < P; ++p) {
        if (n[p] < 0 || n[p] > b->cap[p]) return bfail(DC_ERR_INVALID_ARG, "n[%d] = %lld", p, (long long)n[p]);
        if (n[p] > 0 && (!pos_xy[p] || (reinterpret_cast<uintptr_t>(pos_xy[p]) & 7)))
            return bfail(DC_ERR_INVALID_ARG, "pos_xy[%d]", p);
        const void *q0 = b->ctx[p]->qacc, *s0 = b->ctx[p]->spos;
        if (dc_status st = prepare_regularize(b->ctx[p], n[p], iters, metrics)) return st;
        moved |= q0 != b->ctx[p]->qacc || s0 != b->ctx[p]->spos;
    }
    if (moved) drop_graphs(b);  // cached graphs hold the old buffer addresses
    cudaGraphExec_t exec = nullptr;
    for (auto &e : b->graphs) {
        if (e.iters != iters || e.metrics != metrics) continue;
        bool same = true;
        for (int p = 0; p < P && same; ++p) same = e.pos[p] == pos_xy[p] && e.n[p] == n[p];
        if (same) exec = e.exec;
    }
    if (!exec) {
        if (b->graphs.size() >= 8) {
            drop_entry(b->graphs.front());
            b->graphs.erase(b->graphs.begin());
        }
        dc_batch::Entry en;
        // classes of batchable panels (same resolution); the rest run alone
        std::map<uint32_t, std::vector<int>> classes;
        std::vector<int> alone;
        for (int p = 0; p < P; ++p) {
            if (b->batched && batchable(b->ctx[p])) classes[b->log2[p]].push_back(p);
            else alone.push_back(p);
        }
        std::vector<std::pair<std::vector<int>, const PanelDesc *>> groups;
        for (auto &kv : classes) {
            std::vector<PanelDesc> host;
            for (int p : kv.second) host.push_back(panel_desc(b->ctx[p], pos_xy[p], n[p]));
            void *dev = nullptr;
            if (cudaMalloc(&dev, sizeof(PanelDesc) * host.size()) != cudaSuccess) {
                cudaGetLastError();
                drop_entry(en);
                return bfail(DC_ERR_OOM, "panel table");
            }
            en.tables.push_back(dev);
            if (cudaMemcpy(dev, host.data(), sizeof(PanelDesc) * host.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
                drop_entry(en);
                return bfail(DC_ERR_CUDA, "panel table upload");
            }
            groups.push_back({kv.second, static_cast<const PanelDesc *>(dev)});
        }
        cudaGraph_t graph = nullptr;
        DC_BCUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaEventRecord(b->fork, b->cap_stream);
        // branch k uses the stream and join event of the k-th panel
        int k = 0;
        for (auto &gtab : groups) {
            if (e != cudaSuccess) break;
            const std::vector<int> &ps = gtab.first;
            int64_t max_n = 0;
            for (int p : ps) max_n = std::max(max_n, n[p]);
            e = cudaStreamWaitEvent(b->branch[k], b->fork, 0);
            if (e == cudaSuccess) e = enqueue_class(b->ctx[ps[0]], b->branch[k], gtab.second, (int)ps.size(), max_n,
                                                    iters, metrics);
            if (e == cudaSuccess) e = cudaEventRecord(b->join[k], b->branch[k]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap_stream, b->join[k], 0);
            ++k;
        }
        for (int p : alone) {
            if (e != cudaSuccess) break;
            e = cudaStreamWaitEvent(b->branch[k], b->fork, 0);
            if (e == cudaSuccess) e = enqueue_regularize(b->ctx[p], b->branch[k], pos_xy[p], n[p], iters, metrics);
            if (e == cudaSuccess) e = cudaEventRecord(b->join[k], b->branch[k]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap_stream, b->join[k], 0);
            ++k;
        }
        cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            drop_entry(en);
            return bfail(DC_ERR_CUDA, "batch capture: %s / %s", cudaGetErrorString(e), cudaGetErrorString(e2));
        }
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            drop_entry(en);
            return bfail(DC_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
        }
        en.pos.assign(pos_xy, pos_xy + P);
        en.n.assign(n, n + P);
        en.iters = iters;
        en.metrics = metrics;
        en.exec = exec;
        b->graphs.push_back(en);
    }
    DC_BCUDA(cudaGraphLaunch(exec, b->stream));
    for (int p = 0; p < P; ++p) finish_regularize(b->ctx[p], n[p], iters, metrics);
    if (metrics) {
        std::vector<unsigned long long> acc(3 * (size_t)iters * P);
        for (int p = 0; p < P; ++p)
            DC_BCUDA(cudaMemcpyAsync(acc.data() + 3 * (size_t)iters * p, b->ctx[p]->qacc,
                                     3 * (size_t)iters * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                     b->stream));
        DC_BCUDA(cudaStreamSynchronize(b->stream));
        for (int p = 0; p < P; ++p)
            for (int it = 0; it < iters; ++it) {
                double m[3];
                read_metrics(b->ctx[p], &acc[3 * ((size_t)iters * p + it)], m);
                uniformity_out[(size_t)iters * p + it] = m[0];
            }
    }
    return DC_OK;
}

dc_status declutter_batch_sync(dc_batch *b)
{
    if (!b) return bfail(DC_ERR_INVALID_ARG, "null batch");
    Guard guard(b->device);
    DC_BCUDA(cudaStreamSynchronize(b->stream));
    for (auto *c : b->ctx)
        if (dc_status st = declutter_sync(c)) return st;
    return DC_OK;
}

}  // extern "C"
