// C ABI and runtime of libdeclutter: context, buffers, streams, CUDA-graph
// capture of the iteration, instrumentation, error reporting.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "dc_internal.cuh"

using namespace dc;

namespace {

thread_local std::string g_last_error;

// largest grid of the float (smoothed-density) integral images
constexpr int kFloatMaxN = 2048;

dc_status fail(dc_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

#define DC_CUDA(call)                                                                               \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return fail(DC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (changed) cudaSetDevice(prev);
    }
};

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Launch helper for the profiler: a kernel of kind `dup` is launched twice
// in a row, so that the graph's step time grows by that kernel's own
// in-graph cost.  Every duplicated kernel is idempotent or only changes data
// values (the advection moves samples twice), not the amount of work.
struct Recorder {
    int dup = -1;
    int launches[DC_KERNEL_KINDS] = {};
    int times(int kind) const { return kind == dup ? 2 : 1; }
    void count(int kind) { launches[kind] += 1; }
};

double effective_d0(const dc_ctx *c, int64_t n)
{
    const double NN = (double)c->g.N * (double)c->g.N;
    return c->p.d0 < 0.f ? (double)n / NN : (double)c->p.d0;
}

BandArgs band_args(const dc_ctx *c, const void *src, int mode, int64_t n)
{
    BandArgs a{};
    const double NN = (double)c->g.N * (double)c->g.N;
    a.src = src;
    a.mu = mode == MODE_FLOAT ? (float)((double)n / NN) : 0.0f;
    a.agg = c->agg;
    a.agg_stride = c->g.agg_stride;
    a.carry = c->carry;
    a.pixel_center = c->p.pixel_center;
    const double d0 = effective_d0(c, n);
    a.d0 = (float)d0;
    const double S = c->p.pixel_center ? 2.0 * c->g.N : (double)c->g.N;
    const double den = 2.0 * S * NN * ((double)n + d0 * NN);
    a.inv_den_exact = den > 0.0 ? 1.0 / den : 0.0;
    a.status = c->status;
    return a;
}

// memset + splat of pos into `counts`, then (float mode) the smoothing.
cudaError_t enqueue_density(dc_ctx *c, cudaStream_t s, const float *pos, int64_t n, uint32_t *counts,
                            uint32_t *zero_out, Recorder &rec)
{
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)c->g.N * c->g.N, s);
    if (e != cudaSuccess) return e;
    rec.count(K_SPLAT);
    for (int t = 0; t < rec.times(K_SPLAT) && e == cudaSuccess; ++t)
        e = launch_splat(s, reinterpret_cast<const float2 *>(pos), n, counts, c->g.log2N);
    if (e != cudaSuccess) return e;
    if (c->mode == MODE_FLOAT) {
        rec.count(K_SMOOTH);
        for (int t = 0; t < rec.times(K_SMOOTH) && e == cudaSuccess; ++t)
            e = launch_smooth(s, counts, c->dens, c->g.log2N, c->w, zero_out);
    }
    return e;
}

// With smooth_counts (float mode, c->smooth_agg) the aggregate pass also
// smooths smooth_counts into c->dens (= a.src) and zeroes smooth_zero.
cudaError_t enqueue_inims(dc_ctx *c, cudaStream_t s, const BandArgs &a, int mode, Recorder &rec,
                          const uint32_t *smooth_counts = nullptr, uint32_t *smooth_zero = nullptr)
{
    cudaError_t e = cudaSuccess;
    if (c->fused && mode != MODE_GRID64) {
        // the three phases in one cooperative launch (small grids)
        BandArgs f = a;
        f.zero_out = nullptr;
        rec.count(K_BAND_FUSED);
        const unsigned long long limit_ns =
            (c->p.wait_limit_us > 0 ? (unsigned long long)c->p.wait_limit_us : 1000000ull) * 1000ull;
        const unsigned extra = (c->p.options & DC_OPT_TEST_UNREACHED_BARRIER) ? 1u : 0u;
        for (int t = 0; t < rec.times(K_BAND_FUSED) && e == cudaSuccess; ++t)
            e = launch_band_fused(s, c->g, mode, c->p.carry_mode, a, f, c->status + kBarWord, limit_ns, extra);
        return e;
    }
    if (smooth_counts) {
        rec.count(K_SMOOTH_AGG);
        for (int t = 0; t < rec.times(K_SMOOTH_AGG) && e == cudaSuccess; ++t)
            e = launch_smooth_agg(s, c->g, a, c->w, smooth_counts, c->dens, smooth_zero);
    } else {
        rec.count(K_BAND_AGG);
        for (int t = 0; t < rec.times(K_BAND_AGG) && e == cudaSuccess; ++t) e = launch_band_agg(s, c->g, mode, a);
    }
    if (e != cudaSuccess) return e;
    rec.count(K_CARRY);
    for (int t = 0; t < rec.times(K_CARRY) && e == cudaSuccess; ++t)
        e = launch_carry(s, c->g, mode, c->p.carry_mode, c->agg, c->carry);
    if (e != cudaSuccess) return e;
    BandArgs f = a;
    f.zero_out = nullptr;
    rec.count(K_BAND_FINAL);
    for (int t = 0; t < rec.times(K_BAND_FINAL) && e == cudaSuccess; ++t) e = launch_band_final(s, c->g, mode, f);
    return e;
}

// Pieces of the iteration sequence of Sec. 4.3.  Counts alternate between
// two grids: the advection of iteration it also splats the moved samples
// into the other grid, which the smoothing (float mode) or the aggregate
// kernel (exact mode) of iteration it has zeroed.  Only the first iteration
// has its own memset and splat.

// The first splat, in the caller's order, into grid 0; with the reordering,
// its counts key the counting sort of the samples into c->spos.
cudaError_t enqueue_first_splat(dc_ctx *c, cudaStream_t s, const float *pos, int64_t n, bool reorder, Recorder &rec)
{
    uint32_t *cb[2] = {c->counts_buf[0], c->counts_buf[1]};
    cudaError_t e = cudaMemsetAsync(cb[0], 0, sizeof(uint32_t) * (size_t)c->g.N * c->g.N, s);
    if (e != cudaSuccess) return e;
    rec.count(K_SPLAT);
    const float2 *p2 = reinterpret_cast<const float2 *>(pos);
    // samples in host memory: read once over the link, the scatter reads the
    // device copy the splat leaves in hpos
    float2 *copy = reorder && c->copy_first && c->hpos_cap >= n ? reinterpret_cast<float2 *>(c->hpos) : nullptr;
    // from 8M samples the splat only counts and the scatter's first window
    // claims each sample's slot with an atomic on its pixel's cursor (16M
    // samples: 1.96 against 1.99 ms a step); below, the splat's atomics
    // return the ranks (1M samples: 0.222 against 0.225 ms)
    uint32_t *rank = n >= ((int64_t)1 << 23) ? nullptr : c->rank;
    e = reorder ? launch_splat_rank(s, p2, n, cb[0], c->g.log2N, rank, copy)
                : launch_splat(s, p2, n, cb[0], c->g.log2N);
    // a profiling duplicate goes to the other grid, which is zeroed before
    // its next use, so that these counts stay those of pos
    if (e == cudaSuccess && rec.times(K_SPLAT) > 1) e = launch_splat(s, p2, n, cb[1], c->g.log2N);
    if (e != cudaSuccess || !reorder) return e;
    // the reordering reads only the counts, the ranks and the caller's
    // samples, which the first iteration's grid passes do not write: it runs
    // on a branch beside them, and the first advection joins it
    // (enqueue_iteration with join_reorder)
    e = cudaEventRecord(c->ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->ev_fork, 0);
    rec.count(K_REORDER);
    for (int t = 0; t < rec.times(K_REORDER) && e == cudaSuccess; ++t) {
        e = launch_reorder_scan(c->side, cb[0], c->g.log2N, c->partials, c->cursor);
        if (e == cudaSuccess)
            e = launch_reorder_scatter(c->side, copy ? copy : p2, n, c->g.log2N, c->cursor, rank, c->spos, c->inv,
                                       c->status);
    }
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_join, c->side);
    return e;
}

// Iteration it on count grid `cur`: smoothing (float mode), integral images
// and displacement, advection of the samples ipos (pixel order when they
// are not the caller's pos).  need_next: the moved samples are splatted into
// grid cur ^ 1; qacc (or null): the Sec. 6.2 accumulators of that grid;
// dmax (or null): the largest squared move of the iteration.
cudaError_t enqueue_iteration(dc_ctx *c, cudaStream_t s, const float *pos, float *ipos, int64_t n, int cur,
                              bool need_next, unsigned long long *qacc, unsigned *dmax, Recorder &rec,
                              float *tracers = nullptr, int64_t n_tracers = 0, bool join_reorder = false)
{
    cudaError_t e = cudaSuccess;
    uint32_t *cb[2] = {c->counts_buf[0], c->counts_buf[1]};
    const int nxt = cur ^ 1;
    const bool smooth_fused = c->mode == MODE_FLOAT && c->smooth_agg;
    if (c->mode == MODE_FLOAT && !smooth_fused) {
        rec.count(K_SMOOTH);
        for (int t = 0; t < rec.times(K_SMOOTH) && e == cudaSuccess; ++t)
            e = launch_smooth(s, cb[cur], c->dens, c->g.log2N, c->w, need_next ? cb[nxt] : nullptr);
        if (e != cudaSuccess) return e;
    }
    const void *src = c->mode == MODE_FLOAT ? (const void *)c->dens : (const void *)cb[cur];
    BandArgs a = band_args(c, src, c->mode, n);
    a.disp = c->disp;
    a.zero_out = (c->mode != MODE_FLOAT && need_next) ? cb[nxt] : nullptr;
    e = smooth_fused ? enqueue_inims(c, s, a, c->mode, rec, cb[cur], need_next ? cb[nxt] : nullptr)
                     : enqueue_inims(c, s, a, c->mode, rec);
    if (e != cudaSuccess) return e;
    if (join_reorder && (e = cudaStreamWaitEvent(s, c->ev_join, 0)) != cudaSuccess) return e;
    rec.count(K_ADVECT);
    for (int t = 0; t < rec.times(K_ADVECT) && e == cudaSuccess; ++t)
        e = launch_advect(s, reinterpret_cast<float2 *>(ipos), n, c->disp, c->g.log2N, c->p.pixel_center,
                          c->p.clamp_positions, need_next ? cb[nxt] : nullptr, ipos != pos, dmax);
    if (e != cudaSuccess) return e;
    if (n_tracers > 0) {
        // massless tracers: moved by the same field, not splatted
        e = launch_advect(s, reinterpret_cast<float2 *>(tracers), n_tracers, c->disp, c->g.log2N, c->p.pixel_center,
                          c->p.clamp_positions, nullptr);
        if (e != cudaSuccess) return e;
    }
    if (qacc) {
        rec.count(K_QUALITY);
        e = launch_quality(s, cb[nxt], c->g.log2N, qacc);
    }
    return e;
}

// The iteration of Sec. 4.3, `iters` times.  With metrics, the quality of
// the counts after iteration it goes to accumulator slot it.
cudaError_t enqueue_iterations(dc_ctx *c, cudaStream_t s, float *pos, int64_t n, int iters, int metrics,
                               Recorder &rec, float *tracers = nullptr, int64_t n_tracers = 0)
{
    cudaError_t e = cudaSuccess;
    const bool reorder = c->p.keep_order == 0 && n > 0;
    float *ipos = reorder ? reinterpret_cast<float *>(c->spos) : pos;  // samples the iterations move
    if (metrics) {
        e = cudaMemsetAsync(c->qacc, 0, sizeof(unsigned long long) * 3 * (size_t)iters, s);
        if (e != cudaSuccess) return e;
    }
    int cur = 0;
    for (int it = 0; it < iters; ++it) {
        const bool need_next = (it + 1 < iters) || metrics;
        if (it == 0 && (e = enqueue_first_splat(c, s, pos, n, reorder, rec)) != cudaSuccess) return e;
        e = enqueue_iteration(c, s, pos, ipos, n, cur, need_next, metrics ? c->qacc + 3 * it : nullptr, nullptr, rec,
                              tracers, n_tracers, it == 0 && reorder);
        if (e != cudaSuccess) return e;
        if (need_next) cur ^= 1;
    }
    if (reorder && iters > 0) {
        for (int t = 0; t < rec.times(K_REORDER) && e == cudaSuccess; ++t)
            e = launch_reorder_back(s, c->spos, c->inv, n, reinterpret_cast<float2 *>(pos), c->status);
    }
    return e;
}

// Reordering buffers for n samples; grown outside any capture.  Cached graphs
// hold the old pointers, so they are dropped when the buffers move.
dc_status ensure_sort_buffers(dc_ctx *c, int64_t n)
{
    if (c->p.keep_order != 0 || n <= c->sort_cap) return DC_OK;
    DC_CUDA(cudaStreamSynchronize(c->stream));
    for (auto &ge : c->graphs) cudaGraphExecDestroy(ge.exec);
    c->graphs.clear();
    cudaFree(c->spos);
    cudaFree(c->rank);
    cudaFree(c->inv);
    c->spos = nullptr;
    c->rank = nullptr;
    c->inv = nullptr;
    c->sort_cap = 0;
    if (cudaMalloc(&c->spos, sizeof(float2) * (size_t)n) != cudaSuccess ||
        cudaMalloc(&c->rank, sizeof(uint32_t) * (size_t)n) != cudaSuccess ||
        cudaMalloc(&c->inv, sizeof(uint32_t) * (size_t)n) != cudaSuccess) {
        cudaGetLastError();
        return fail(DC_ERR_OOM, "reordering buffers for %lld samples", (long long)n);
    }
    c->sort_cap = n;
    return DC_OK;
}

// Capture the iteration sequence into an executable graph.
dc_status capture_iterations(dc_ctx *c, float *pos, int64_t n, int iters, int metrics, int dup,
                             cudaGraphExec_t *out, Recorder *rec_out)
{
    cudaGraph_t graph = nullptr;
    DC_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    Recorder rec;
    rec.dup = dup;
    cudaError_t e = enqueue_iterations(c, c->cap_stream, pos, n, iters, metrics, rec);
    cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(DC_ERR_CUDA, "graph capture: %s / %s", cudaGetErrorString(e), cudaGetErrorString(e2));
    }
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(DC_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    if (rec_out) *rec_out = rec;
    return DC_OK;
}

// regularize_adaptive's device state for up to `cap` iterations (AdaptState,
// cv[cap], move_px[cap], dmax[cap]); graphs that point at an old buffer are
// dropped when it moves.
constexpr size_t kAdaptHead = 64;
size_t adapt_bytes(int cap) { return kAdaptHead + (size_t)cap * (2 * sizeof(double) + sizeof(unsigned)); }
double *adapt_cv(const dc_ctx *c) { return reinterpret_cast<double *>(static_cast<char *>(c->adapt) + kAdaptHead); }
double *adapt_move(const dc_ctx *c) { return adapt_cv(c) + c->adapt_cap; }
unsigned *adapt_dmax(const dc_ctx *c) { return reinterpret_cast<unsigned *>(adapt_move(c) + c->adapt_cap); }

dc_status ensure_adapt(dc_ctx *c, int cap)
{
    if (cap <= c->adapt_cap) return DC_OK;
    DC_CUDA(cudaStreamSynchronize(c->stream));
    for (auto it = c->graphs.begin(); it != c->graphs.end();) {
        if (it->adaptive) {
            cudaGraphExecDestroy(it->exec);
            it = c->graphs.erase(it);
        } else {
            ++it;
        }
    }
    cudaFree(c->adapt);
    c->adapt = nullptr;
    c->adapt_cap = 0;
    if (cudaMalloc(&c->adapt, adapt_bytes(cap)) != cudaSuccess) {
        cudaGetLastError();
        return fail(DC_ERR_OOM, "adaptive state for %d iterations", cap);
    }
    c->adapt_cap = cap;
    return DC_OK;
}

// regularize_adaptive's graph: the first iteration, then iterations 1 ..
// max_iters - 1 each inside an IF conditional node whose condition the
// previous iteration's check kernel sets (default 0 at every launch), so the
// number of iterations is bounded by construction; the way back to the
// caller's order runs after them in any case.
dc_status capture_adaptive(dc_ctx *c, float *pos, int64_t n, int max_iters, cudaGraphExec_t *out)
{
    const bool reorder = c->p.keep_order == 0 && n > 0;
    float *ipos = reorder ? reinterpret_cast<float *>(c->spos) : pos;
    AdaptState *st = static_cast<AdaptState *>(c->adapt);
    double *cv = adapt_cv(c), *mv = adapt_move(c);
    unsigned *dmax = adapt_dmax(c);
    Recorder rec;
    DC_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaStream_t s = c->cap_stream;
    cudaGraph_t cg = nullptr;
    cudaStreamCaptureStatus cs;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, nullptr, nullptr, nullptr);
    std::vector<cudaGraphConditionalHandle> h((size_t)max_iters + 1, 0);
    for (int it = 1; it < max_iters && e == cudaSuccess; ++it)
        e = cudaGraphConditionalHandleCreate(&h[it], cg, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->qacc, 0, sizeof(unsigned long long) * 3 * (size_t)max_iters, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dmax, 0, sizeof(unsigned) * (size_t)max_iters, s);
    if (e == cudaSuccess) e = launch_adapt_start(s, st);
    if (e == cudaSuccess) e = enqueue_first_splat(c, s, pos, n, reorder, rec);
    if (e == cudaSuccess) e = enqueue_iteration(c, s, pos, ipos, n, 0, true, c->qacc, dmax, rec, nullptr, 0, reorder);
    if (e == cudaSuccess)
        e = launch_adapt_check(s, c->qacc, dmax, st, cv, mv, 0, c->g.log2N, h[1], max_iters > 1 ? 1 : 0);
    for (int it = 1; it < max_iters && e == cudaSuccess; ++it) {
        const cudaGraphNode_t *deps = nullptr;
        const cudaGraphEdgeData *edges = nullptr;
        size_t nd = 0;
        e = cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &deps, &edges, &nd);
        if (e != cudaSuccess) break;
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h[it];
        np.conditional.type = cudaGraphCondTypeIf;
        np.conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        e = cudaGraphAddNode(&node, cg, deps, edges, nd, &np);
        if (e != cudaSuccess) break;
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(c->cap_stream2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        cudaError_t eb = enqueue_iteration(c, c->cap_stream2, pos, ipos, n, it & 1, true, c->qacc + 3 * it,
                                           dmax + it, rec);
        if (eb == cudaSuccess)
            eb = launch_adapt_check(c->cap_stream2, c->qacc + 3 * it, dmax, st, cv, mv, it, c->g.log2N, h[it + 1],
                                    it + 1 < max_iters ? 1 : 0);
        cudaGraph_t body_out = nullptr;
        e = cudaStreamEndCapture(c->cap_stream2, &body_out);
        if (eb != cudaSuccess) e = eb;
        if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    }
    if (e == cudaSuccess && reorder)
        e = launch_reorder_back(s, c->spos, c->inv, n, reinterpret_cast<float2 *>(pos), c->status);
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(s, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail(DC_ERR_CUDA, "adaptive graph capture: %s / %s", cudaGetErrorString(e), cudaGetErrorString(e2));
    }
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(DC_ERR_CUDA, "adaptive graph instantiate: %s", cudaGetErrorString(e));
    return DC_OK;
}

dc_status ensure_qslots(dc_ctx *c, int slots)
{
    if (slots <= c->qslots) return DC_OK;
    DC_CUDA(cudaStreamSynchronize(c->stream));
    if (c->qacc) cudaFree(c->qacc);
    c->qacc = nullptr;
    c->qslots = 0;
    if (cudaMalloc(&c->qacc, sizeof(unsigned long long) * 3 * (size_t)slots) != cudaSuccess) {
        cudaGetLastError();
        return fail(DC_ERR_OOM, "cannot allocate %d metric slots", slots);
    }
    c->qslots = slots;
    // graphs that recorded metrics point at the freed accumulators
    for (auto it = c->graphs.begin(); it != c->graphs.end();) {
        if (it->metrics) {
            cudaGraphExecDestroy(it->exec);
            it = c->graphs.erase(it);
        } else {
            ++it;
        }
    }
    return DC_OK;
}

void metrics_from_acc(const dc_ctx *c, const unsigned long long *acc, double *out3)
{
    const double B = (double)(c->g.N / 4);
    const double nbins = B * B;
    const double n = (double)acc[2];
    const double mean = n / nbins;
    double var = (double)acc[0] / nbins - mean * mean;
    if (var < 0.0) var = 0.0;
    const double sd = std::sqrt(var);
    out3[0] = sd;
    out3[1] = mean > 0.0 ? sd / mean : 0.0;
    out3[2] = n > 0.0 ? (n - (double)acc[1]) / n : 0.0;
}

dc_status check_ctx(const dc_ctx *c)
{
    if (!c) return fail(DC_ERR_INVALID_ARG, "null context");
    return DC_OK;
}

dc_status check_samples(const dc_ctx *, const void *pos, int64_t n)
{
    if (n < 0 || n >= (int64_t(1) << 32)) return fail(DC_ERR_INVALID_ARG, "n = %lld outside [0, 2^32)", (long long)n);
    if (n > 0 && !pos) return fail(DC_ERR_INVALID_ARG, "null sample pointer");
    if (n > 0 && !aligned(pos, 8)) return fail(DC_ERR_INVALID_ARG, "sample pointer not 8-byte aligned");
    return DC_OK;
}

const char *kKernelNames[DC_KERNEL_KINDS] = {"splat",  "smooth",  "band_aggregate", "band_carry", "band_final",
                                             "advect", "quality", "reorder",        "band_fused", "smooth_aggregate"};

}  // namespace

void dc::set_last_error(const char *msg) { g_last_error = msg ? msg : ""; }

dc_status dc::prepare_regularize(dc_ctx *c, int64_t n, int iters, int metrics)
{
    if (dc_status st = check_samples(c, reinterpret_cast<const void *>(16), n)) return st;
    if (metrics)
        if (dc_status st = ensure_qslots(c, iters)) return st;
    return ensure_sort_buffers(c, n);
}

cudaError_t dc::enqueue_regularize(dc_ctx *c, cudaStream_t s, float *pos, int64_t n, int iters, int metrics)
{
    Recorder rec;
    return enqueue_iterations(c, s, pos, n, iters, metrics, rec);
}

void dc::finish_regularize(dc_ctx *c, int64_t n, int iters, int metrics)
{
    c->n_last = n;
    c->have_disp = true;
    c->cur_counts = metrics ? (iters & 1) : ((iters - 1) & 1);
}

void dc::read_metrics(const dc_ctx *c, const unsigned long long *acc, double *out3) { metrics_from_acc(c, acc, out3); }

PanelDesc dc::panel_desc(const dc_ctx *c, float *pos, int64_t n)
{
    PanelDesc d{};
    d.pos = reinterpret_cast<float2 *>(pos);
    d.n = n;
    d.counts[0] = c->counts_buf[0];
    d.counts[1] = c->counts_buf[1];
    d.dens = c->dens;
    d.disp = c->disp;
    d.spos = c->spos;
    d.rank = c->rank;
    d.inv = c->inv;
    d.cursor = c->cursor;
    d.partials = c->partials;
    d.qacc = c->qacc;
    d.status = c->status;
    d.band = band_args(c, nullptr, c->mode, n);
    d.band.disp = c->disp;
    return d;
}

int dc::device_sms()
{
    constexpr int kMaxDev = 256;
    static std::atomic<int> cache[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        return 1;
    }
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
        cudaGetLastError();
        return 1;
    }
    cache[dev].store(v, std::memory_order_relaxed);
    return v;
}

extern "C" {

const char *declutter_status_string(dc_status s)
{
    switch (s) {
    case DC_OK: return "ok";
    case DC_ERR_INVALID_ARG: return "invalid argument";
    case DC_ERR_NOT_POW2: return "resolution must be 2^4 .. 2^13";
    case DC_ERR_OOM: return "out of device memory";
    case DC_ERR_CUDA: return "CUDA error";
    case DC_ERR_TIMEOUT: return "device wait timed out";
    case DC_ERR_RANGE: return "device range check failed";
    case DC_ERR_STATE: return "call out of order";
    }
    return "unknown status";
}

const char *declutter_last_error(void) { return g_last_error.c_str(); }

const char *declutter_kernel_name(int32_t k)
{
    return (k >= 0 && k < DC_KERNEL_KINDS) ? kKernelNames[k] : nullptr;
}

dc_status declutter_create(const dc_params *params, int device, void *cuda_stream, dc_ctx **out)
{
    if (!params || !out) return fail(DC_ERR_INVALID_ARG, "null params or out");
    *out = nullptr;
    const dc_params p = *params;
    if (p.log2_res < 4 || p.log2_res > 13) return fail(DC_ERR_NOT_POW2, "log2_res = %u", p.log2_res);
    if (p.reserved[0] != 0) return fail(DC_ERR_INVALID_ARG, "reserved fields must be zero");
    constexpr int kKnownOpts = DC_OPT_FUSED_BANDS | DC_OPT_SEPARATE_SMOOTH | DC_OPT_STAGE_HOST |
                               DC_OPT_BATCHED_LAUNCHES | DC_OPT_TEST_UNREACHED_BARRIER;
    if (p.options & ~kKnownOpts) return fail(DC_ERR_INVALID_ARG, "unknown options 0x%x", p.options & ~kKnownOpts);
    if (p.wait_limit_us < 0 || p.wait_limit_us > 10000000)
        return fail(DC_ERR_INVALID_ARG, "wait_limit_us = %d (0..10^7)", p.wait_limit_us);
    if (p.keep_order != 0 && p.keep_order != 1) return fail(DC_ERR_INVALID_ARG, "keep_order");
    const int N = 1 << p.log2_res;
    int r = p.kernel_r;
    if (r < 0) r = N / 128 < 2 ? 2 : N / 128;
    if (r > 64 || r >= N) return fail(DC_ERR_INVALID_ARG, "kernel_r = %d (max 64, < N)", r);
    // float (smoothed) mode keeps its 1e-4 px bound against FP64 only up to
    // 2048^2: above, the FP32 region sums alone err by about 2^-24 N / 2 px
    if (r > 0 && N > kFloatMaxN)
        return fail(DC_ERR_INVALID_ARG,
                    "float (smoothed) mode is limited to N <= %d (its FP32 sums miss the 1e-4 px bound above); "
                    "kernel_r = 0 gives the exact integer mode at any N",
                    kFloatMaxN);
    if (p.pixel_center != 0 && p.pixel_center != 1) return fail(DC_ERR_INVALID_ARG, "pixel_center");
    if (p.clamp_positions != 0 && p.clamp_positions != 1) return fail(DC_ERR_INVALID_ARG, "clamp_positions");
    if (p.carry_mode != DC_CARRY_COMPENSATED && p.carry_mode != DC_CARRY_F64)
        return fail(DC_ERR_INVALID_ARG, "carry_mode");
    if (p.band_rows != 0) {
        const int T = p.band_rows;
        if (T < 1 || T > 64 || T > N) return fail(DC_ERR_INVALID_ARG, "band_rows = %d", T);
    }
    if (!(p.sigma == p.sigma) || !(p.d0 == p.d0)) return fail(DC_ERR_INVALID_ARG, "NaN parameter");

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(DC_ERR_CUDA, "no CUDA device available");
    }
    if (device < 0 || device >= ndev) return fail(DC_ERR_INVALID_ARG, "device %d of %d", device, ndev);
    DeviceGuard guard(device);

    dc_ctx *c = new dc_ctx();
    c->p = p;
    c->device = device;
    c->r = r;
    c->mode = r > 0 ? MODE_FLOAT : MODE_COUNT;
    c->g = make_band_geom((int)p.log2_res, p.band_rows, device_sms());
    c->sigma = r > 0 ? (p.sigma > 0.f ? p.sigma : (float)r / 3.0f) : 0.f;
    if (r > 0) {
        double g[129], s = 0.0;
        const double sg = (double)c->sigma;
        for (int k = -r; k <= r; ++k) {
            g[k + r] = std::exp(-(double)k * (double)k / (2.0 * sg * sg));
            s += g[k + r];
        }
        for (int k = 0; k <= 2 * r; ++k) c->w.g[k] = (float)(g[k] / s);
    }
    c->w.r = r;

    auto bail = [&](dc_status st) {
        declutter_destroy(c);
        return st;
    };
    if (cuda_stream) {
        c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreate(&c->stream) != cudaSuccess) return bail(fail(DC_ERR_CUDA, "cudaStreamCreate"));
        c->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cap_stream2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(DC_ERR_CUDA, "cudaStreamCreateWithFlags"));
    if (cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(DC_ERR_CUDA, "cudaEventCreateWithFlags"));
    const size_t NN = (size_t)N * N;
    const size_t agg_bytes = (size_t)c->g.nb * c->g.agg_stride * 8;
    const size_t carry_bytes = (size_t)(c->g.nb + 1) * c->g.lanes * 8;
    struct {
        void **p;
        size_t bytes;
    } allocs[] = {
        {(void **)&c->counts_buf[0], NN * sizeof(uint32_t)},
        {(void **)&c->counts_buf[1], NN * sizeof(uint32_t)},
        {(void **)&c->disp, NN * sizeof(float2)},
        {&c->agg, agg_bytes},
        {&c->carry, carry_bytes},
        {(void **)&c->status, 256},
        {(void **)&c->cursor, NN * sizeof(uint32_t)},
        {(void **)&c->partials, 1024 * sizeof(uint32_t)},
    };
    for (auto &al : allocs) {
        if (cudaMalloc(al.p, al.bytes) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(DC_ERR_OOM, "cudaMalloc(%zu)", al.bytes));
        }
        c->scratch_bytes += (int64_t)al.bytes;
    }
    if (c->mode == MODE_FLOAT) {
        if (cudaMalloc(&c->dens, NN * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(DC_ERR_OOM, "cudaMalloc density"));
        }
        c->scratch_bytes += (int64_t)(NN * sizeof(float));
    }
    if (ensure_qslots(c, 1) != DC_OK) return bail(DC_ERR_OOM);
    if (cudaMemset(c->status, 0, 256) != cudaSuccess) return bail(fail(DC_ERR_CUDA, "cudaMemset status"));
    if (cudaMallocHost(&c->status_host, sizeof(unsigned)) != cudaSuccess) {
        c->status_host = nullptr;
        return bail(fail(DC_ERR_OOM, "pinned status word"));
    }
    if (prepare_kernels() != cudaSuccess) return bail(fail(DC_ERR_CUDA, "kernel attributes"));
    // DC_OPT_FUSED_BANDS: the three band phases as one cooperative launch on
    // small grids (measured slower than three launches at 512^2)
    c->fused = (p.options & DC_OPT_FUSED_BANDS) && band_fused_available(c->g, c->mode, c->p.carry_mode, c->device);
    // the smoothing runs inside the aggregate pass where it fits
    // (DC_OPT_SEPARATE_SMOOTH: separate launches, the same bits)
    c->smooth_agg = !(p.options & DC_OPT_SEPARATE_SMOOTH) && !c->fused && c->mode == MODE_FLOAT &&
                    smooth_agg_available(c->g, c->w);
    *out = c;
    return DC_OK;
}

dc_status declutter_destroy(dc_ctx *c)
{
    if (!c) return DC_OK;
    DeviceGuard guard(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto &ge : c->graphs)
        if (ge.exec) cudaGraphExecDestroy(ge.exec);
    for (int k = 0; k < 2; ++k)
        if (c->prof_ev[k]) cudaEventDestroy(c->prof_ev[k]);
    cudaFree(c->counts_buf[0]);
    cudaFree(c->counts_buf[1]);
    cudaFree(c->dens);
    cudaFree(c->disp);
    cudaFree(c->agg);
    cudaFree(c->carry);
    cudaFree(c->status);
    if (c->status_host) cudaFreeHost(c->status_host);
    cudaFree(c->qacc);
    cudaFree(c->hpos);
    cudaFree(c->spos);
    cudaFree(c->rank);
    cudaFree(c->inv);
    cudaFree(c->cursor);
    cudaFree(c->partials);
    cudaFree(c->adapt);
    cudaFree(c->lq);
    cudaFree(c->lterms);
    cudaFree(c->wcover);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->cap_stream2) cudaStreamDestroy(c->cap_stream2);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return DC_OK;
}

dc_status declutter_get_info(const dc_ctx *c, dc_info *out)
{
    if (check_ctx(c) != DC_OK || !out) return fail(DC_ERR_INVALID_ARG, "null argument");
    out->N = c->g.N;
    out->kernel_r = c->r;
    out->sigma = c->sigma;
    out->band_rows = c->g.T;
    out->n_bands = c->g.nb;
    out->band_threads = c->g.NT;
    out->kernels_per_iter = c->mode == MODE_FLOAT ? 5 : 4;  // after the first, which adds a splat
    out->device = c->device;
    out->scratch_bytes = c->scratch_bytes;
    return DC_OK;
}

dc_status splat_density(dc_ctx *c, const float *pos, int64_t n, uint32_t *counts_out, float *density_out)
{
    if (dc_status st = check_ctx(c)) return st;
    if (dc_status st = check_samples(c, pos, n)) return st;
    if (density_out && c->mode != MODE_FLOAT) return fail(DC_ERR_INVALID_ARG, "no density in exact mode");
    DeviceGuard guard(c->device);
    Recorder rec;
    DC_CUDA(enqueue_density(c, c->stream, pos, n, c->counts_buf[0], nullptr, rec));
    c->cur_counts = 0;
    const size_t NN = (size_t)c->g.N * c->g.N;
    if (counts_out) DC_CUDA(cudaMemcpyAsync(counts_out, c->counts_buf[0], NN * 4, cudaMemcpyDeviceToDevice, c->stream));
    if (density_out) DC_CUDA(cudaMemcpyAsync(density_out, c->dens, NN * 4, cudaMemcpyDeviceToDevice, c->stream));
    c->n_last = n;
    c->have_disp = false;
    return DC_OK;
}

dc_status splat_counts(dc_ctx *c, const float *pos, int64_t n, uint32_t *counts_out)
{
    if (dc_status st = check_ctx(c)) return st;
    if (dc_status st = check_samples(c, pos, n)) return st;
    if (!counts_out || !aligned(counts_out, 16)) return fail(DC_ERR_INVALID_ARG, "counts_out null or misaligned");
    DeviceGuard guard(c->device);
    DC_CUDA(cudaMemsetAsync(counts_out, 0, sizeof(uint32_t) * (size_t)c->g.N * c->g.N, c->stream));
    DC_CUDA(launch_splat(c->stream, reinterpret_cast<const float2 *>(pos), n, counts_out, c->g.log2N));
    return DC_OK;
}

dc_status density_from_counts(dc_ctx *c, const uint32_t *counts, int64_t n)
{
    if (dc_status st = check_ctx(c)) return st;
    if (!counts || !aligned(counts, 16)) return fail(DC_ERR_INVALID_ARG, "counts null or misaligned");
    if (n < 0 || n >= (int64_t(1) << 32)) return fail(DC_ERR_INVALID_ARG, "n = %lld", (long long)n);
    DeviceGuard guard(c->device);
    const size_t NN = (size_t)c->g.N * c->g.N;
    DC_CUDA(cudaMemcpyAsync(c->counts_buf[0], counts, NN * 4, cudaMemcpyDeviceToDevice, c->stream));
    if (c->mode == MODE_FLOAT) DC_CUDA(launch_smooth(c->stream, c->counts_buf[0], c->dens, c->g.log2N, c->w, nullptr));
    c->cur_counts = 0;
    c->n_last = n;
    c->have_disp = false;
    return DC_OK;
}

dc_status integral_images(dc_ctx *c, void *alpha_out, void *alpha_t_out)
{
    if (dc_status st = check_ctx(c)) return st;
    if (c->n_last < 0) return fail(DC_ERR_STATE, "integral_images before splat_density");
    if ((alpha_out && !aligned(alpha_out, 16)) || (alpha_t_out && !aligned(alpha_t_out, 16)))
        return fail(DC_ERR_INVALID_ARG, "outputs must be 16-byte aligned");
    DeviceGuard guard(c->device);
    const void *src = c->mode == MODE_FLOAT ? (const void *)c->dens : (const void *)c->counts_buf[c->cur_counts];
    BandArgs a = band_args(c, src, c->mode, c->n_last);
    a.alpha_out = alpha_out;
    a.alpha_t_out = alpha_t_out;
    Recorder rec;
    DC_CUDA(enqueue_inims(c, c->stream, a, c->mode, rec));
    return DC_OK;
}

dc_status integral_images_u32(dc_ctx *c, const uint32_t *grid, uint64_t *alpha_out, uint64_t *alpha_t_out)
{
    if (dc_status st = check_ctx(c)) return st;
    if (!grid || !aligned(grid, 16)) return fail(DC_ERR_INVALID_ARG, "grid null or not 16-byte aligned");
    if ((alpha_out && !aligned(alpha_out, 16)) || (alpha_t_out && !aligned(alpha_t_out, 16)))
        return fail(DC_ERR_INVALID_ARG, "outputs must be 16-byte aligned");
    DeviceGuard guard(c->device);
    BandArgs a = band_args(c, grid, MODE_GRID64, 0);
    a.alpha_out = alpha_out;
    a.alpha_t_out = alpha_t_out;
    Recorder rec;
    DC_CUDA(enqueue_inims(c, c->stream, a, MODE_GRID64, rec));
    return DC_OK;
}

dc_status displacement_field(dc_ctx *c, float *disp_out)
{
    if (dc_status st = check_ctx(c)) return st;
    if (c->n_last < 0) return fail(DC_ERR_STATE, "displacement_field before splat_density");
    if (disp_out && !aligned(disp_out, 16)) return fail(DC_ERR_INVALID_ARG, "output must be 16-byte aligned");
    DeviceGuard guard(c->device);
    const void *src = c->mode == MODE_FLOAT ? (const void *)c->dens : (const void *)c->counts_buf[c->cur_counts];
    BandArgs a = band_args(c, src, c->mode, c->n_last);
    a.disp = c->disp;
    Recorder rec;
    DC_CUDA(enqueue_inims(c, c->stream, a, c->mode, rec));
    if (disp_out)
        DC_CUDA(cudaMemcpyAsync(disp_out, c->disp, sizeof(float2) * (size_t)c->g.N * c->g.N,
                                cudaMemcpyDeviceToDevice, c->stream));
    c->have_disp = true;
    return DC_OK;
}

dc_status lens_field(dc_ctx *c, const float *density, float density_mean, float *disp_out)
{
    if (dc_status st = check_ctx(c)) return st;
    if (!density) return fail(DC_ERR_INVALID_ARG, "null density");
    if (!aligned(density, 16)) return fail(DC_ERR_INVALID_ARG, "density must be 16-byte aligned");
    if (disp_out && !aligned(disp_out, 16)) return fail(DC_ERR_INVALID_ARG, "output must be 16-byte aligned");
    if (!(density_mean >= 0.f) || !std::isfinite(density_mean))
        return fail(DC_ERR_INVALID_ARG, "density_mean = %g", (double)density_mean);
    if (c->g.N > kFloatMaxN) return fail(DC_ERR_INVALID_ARG, "lens_field runs the float passes: N <= %d", kFloatMaxN);
    DeviceGuard guard(c->device);
    // float-mode band passes over the caller's grid; mu = the mean hint only
    // centres the sums (any constant gives the same mapping), d0 = 0
    BandArgs a = band_args(c, density, MODE_FLOAT, 0);
    a.mu = density_mean;
    a.d0 = 0.f;
    a.lens = 1;
    a.disp = c->disp;
    Recorder rec;
    DC_CUDA(enqueue_inims(c, c->stream, a, MODE_FLOAT, rec));
    if (disp_out)
        DC_CUDA(cudaMemcpyAsync(disp_out, c->disp, sizeof(float2) * (size_t)c->g.N * c->g.N,
                                cudaMemcpyDeviceToDevice, c->stream));
    c->have_disp = true;
    return DC_OK;
}

dc_status contour_segments(dc_ctx *c, const float *field, float level, float *segs_out)
{
    if (dc_status st = check_ctx(c)) return st;
    if (!field || !segs_out) return fail(DC_ERR_INVALID_ARG, "null field or output");
    if (!aligned(field, 4)) return fail(DC_ERR_INVALID_ARG, "field must be 4-byte aligned");
    if (!aligned(segs_out, 16)) return fail(DC_ERR_INVALID_ARG, "output must be 16-byte aligned");
    if (!std::isfinite(level)) return fail(DC_ERR_INVALID_ARG, "level = %g", (double)level);
    DeviceGuard guard(c->device);
    DC_CUDA(launch_contour(c->stream, field, c->g.log2N, level, c->p.pixel_center,
                           reinterpret_cast<float4 *>(segs_out)));
    return DC_OK;
}

dc_status advect_samples(dc_ctx *c, float *pos, int64_t n)
{
    if (dc_status st = check_ctx(c)) return st;
    if (dc_status st = check_samples(c, pos, n)) return st;
    if (!c->have_disp) return fail(DC_ERR_STATE, "advect_samples before displacement_field");
    DeviceGuard guard(c->device);
    DC_CUDA(launch_advect(c->stream, reinterpret_cast<float2 *>(pos), n, c->disp, c->g.log2N, c->p.pixel_center,
                          c->p.clamp_positions, nullptr));
    return DC_OK;
}

dc_status declutter_sync(dc_ctx *c)
{
    if (dc_status st = check_ctx(c)) return st;
    DeviceGuard guard(c->device);
    // the status word comes back with the same synchronisation
    DC_CUDA(cudaMemcpyAsync(c->status_host, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    DC_CUDA(cudaStreamSynchronize(c->stream));
    const unsigned st = *c->status_host;
    if (st != 0) {
        cudaMemset(c->status, 0, 256);  // the status word and the grid-barrier words
        return fail((dc_status)st, "device status %u", st);
    }
    return DC_OK;
}

dc_status regularize(dc_ctx *c, float *pos, int64_t n, int32_t iters, double *uniformity_out)
{
    if (dc_status st = check_ctx(c)) return st;
    if (dc_status st = check_samples(c, pos, n)) return st;
    if (iters < 0) return fail(DC_ERR_INVALID_ARG, "iters = %d", iters);
    if (iters == 0) return DC_OK;
    DeviceGuard guard(c->device);
    const int metrics = uniformity_out ? 1 : 0;
    if (metrics)
        if (dc_status st = ensure_qslots(c, iters)) return st;
    if (dc_status st = ensure_sort_buffers(c, n)) return st;
    cudaGraphExec_t exec = nullptr;
    for (auto &ge : c->graphs)
        if (ge.pos == pos && ge.n == n && ge.iters == iters && ge.metrics == metrics && !ge.adaptive) exec = ge.exec;
    if (!exec) {
        if (c->graphs.size() >= 16) {
            cudaGraphExecDestroy(c->graphs.front().exec);
            c->graphs.erase(c->graphs.begin());
        }
        if (dc_status st = capture_iterations(c, pos, n, iters, metrics, -1, &exec, nullptr)) return st;
        GraphEntry ge;
        ge.pos = pos;
        ge.n = n;
        ge.iters = iters;
        ge.metrics = metrics;
        ge.exec = exec;
        c->graphs.push_back(ge);
    }
    DC_CUDA(cudaGraphLaunch(exec, c->stream));
    c->n_last = n;
    c->have_disp = true;
    c->cur_counts = metrics ? (iters & 1) : ((iters - 1) & 1);  // grid of the last splat performed
    if (metrics) {
        std::vector<unsigned long long> acc(3 * (size_t)iters);
        DC_CUDA(cudaMemcpyAsync(acc.data(), c->qacc, acc.size() * sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, c->stream));
        if (dc_status st = declutter_sync(c)) return st;
        for (int it = 0; it < iters; ++it) {
            double m[3];
            metrics_from_acc(c, &acc[3 * (size_t)it], m);
            uniformity_out[it] = m[0];
        }
    }
    return DC_OK;
}

dc_status regularize_tracers(dc_ctx *c, float *pos, int64_t n, float *tracer_xy, int64_t n_tracers, int32_t iters)
{
    if (dc_status st = check_ctx(c)) return st;
    if (dc_status st = check_samples(c, pos, n)) return st;
    if (dc_status st = check_samples(c, tracer_xy, n_tracers)) return st;
    if (iters < 0) return fail(DC_ERR_INVALID_ARG, "iters = %d", iters);
    if (iters == 0) return DC_OK;
    DeviceGuard guard(c->device);
    if (dc_status st = ensure_sort_buffers(c, n)) return st;
    Recorder rec;
    DC_CUDA(enqueue_iterations(c, c->stream, pos, n, iters, 0, rec, tracer_xy, n_tracers));
    c->n_last = n;
    c->have_disp = true;
    c->cur_counts = (iters - 1) & 1;
    return DC_OK;
}

// Device address of host memory the device can reach directly (pinned or
// registered under unified addressing), 8-byte aligned; else null.
static float *device_alias(float *host_pos)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, host_pos) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
    float *dp = static_cast<float *>(at.devicePointer);
    return (reinterpret_cast<uintptr_t>(dp) & 7) ? nullptr : dp;
}

dc_status regularize_host(dc_ctx *c, float *host_pos, int64_t n, int32_t iters, double *uniformity_out)
{
    if (dc_status st = check_ctx(c)) return st;
    if (n < 0 || n >= (int64_t(1) << 32)) return fail(DC_ERR_INVALID_ARG, "n");
    if (n > 0 && !host_pos) return fail(DC_ERR_INVALID_ARG, "null host pointer");
    DeviceGuard guard(c->device);
    // Pinned (or registered) host memory is addressable by the device: with
    // the samples reordered, the iterations touch the caller's array only in
    // the first splat (one read, leaving a device copy for the reordering)
    // and in the way back (one write), so they run on it directly over the
    // host link, without staging copies (DC_OPT_STAGE_HOST: always stage).
    // the device buffer hpos: the staged copy, or the splat's copy of
    // samples used in place; cached graphs hold its address, so they are
    // dropped when it moves
    if (n > c->hpos_cap) {
        DC_CUDA(cudaStreamSynchronize(c->stream));
        for (auto &ge : c->graphs) cudaGraphExecDestroy(ge.exec);
        c->graphs.clear();
        cudaFree(c->hpos);
        c->hpos = nullptr;
        c->hpos_cap = 0;
        if (cudaMalloc(&c->hpos, sizeof(float) * 2 * (size_t)n) != cudaSuccess) {
            cudaGetLastError();
            return fail(DC_ERR_OOM, "staging buffer");
        }
        c->hpos_cap = n;
    }
    if (n > 0 && c->p.keep_order == 0 && !(c->p.options & DC_OPT_STAGE_HOST))
        if (float *dp = device_alias(host_pos)) {
            c->copy_first = true;
            const dc_status st = regularize(c, dp, n, iters, uniformity_out);
            c->copy_first = false;
            if (st != DC_OK) return st;
            return declutter_sync(c);
        }
    const size_t bytes = sizeof(float) * 2 * (size_t)n;
    if (n > 0) DC_CUDA(cudaMemcpyAsync(c->hpos, host_pos, bytes, cudaMemcpyHostToDevice, c->stream));
    if (dc_status st = regularize(c, c->hpos, n, iters, uniformity_out)) return st;
    if (n > 0) DC_CUDA(cudaMemcpyAsync(host_pos, c->hpos, bytes, cudaMemcpyDeviceToHost, c->stream));
    return declutter_sync(c);
}

dc_status regularize_adaptive(dc_ctx *c, float *pos, int64_t n, int32_t max_iters, double target_cv,
                              double min_move_px, double max_ms, int32_t *iters_out, double *cv_out,
                              double *move_px_out)
{
    if (dc_status st = check_ctx(c)) return st;
    if (dc_status st = check_samples(c, pos, n)) return st;
    if (max_iters < 1 || max_iters > 1024) return fail(DC_ERR_INVALID_ARG, "max_iters = %d (1..1024)", max_iters);
    if (!(target_cv >= 0.0) || !(min_move_px >= 0.0) || !(max_ms >= 0.0) || !std::isfinite(target_cv) ||
        !std::isfinite(min_move_px) || !std::isfinite(max_ms))
        return fail(DC_ERR_INVALID_ARG, "criteria must be finite and >= 0");
    if (n == 0) return fail(DC_ERR_INVALID_ARG, "no samples");
    DeviceGuard guard(c->device);
    if (dc_status st = ensure_qslots(c, max_iters)) return st;
    if (dc_status st = ensure_adapt(c, max_iters)) return st;
    if (dc_status st = ensure_sort_buffers(c, n)) return st;
    cudaGraphExec_t exec = nullptr;
    for (auto &ge : c->graphs)
        if (ge.adaptive && ge.pos == pos && ge.n == n && ge.iters == max_iters) exec = ge.exec;
    if (!exec) {
        if (c->graphs.size() >= 16) {
            cudaGraphExecDestroy(c->graphs.front().exec);
            c->graphs.erase(c->graphs.begin());
        }
        if (dc_status st = capture_adaptive(c, pos, n, max_iters, &exec)) return st;
        GraphEntry ge;
        ge.pos = pos;
        ge.n = n;
        ge.iters = max_iters;
        ge.metrics = 1;
        ge.adaptive = 1;
        ge.exec = exec;
        c->graphs.push_back(ge);
    }
    AdaptState hs{};
    hs.target_cv = target_cv;
    hs.min_move_px = min_move_px;
    hs.max_ns = max_ms * 1e6;
    DC_CUDA(cudaMemcpyAsync(c->adapt, &hs, sizeof(hs), cudaMemcpyHostToDevice, c->stream));
    DC_CUDA(cudaGraphLaunch(exec, c->stream));
    std::vector<double> cvs((size_t)max_iters), mvs((size_t)max_iters);
    DC_CUDA(cudaMemcpyAsync(&hs, c->adapt, sizeof(hs), cudaMemcpyDeviceToHost, c->stream));
    DC_CUDA(cudaMemcpyAsync(cvs.data(), adapt_cv(c), sizeof(double) * max_iters, cudaMemcpyDeviceToHost, c->stream));
    DC_CUDA(cudaMemcpyAsync(mvs.data(), adapt_move(c), sizeof(double) * max_iters, cudaMemcpyDeviceToHost, c->stream));
    const dc_status st = declutter_sync(c);
    const int done = hs.iters;
    c->n_last = n;
    c->have_disp = true;
    c->cur_counts = done & 1;  // every iteration splatted its moved samples
    if (st != DC_OK) return st;
    if (done < 1 || done > max_iters) return fail(DC_ERR_RANGE, "iterations done = %d", done);
    if (iters_out) *iters_out = done;
    for (int k = 0; k < done; ++k) {
        if (cv_out) cv_out[k] = cvs[k];
        if (move_px_out) move_px_out[k] = mvs[k];
    }
    return DC_OK;
}

dc_status transition_positions(dc_ctx *c, const float *from_xy, const float *to_xy, int64_t n, float s,
                               float *out_xy)
{
    if (dc_status st = check_ctx(c)) return st;
    if (dc_status st = check_samples(c, from_xy, n)) return st;
    if (dc_status st = check_samples(c, to_xy, n)) return st;
    if (dc_status st = check_samples(c, out_xy, n)) return st;
    if (!(s >= 0.0f && s <= 1.0f)) return fail(DC_ERR_INVALID_ARG, "s = %g outside [0, 1]", (double)s);
    DeviceGuard guard(c->device);
    DC_CUDA(launch_transition(c->stream, from_xy, to_xy, 2 * n, s, out_xy));
    return DC_OK;
}

dc_status layout_metrics(dc_ctx *c, const float *orig_xy, const float *reg_xy, int64_t n, const uint32_t *queries,
                         int32_t n_queries, int32_t k, double *out, int64_t *terms_out)
{
    if (dc_status st = check_ctx(c)) return st;
    if (dc_status st = check_samples(c, orig_xy, n)) return st;
    if (dc_status st = check_samples(c, reg_xy, n)) return st;
    if (!out) return fail(DC_ERR_INVALID_ARG, "null out");
    if (n >= (int64_t(1) << 31)) return fail(DC_ERR_INVALID_ARG, "n = %lld (< 2^31)", (long long)n);
    if (k < 1 || k > 32 || 2 * (int64_t)k >= n)
        return fail(DC_ERR_INVALID_ARG, "k = %d (1..32, k < n / 2)", k);
    if (n_queries < 1 || n_queries > (1 << 24) || (!queries && n_queries > n))
        return fail(DC_ERR_INVALID_ARG, "n_queries = %d", n_queries);
    if (queries && !aligned(queries, 4)) return fail(DC_ERR_INVALID_ARG, "queries not 4-byte aligned");
    DeviceGuard guard(c->device);
    if (n > c->lq_cap || n_queries > c->lterms_cap) {
        DC_CUDA(cudaStreamSynchronize(c->stream));
        if (n > c->lq_cap) {
            cudaFree(c->lq);
            c->lq = nullptr;
            c->lq_cap = 0;
            if (cudaMalloc(&c->lq, sizeof(uint32_t) * 2 * (size_t)n) != cudaSuccess) {
                cudaGetLastError();
                return fail(DC_ERR_OOM, "layout scratch");
            }
            c->lq_cap = n;
        }
        if (n_queries > c->lterms_cap) {
            cudaFree(c->lterms);
            c->lterms = nullptr;
            c->lterms_cap = 0;
            if (cudaMalloc(&c->lterms, sizeof(long long) * 2 * (size_t)n_queries) != cudaSuccess) {
                cudaGetLastError();
                return fail(DC_ERR_OOM, "layout terms");
            }
            c->lterms_cap = n_queries;
        }
    }
    DC_CUDA(launch_layout_terms(c->stream, reinterpret_cast<const float2 *>(orig_xy),
                                reinterpret_cast<const float2 *>(reg_xy), n, queries, n_queries, k, c->lq,
                                c->lq + n, c->lterms));
    std::vector<long long> terms(2 * (size_t)n_queries);
    DC_CUDA(cudaMemcpyAsync(terms.data(), c->lterms, sizeof(long long) * terms.size(), cudaMemcpyDeviceToHost,
                            c->stream));
    if (dc_status st = declutter_sync(c)) return st;
    double tsum = 0.0, osum = 0.0;
    for (int q = 0; q < n_queries; ++q) {
        if (terms[2 * (size_t)q] < 0) return fail(DC_ERR_RANGE, "query %d: index outside [0, n)", q);
        tsum += (double)terms[2 * (size_t)q];
        osum += (double)terms[2 * (size_t)q + 1];
    }
    if (terms_out)
        for (size_t q = 0; q < terms.size(); ++q) terms_out[q] = (int64_t)terms[q];
    const double m = (double)n_queries, nn = (double)n, kk = (double)k;
    out[0] = 1.0 - 2.0 / (m * kk * (2.0 * nn - 3.0 * kk - 1.0)) * tsum;
    out[1] = 1.0 - osum / (m * (nn - 1.0));
    return DC_OK;
}

dc_status warp_texture(dc_ctx *c, const float *nodes_xy, const float *texture, int32_t out_log2, int32_t mode,
                       float *out, int32_t *tri_out)
{
    if (dc_status st = check_ctx(c)) return st;
    if (!nodes_xy || !texture || !out) return fail(DC_ERR_INVALID_ARG, "null nodes, texture or output");
    if (!aligned(nodes_xy, 8) || !aligned(texture, 4) || !aligned(out, 4) || (tri_out && !aligned(tri_out, 4)))
        return fail(DC_ERR_INVALID_ARG, "misaligned pointer");
    if (out_log2 < 4 || out_log2 > 13) return fail(DC_ERR_INVALID_ARG, "out_log2 = %d (4..13)", out_log2);
    if (mode != DC_WARP_VALUE && mode != DC_WARP_MASS) return fail(DC_ERR_INVALID_ARG, "mode = %d", mode);
    DeviceGuard guard(c->device);
    const int64_t MM = (int64_t)1 << (2 * out_log2);
    uint32_t *cover = reinterpret_cast<uint32_t *>(tri_out);
    if (!cover) {
        if (MM > c->wcover_cap) {
            DC_CUDA(cudaStreamSynchronize(c->stream));
            cudaFree(c->wcover);
            c->wcover = nullptr;
            c->wcover_cap = 0;
            if (cudaMalloc(&c->wcover, sizeof(uint32_t) * (size_t)MM) != cudaSuccess) {
                cudaGetLastError();
                return fail(DC_ERR_OOM, "coverage scratch");
            }
            c->wcover_cap = MM;
        }
        cover = c->wcover;
    }
    DC_CUDA(launch_warp_texture(c->stream, reinterpret_cast<const float2 *>(nodes_xy), texture, c->g.log2N, out_log2,
                                mode == DC_WARP_MASS, cover, out));
    return DC_OK;
}

dc_status transfer_function(dc_ctx *c, const float *values, int64_t count, float lo, float hi, const uint32_t *lut,
                            uint32_t *rgba_out)
{
    if (dc_status st = check_ctx(c)) return st;
    if (count < 0) return fail(DC_ERR_INVALID_ARG, "count = %lld", (long long)count);
    if (count > 0 && (!values || !lut || !rgba_out)) return fail(DC_ERR_INVALID_ARG, "null pointer");
    if (!aligned(values, 4) || !aligned(lut, 4) || !aligned(rgba_out, 4))
        return fail(DC_ERR_INVALID_ARG, "misaligned pointer");
    if (!std::isfinite(lo) || !std::isfinite(hi) || !(hi > lo)) return fail(DC_ERR_INVALID_ARG, "need lo < hi, finite");
    DeviceGuard guard(c->device);
    DC_CUDA(launch_transfer(c->stream, values, count, lo, hi, lut, rgba_out));
    return DC_OK;
}

dc_status declutter_counts(dc_ctx *c, uint32_t *counts_out)
{
    if (dc_status st = check_ctx(c)) return st;
    if (!counts_out || !aligned(counts_out, 4)) return fail(DC_ERR_INVALID_ARG, "counts_out null or misaligned");
    if (c->n_last < 0) return fail(DC_ERR_STATE, "declutter_counts before any splat");
    DeviceGuard guard(c->device);
    DC_CUDA(cudaMemcpyAsync(counts_out, c->counts_buf[c->cur_counts], sizeof(uint32_t) * (size_t)c->g.N * c->g.N,
                            cudaMemcpyDeviceToDevice, c->stream));
    return DC_OK;
}

dc_status quality_metrics(dc_ctx *c, double *out)
{
    if (dc_status st = check_ctx(c)) return st;
    if (!out) return fail(DC_ERR_INVALID_ARG, "null out");
    if (c->n_last < 0) return fail(DC_ERR_STATE, "quality_metrics before splat_density");
    DeviceGuard guard(c->device);
    unsigned long long acc[3];
    DC_CUDA(cudaMemsetAsync(c->qacc, 0, sizeof(acc), c->stream));
    DC_CUDA(launch_quality(c->stream, c->counts_buf[c->cur_counts], c->g.log2N, c->qacc));
    DC_CUDA(cudaMemcpyAsync(acc, c->qacc, sizeof(acc), cudaMemcpyDeviceToHost, c->stream));
    if (dc_status st = declutter_sync(c)) return st;
    metrics_from_acc(c, acc, out);
    return DC_OK;
}

dc_status declutter_profile_regularize(dc_ctx *c, float *pos, const float *reset_src, int64_t n, int32_t iters,
                                       int32_t reps, float *step_ms_out, float *kernel_ms_out,
                                       int32_t *launches_out)
{
    if (dc_status st = check_ctx(c)) return st;
    if (dc_status st = check_samples(c, pos, n)) return st;
    if (iters < 1 || reps < 1) return fail(DC_ERR_INVALID_ARG, "iters = %d, reps = %d", iters, reps);
    if (reset_src && !aligned(reset_src, 8)) return fail(DC_ERR_INVALID_ARG, "reset_src alignment");
    DeviceGuard guard(c->device);
    if (dc_status st = ensure_sort_buffers(c, n)) return st;
    if (!c->prof_ev[0])
        for (int k = 0; k < 2; ++k) DC_CUDA(cudaEventCreate(&c->prof_ev[k]));
    const size_t bytes = sizeof(float) * 2 * (size_t)n;
    float base_ms = 0.f;
    float kernel_ms[DC_KERNEL_KINDS] = {};
    int32_t launches[DC_KERNEL_KINDS] = {};
    // dup = -1 first: the plain step; then each kind launched twice
    for (int dup = -1; dup < DC_KERNEL_KINDS; ++dup) {
        if (dup >= 0 && launches[dup] == 0) continue;
        cudaGraphExec_t exec = nullptr;
        Recorder rec;
        if (dc_status st = capture_iterations(c, pos, n, iters, 0, dup, &exec, &rec)) return st;
        if (dup < 0) std::memcpy(launches, rec.launches, sizeof(launches));
        float total = 0.f;
        cudaError_t e = cudaSuccess;
        for (int r = -2; r < reps && e == cudaSuccess; ++r) {  // two untimed warm-up runs
            if (reset_src && n > 0)
                e = cudaMemcpyAsync(pos, reset_src, bytes, cudaMemcpyDeviceToDevice, c->stream);
            if (e == cudaSuccess) e = cudaEventRecord(c->prof_ev[0], c->stream);
            if (e == cudaSuccess) e = cudaGraphLaunch(exec, c->stream);
            if (e == cudaSuccess) e = cudaEventRecord(c->prof_ev[1], c->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(c->prof_ev[1]);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, c->prof_ev[0], c->prof_ev[1]);
            if (r >= 0) total += t;
        }
        cudaGraphExecDestroy(exec);
        if (e != cudaSuccess) return fail(DC_ERR_CUDA, "profiling run: %s", cudaGetErrorString(e));
        const float ms = total / reps;
        if (dup < 0) base_ms = ms;
        else kernel_ms[dup] = ms > base_ms ? ms - base_ms : 0.f;
    }
    c->n_last = n;
    c->have_disp = true;
    c->cur_counts = (iters - 1) & 1;
    if (step_ms_out) *step_ms_out = base_ms;
    if (kernel_ms_out) std::memcpy(kernel_ms_out, kernel_ms, sizeof(kernel_ms));
    if (launches_out) std::memcpy(launches_out, launches, sizeof(launches));
    return declutter_sync(c);
}

}  // extern "C"
