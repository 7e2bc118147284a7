// C ABI and runtime of libdeclutter: context, buffers, streams, CUDA-graph
// capture of the iteration, instrumentation, error reporting.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "dc_internal.cuh"

using namespace dc;

namespace {

thread_local std::string g_last_error;

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

// Records (kind, start, end) event pairs around launches when profiling.
struct Recorder {
    dc_ctx *ctx = nullptr;
    int used = 0;
    int kinds[64];
    bool overflow = false;
    void before(cudaStream_t s, int kind)
    {
        if (!ctx) return;
        if (used >= 64) { overflow = true; return; }
        kinds[used] = kind;
        cudaEventRecord(ctx->prof_ev[2 * used], s);
    }
    void after(cudaStream_t s)
    {
        if (!ctx || overflow) return;
        cudaEventRecord(ctx->prof_ev[2 * used + 1], s);
        ++used;
    }
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
    return a;
}

cudaError_t enqueue_density(dc_ctx *c, cudaStream_t s, const float *pos, int64_t n, Recorder &rec)
{
    cudaError_t e;
    rec.before(s, K_MEMSET);
    e = cudaMemsetAsync(c->counts, 0, sizeof(uint32_t) * (size_t)c->g.N * c->g.N, s);
    rec.after(s);
    if (e != cudaSuccess) return e;
    rec.before(s, K_SPLAT);
    e = launch_splat(s, reinterpret_cast<const float2 *>(pos), n, c->counts, c->g.log2N);
    rec.after(s);
    if (e != cudaSuccess) return e;
    if (c->mode == MODE_FLOAT) {
        rec.before(s, K_SMOOTH);
        e = launch_smooth(s, c->counts, c->dens, c->g.log2N, c->w);
        rec.after(s);
    }
    return e;
}

cudaError_t enqueue_inims(dc_ctx *c, cudaStream_t s, const BandArgs &a, int mode, Recorder &rec)
{
    cudaError_t e;
    rec.before(s, K_BAND_AGG);
    e = launch_band_agg(s, c->g, mode, a);
    rec.after(s);
    if (e != cudaSuccess) return e;
    rec.before(s, K_CARRY);
    e = launch_carry(s, c->g, mode, c->p.carry_mode, c->agg, c->carry);
    rec.after(s);
    if (e != cudaSuccess) return e;
    rec.before(s, K_BAND_FINAL);
    e = launch_band_final(s, c->g, mode, a);
    rec.after(s);
    return e;
}

cudaError_t enqueue_iterations(dc_ctx *c, cudaStream_t s, float *pos, int64_t n, int iters, int metrics,
                               Recorder &rec)
{
    cudaError_t e = cudaSuccess;
    const void *src = c->mode == MODE_FLOAT ? (const void *)c->dens : (const void *)c->counts;
    BandArgs a = band_args(c, src, c->mode, n);
    a.disp = c->disp;
    if (metrics) {
        e = cudaMemsetAsync(c->qacc, 0, sizeof(unsigned long long) * 3 * (size_t)iters, s);
        if (e != cudaSuccess) return e;
    }
    for (int it = 0; it < iters; ++it) {
        if ((e = enqueue_density(c, s, pos, n, rec)) != cudaSuccess) return e;
        if (metrics && it > 0) {
            rec.before(s, K_QUALITY);
            e = launch_quality(s, c->counts, c->g.log2N, c->qacc + 3 * (it - 1));
            rec.after(s);
            if (e != cudaSuccess) return e;
        }
        if ((e = enqueue_inims(c, s, a, c->mode, rec)) != cudaSuccess) return e;
        rec.before(s, K_ADVECT);
        e = launch_advect(s, reinterpret_cast<float2 *>(pos), n, c->disp, c->g.log2N, c->p.pixel_center,
                          c->p.clamp_positions);
        rec.after(s);
        if (e != cudaSuccess) return e;
    }
    if (metrics && iters > 0) {
        if ((e = enqueue_density(c, s, pos, n, rec)) != cudaSuccess) return e;
        rec.before(s, K_QUALITY);
        e = launch_quality(s, c->counts, c->g.log2N, c->qacc + 3 * (iters - 1));
        rec.after(s);
    }
    return e;
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

const char *kKernelNames[DC_KERNEL_KINDS] = {"splat",  "smooth", "band_aggregate", "band_carry",
                                             "band_final", "advect", "quality",   "memset"};

}  // namespace

void dc::set_last_error(const char *msg) { g_last_error = msg ? msg : ""; }

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
    for (int k = 0; k < 4; ++k)
        if (p.reserved[k] != 0) return fail(DC_ERR_INVALID_ARG, "reserved fields must be zero");
    const int N = 1 << p.log2_res;
    int r = p.kernel_r;
    if (r < 0) r = N / 128 < 2 ? 2 : N / 128;
    if (r > 64 || r >= N) return fail(DC_ERR_INVALID_ARG, "kernel_r = %d (max 64, < N)", r);
    if (p.pixel_center != 0 && p.pixel_center != 1) return fail(DC_ERR_INVALID_ARG, "pixel_center");
    if (p.clamp_positions != 0 && p.clamp_positions != 1) return fail(DC_ERR_INVALID_ARG, "clamp_positions");
    if (p.carry_mode != DC_CARRY_COMPENSATED && p.carry_mode != DC_CARRY_F64)
        return fail(DC_ERR_INVALID_ARG, "carry_mode");
    if (p.band_rows != 0) {
        const int T = p.band_rows;
        if (T < 1 || T > 64 || (T & (T - 1)) || T > N) return fail(DC_ERR_INVALID_ARG, "band_rows = %d", T);
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
    c->g = make_band_geom((int)p.log2_res, p.band_rows);
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
    if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(DC_ERR_CUDA, "cudaStreamCreateWithFlags"));
    const size_t NN = (size_t)N * N;
    const size_t agg_bytes = (size_t)c->g.nb * c->g.agg_stride * 8;
    const size_t carry_bytes = (size_t)(c->g.nb + 1) * c->g.lanes * 8;
    struct {
        void **p;
        size_t bytes;
    } allocs[] = {
        {(void **)&c->counts, NN * sizeof(uint32_t)},
        {(void **)&c->disp, NN * sizeof(float2)},
        {&c->agg, agg_bytes},
        {&c->carry, carry_bytes},
        {(void **)&c->status, 256},
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
    if (prepare_kernels() != cudaSuccess) return bail(fail(DC_ERR_CUDA, "kernel attributes"));
    for (int k = 0; k < 128; ++k)
        if (cudaEventCreate(&c->prof_ev[k]) != cudaSuccess) return bail(fail(DC_ERR_CUDA, "cudaEventCreate"));
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
    for (int k = 0; k < 128; ++k)
        if (c->prof_ev[k]) cudaEventDestroy(c->prof_ev[k]);
    cudaFree(c->counts);
    cudaFree(c->dens);
    cudaFree(c->disp);
    cudaFree(c->agg);
    cudaFree(c->carry);
    cudaFree(c->status);
    cudaFree(c->qacc);
    cudaFree(c->hpos);
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
    out->kernels_per_iter = c->mode == MODE_FLOAT ? 6 : 5;
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
    DC_CUDA(enqueue_density(c, c->stream, pos, n, rec));
    const size_t NN = (size_t)c->g.N * c->g.N;
    if (counts_out) DC_CUDA(cudaMemcpyAsync(counts_out, c->counts, NN * 4, cudaMemcpyDeviceToDevice, c->stream));
    if (density_out) DC_CUDA(cudaMemcpyAsync(density_out, c->dens, NN * 4, cudaMemcpyDeviceToDevice, c->stream));
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
    const void *src = c->mode == MODE_FLOAT ? (const void *)c->dens : (const void *)c->counts;
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
    const void *src = c->mode == MODE_FLOAT ? (const void *)c->dens : (const void *)c->counts;
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

dc_status advect_samples(dc_ctx *c, float *pos, int64_t n)
{
    if (dc_status st = check_ctx(c)) return st;
    if (dc_status st = check_samples(c, pos, n)) return st;
    if (!c->have_disp) return fail(DC_ERR_STATE, "advect_samples before displacement_field");
    DeviceGuard guard(c->device);
    DC_CUDA(launch_advect(c->stream, reinterpret_cast<float2 *>(pos), n, c->disp, c->g.log2N, c->p.pixel_center,
                          c->p.clamp_positions));
    return DC_OK;
}

dc_status declutter_sync(dc_ctx *c)
{
    if (dc_status st = check_ctx(c)) return st;
    DeviceGuard guard(c->device);
    DC_CUDA(cudaStreamSynchronize(c->stream));
    unsigned st = 0;
    DC_CUDA(cudaMemcpy(&st, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (st != 0) {
        cudaMemset(c->status, 0, sizeof(unsigned));
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
    cudaGraphExec_t exec = nullptr;
    for (auto &ge : c->graphs)
        if (ge.pos == pos && ge.n == n && ge.iters == iters && ge.metrics == metrics) exec = ge.exec;
    if (!exec) {
        if (c->graphs.size() >= 16) {
            cudaGraphExecDestroy(c->graphs.front().exec);
            c->graphs.erase(c->graphs.begin());
        }
        cudaGraph_t graph = nullptr;
        DC_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        Recorder rec;
        cudaError_t e = enqueue_iterations(c, c->cap_stream, pos, n, iters, metrics, rec);
        cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(DC_ERR_CUDA, "graph capture: %s / %s", cudaGetErrorString(e), cudaGetErrorString(e2));
        }
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(DC_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
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

dc_status regularize_host(dc_ctx *c, float *host_pos, int64_t n, int32_t iters, double *uniformity_out)
{
    if (dc_status st = check_ctx(c)) return st;
    if (n < 0 || n >= (int64_t(1) << 32)) return fail(DC_ERR_INVALID_ARG, "n");
    if (n > 0 && !host_pos) return fail(DC_ERR_INVALID_ARG, "null host pointer");
    DeviceGuard guard(c->device);
    if (n > c->hpos_cap) {
        DC_CUDA(cudaStreamSynchronize(c->stream));
        cudaFree(c->hpos);
        c->hpos = nullptr;
        c->hpos_cap = 0;
        if (cudaMalloc(&c->hpos, sizeof(float) * 2 * (size_t)n) != cudaSuccess) {
            cudaGetLastError();
            return fail(DC_ERR_OOM, "staging buffer");
        }
        c->hpos_cap = n;
    }
    const size_t bytes = sizeof(float) * 2 * (size_t)n;
    if (n > 0) DC_CUDA(cudaMemcpyAsync(c->hpos, host_pos, bytes, cudaMemcpyHostToDevice, c->stream));
    if (dc_status st = regularize(c, c->hpos, n, iters, uniformity_out)) return st;
    if (n > 0) DC_CUDA(cudaMemcpyAsync(host_pos, c->hpos, bytes, cudaMemcpyDeviceToHost, c->stream));
    return declutter_sync(c);
}

dc_status quality_metrics(dc_ctx *c, double *out)
{
    if (dc_status st = check_ctx(c)) return st;
    if (!out) return fail(DC_ERR_INVALID_ARG, "null out");
    if (c->n_last < 0) return fail(DC_ERR_STATE, "quality_metrics before splat_density");
    DeviceGuard guard(c->device);
    unsigned long long acc[3];
    DC_CUDA(cudaMemsetAsync(c->qacc, 0, sizeof(acc), c->stream));
    DC_CUDA(launch_quality(c->stream, c->counts, c->g.log2N, c->qacc));
    DC_CUDA(cudaMemcpyAsync(acc, c->qacc, sizeof(acc), cudaMemcpyDeviceToHost, c->stream));
    if (dc_status st = declutter_sync(c)) return st;
    metrics_from_acc(c, acc, out);
    return DC_OK;
}

dc_status declutter_profile_regularize(dc_ctx *c, float *pos, int64_t n, int32_t iters, float *kernel_ms_out,
                                       int32_t *launches_out)
{
    if (dc_status st = check_ctx(c)) return st;
    if (dc_status st = check_samples(c, pos, n)) return st;
    if (iters < 0) return fail(DC_ERR_INVALID_ARG, "iters");
    DeviceGuard guard(c->device);
    float ms[DC_KERNEL_KINDS] = {};
    int32_t cnt[DC_KERNEL_KINDS] = {};
    for (int it = 0; it < iters; ++it) {
        Recorder rec;
        rec.ctx = c;
        DC_CUDA(enqueue_iterations(c, c->stream, pos, n, 1, 0, rec));
        if (rec.overflow) return fail(DC_ERR_INVALID_ARG, "too many launches to record");
        DC_CUDA(cudaStreamSynchronize(c->stream));
        for (int k = 0; k < rec.used; ++k) {
            float t = 0.f;
            DC_CUDA(cudaEventElapsedTime(&t, c->prof_ev[2 * k], c->prof_ev[2 * k + 1]));
            ms[rec.kinds[k]] += t;
            cnt[rec.kinds[k]] += 1;
        }
    }
    c->n_last = n;
    c->have_disp = true;
    if (kernel_ms_out) std::memcpy(kernel_ms_out, ms, sizeof(ms));
    if (launches_out) std::memcpy(launches_out, cnt, sizeof(cnt));
    return declutter_sync(c);
}

}  // extern "C"
