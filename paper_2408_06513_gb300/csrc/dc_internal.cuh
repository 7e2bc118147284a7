// Internal declarations shared by the translation units of libdeclutter.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "declutter.h"

namespace dc {

// Programmatic dependent launch.  Every kernel is launched with programmatic
// stream serialisation, so that its launch overlaps the tail of the kernel
// before it; every CTA of every kernel calls pdl_wait() before it touches any
// global memory and before any early return: it blocks until the preceding
// grid has completed and its writes are visible.  No kernel releases its
// dependents early (griddepcontrol.launch_dependents): that measured slower
// (0.243 against 0.237 ms a 512^2 step, 2.47 against 2.02 ms at 16M samples).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                          Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// word of the context's status buffer where the fused band kernel's grid
// barrier (arrivals, generation) lives
constexpr int kBarWord = 16;

// Kernel kinds, in the order reported by declutter_profile_regularize().
enum KernelKind {
    K_SPLAT = 0,
    K_SMOOTH = 1,
    K_BAND_AGG = 2,
    K_CARRY = 3,
    K_BAND_FINAL = 4,
    K_ADVECT = 5,
    K_QUALITY = 6,
    K_REORDER = 7,  // counting sort of the samples by pixel, and the way back
    K_BAND_FUSED = 8,  // aggregate + carries + final pass in one cooperative launch
    K_SMOOTH_AGG = 9,  // smoothing and the aggregate pass in one launch (float mode, 128^2 .. 1024^2)
};

// Accumulation mode of the integral-image kernels.
enum Mode {
    MODE_COUNT = 0,  // uint32 counts, uint32 arithmetic (exact: all sums < 2^32)
    MODE_FLOAT = 1,  // float d_r minus the mean mu, float arithmetic
    MODE_GRID64 = 2, // arbitrary uint32 grid, uint64 arithmetic
};

// Band decomposition of the N x N grid for the integral-image kernels:
// nb bands of T full-width rows; each band is one CTA of NT threads, thread t
// owning columns [t*CPT, t*CPT + CPT).
struct BandGeom {
    int N = 0, log2N = 0;
    int T = 0, nb = 0;
    int NT = 0, CPT = 0;
    int agg_stride = 0; // elements per band in the compact aggregate array
    int lanes = 0;      // 5N absolute carry lanes
    int sms = 0;        // SMs of the device (band and carry launch shapes)
};

// band_rows = 0: automatic height for a device of `sms` SMs
BandGeom make_band_geom(int log2N, int band_rows, int sms);
// SM count of the calling thread's current device (cached per device; 1 if
// it cannot be queried)
int device_sms();

// Gaussian weights passed by value (kernel parameter space).
struct GaussW {
    float g[129];
    int r;
};

// Per-launch arguments of the band kernels.
struct BandArgs {
    const void *src;          // uint32 (COUNT, GRID64) or float (FLOAT), N*N
    float mu;                 // FLOAT: mean subtracted from d_r
    void *agg;                // compact aggregates [nb][agg_stride]
    int agg_stride;
    const void *carry;        // carries [nb + 1][lanes]
    // final-kernel outputs (any may be null)
    float2 *disp;             // domain units
    void *alpha_out;          // uint64 (COUNT, GRID64) or float (FLOAT)
    void *alpha_t_out;
    uint32_t *zero_out;       // aggregate kernel: zero this N*N grid (band rows), or null
    // displacement constants
    int pixel_center;
    float d0;                 // regularising constant (>= 0)
    double inv_den_exact;     // COUNT: 1 / (2 S N^2 (n + d0 N^2))
    int lens;                 // FLOAT final pass: t(x, y; d) - (x, y) (eq. (map) without the defect)
    unsigned *status;         // sticky device status word (DC_ERR_TIMEOUT), or null
};

// One panel of a batch of same-resolution panels, for the batched launches:
// kernel wrappers take a device array of these and read their panel's
// buffers from entry blockIdx.y (blockIdx.z for the 2D smoothing grid).
struct PanelDesc {
    float2 *pos;              // the caller's samples
    int64_t n;
    uint32_t *counts[2];      // count grids (iterations alternate)
    float *dens;
    float2 *disp;
    float2 *spos;             // samples in pixel order
    uint32_t *rank, *inv, *cursor, *partials;
    unsigned long long *qacc; // [3 * iters]
    unsigned *status;
    BandArgs band;            // agg, carry, disp, mu, d0, inv_den_exact, status (src and zero_out per launch)
};

struct GraphEntry {
    const void *pos = nullptr;
    int64_t n = 0;
    int iters = 0;
    int metrics = 0;
    int adaptive = 0;  // regularize_adaptive's graph (conditional iterations)
    cudaGraphExec_t exec = nullptr;
};

// Launchers (all enqueue on `s`; return cudaGetLastError()).
cudaError_t launch_splat(cudaStream_t s, const float2 *pos, int64_t n, uint32_t *counts, int log2N);
// counts_next: if not null, the moved samples are also splatted into it (must
// be zero); sorted: the samples are in pixel order (run aggregation pays);
// dmax: if not null, the largest squared move of a sample (domain units) is
// maxed into it as float bits
cudaError_t launch_advect(cudaStream_t s, float2 *pos, int64_t n, const float2 *disp, int log2N,
                          int pixel_center, int clamp, uint32_t *counts_next, bool sorted = false,
                          unsigned *dmax = nullptr);
cudaError_t launch_quality(cudaStream_t s, const uint32_t *counts, int log2N, unsigned long long *acc);
// reordering of the samples by pixel: the first splat also records each
// sample's rank within its pixel (rank not null); exclusive scan of the
// counts into cursor (partials: at most 1024 entries); scatter into spos with
// inv[k] = slot of sample k (without ranks, slots are claimed by atomic
// increments of cursor); gather back pos[k] = spos[inv[k]]
cudaError_t launch_splat_rank(cudaStream_t s, const float2 *pos, int64_t n, uint32_t *counts, int log2N,
                              uint32_t *rank, float2 *copy_out = nullptr);
int64_t reorder_scan_chunk(int log2N);
cudaError_t launch_reorder_scan(cudaStream_t s, const uint32_t *counts, int log2N, uint32_t *partials,
                                uint32_t *cursor);
cudaError_t launch_reorder_scatter(cudaStream_t s, const float2 *pos, int64_t n, int log2N, uint32_t *cursor,
                                   const uint32_t *rank, float2 *spos, uint32_t *inv, unsigned *status);
cudaError_t launch_reorder_back(cudaStream_t s, const float2 *spos, const uint32_t *inv, int64_t n, float2 *pos,
                                unsigned *status);
cudaError_t launch_smooth(cudaStream_t s, const uint32_t *counts, float *dens, int log2N, const GaussW &w,
                          uint32_t *zero_out);
cudaError_t launch_band_agg(cudaStream_t s, const BandGeom &g, int mode, const BandArgs &a);
// marching squares on a float N x N field: two float4 segment slots per cell
// ((N-1)^2 cells, row-major), NaN for empty slots
cudaError_t launch_contour(cudaStream_t s, const float *field, int log2N, float level, int pixel_center,
                           float4 *segs);
// smoothing of counts into dens fused with the float-mode aggregate pass
// (a.src = dens); zero_out as in launch_smooth
bool smooth_agg_available(const BandGeom &g, const GaussW &w);
cudaError_t launch_smooth_agg(cudaStream_t s, const BandGeom &g, const BandArgs &a, const GaussW &w,
                              const uint32_t *counts, float *dens, uint32_t *zero_out);
cudaError_t launch_carry(cudaStream_t s, const BandGeom &g, int mode, int carry_mode, const void *agg,
                         void *carry);
cudaError_t launch_band_final(cudaStream_t s, const BandGeom &g, int mode, const BandArgs &a);
// one cooperative launch of the three band phases (grids below 2048^2);
// available when all CTAs fit on the device at once; bar: two device words
// bar: two device words; each grid-barrier wait gives up after limit_ns
// (DC_ERR_TIMEOUT); extra_arrivals > 0 makes the barrier wait for that many
// CTAs more than the grid holds (testing the timeout path)
bool band_fused_available(const BandGeom &g, int mode, int carry_mode, int device);
cudaError_t launch_band_fused(cudaStream_t s, const BandGeom &g, int mode, int carry_mode, const BandArgs &aagg,
                              const BandArgs &afin, unsigned *bar, unsigned long long limit_ns,
                              unsigned extra_arrivals);
int smooth_smem_bytes(int r);
// batched launches over P same-resolution panels (tab: device PanelDesc[P]);
// max_n: the largest n; which / cur: count grid index; nxt: grid to splat the
// moved samples into, or -1
cudaError_t launch_zero_batched(cudaStream_t s, const PanelDesc *tab, int P, int log2N, int which, int qacc_words);
cudaError_t launch_splat_rank_batched(cudaStream_t s, const PanelDesc *tab, int P, int64_t max_n, int log2N);
cudaError_t launch_reorder_batched(cudaStream_t s, const PanelDesc *tab, int P, int64_t max_n, int log2N);
cudaError_t launch_advect_batched(cudaStream_t s, const PanelDesc *tab, int P, int64_t max_n, int log2N,
                                  int pixel_center, int clamp, int nxt, bool sorted);
cudaError_t launch_quality_batched(cudaStream_t s, const PanelDesc *tab, int P, int log2N, int which, int slot);
cudaError_t launch_back_batched(cudaStream_t s, const PanelDesc *tab, int P, int64_t max_n);
cudaError_t launch_smooth_batched(cudaStream_t s, const PanelDesc *tab, int P, int log2N, const GaussW &w, int cur,
                                  bool zero_next);
// aggregate, carries and final pass (grids below 2048^2, the per-thread-contiguous band kernels)
cudaError_t launch_band_batched(cudaStream_t s, const BandGeom &g, int mode, int carry_mode, const PanelDesc *tab,
                                int P, int cur, bool zero_next);
// out[k] = (1 - t) a[k] + t b[k] for count floats, rounded as written
cudaError_t launch_transition(cudaStream_t s, const float *a, const float *b, int64_t count, float t, float *out);
// per-query terms of the Sec. 6.2 layout measures (trustworthiness, orthogonal
// ordering) of reg against orig: terms[2q] = sum of (rank - k) over the new
// k-neighbours of query q missing from its original k-neighbourhood,
// terms[2q + 1] = samples whose orthogonal order relative to q changed (-1, -1
// for a query index outside [0, n)); qo, qn: uint32[n] scratch; queries: device
// uint32[n_queries] or null for 0 .. n_queries - 1; 1 <= k <= 32
cudaError_t launch_layout_terms(cudaStream_t s, const float2 *orig, const float2 *reg, int64_t n,
                                const uint32_t *queries, int n_queries, int k, uint32_t *qo, uint32_t *qn,
                                long long *terms);
// Sec. 4.3 step 4, inside a graph: the start kernel stamps the time; the
// check kernel of iteration it reads its Sec. 6.2 accumulators and largest
// move, records them, and sets the condition of iteration it + 1 (when
// has_next) to 0 once a criterion holds
struct AdaptState {
    double target_cv;      // stop when bin std / mean <= target_cv (> 0)
    double min_move_px;    // stop when the largest move <= min_move_px (> 0)
    double max_ns;         // stop when the elapsed device time >= max_ns (> 0)
    unsigned long long t0; // %globaltimer at the start of the graph
    int iters;             // iterations done
    int pad;
};
cudaError_t launch_adapt_start(cudaStream_t s, AdaptState *st);
cudaError_t launch_adapt_check(cudaStream_t s, const unsigned long long *qacc, const unsigned *dmax, AdaptState *st,
                               double *cv, double *move_px, int it, int log2N, cudaGraphConditionalHandle next,
                               int has_next);
// Sec. 5 density texture on the deformed node mesh (N = 2^log2N nodes a
// side, texture N x N) rasterised into M x M, M = 2^log2M: cover[M*M]
// receives the winning triangle per pixel (0xffffffff: none), out[M*M] the
// value (push-forward density with mass); and the transfer function
// value -> lut[rint((v - lo) 255 / (hi - lo))] (RGBA8)
cudaError_t launch_warp_texture(cudaStream_t s, const float2 *nodes, const float *tex, int log2N, int log2M,
                                int mass, uint32_t *cover, float *out);
cudaError_t launch_transfer(cudaStream_t s, const float *v, int64_t count, float lo, float hi, const uint32_t *lut,
                            uint32_t *rgba);
cudaError_t prepare_kernels();  // per-device kernel attributes; call with the device current
cudaError_t prepare_point_kernels();  // part of prepare_kernels: launch shapes of the sample kernels
void set_last_error(const char *msg);  // message returned by declutter_last_error()
// regularize() building blocks for the batched runtime: buffers for n samples
// (outside any capture), the iteration sequence on stream s, and the
// context's state after it; Sec. 6.2 measures from quality accumulators
dc_status prepare_regularize(dc_ctx *c, int64_t n, int iters, int metrics);
cudaError_t enqueue_regularize(dc_ctx *c, cudaStream_t s, float *pos, int64_t n, int iters, int metrics);
void finish_regularize(dc_ctx *c, int64_t n, int iters, int metrics);
void read_metrics(const dc_ctx *c, const unsigned long long *acc, double *out3);
// the panel table entry of a context and its samples (after prepare_regularize)
PanelDesc panel_desc(const dc_ctx *c, float *pos, int64_t n);

}  // namespace dc

struct dc_ctx {
    dc_params p{};
    int device = 0;
    cudaStream_t stream = nullptr;      // where everything runs
    bool own_stream = false;
    cudaStream_t cap_stream = nullptr;  // private stream used only for graph capture
    dc::BandGeom g;
    int r = 0;
    float sigma = 0.f;
    dc::GaussW w{};
    int mode = dc::MODE_COUNT;          // MODE_COUNT (r == 0) or MODE_FLOAT

    uint32_t *counts_buf[2] = {nullptr, nullptr}; // count grids (regularize alternates them)
    int cur_counts = 0;                 // which one holds the density the other calls use
    float *dens = nullptr;
    float2 *disp = nullptr;
    void *agg = nullptr;
    void *carry = nullptr;
    unsigned *status = nullptr;         // [0] sticky status; [kBarWord, +2) grid barrier of the fused band kernel
    bool fused = false;                 // band phases as one cooperative launch (see band_fused_available)
    bool smooth_agg = false;            // smoothing fused into the aggregate pass (see smooth_agg_available)
    unsigned *status_host = nullptr;    // pinned copy of the status word read by declutter_sync
    unsigned long long *qacc = nullptr; // [3 * (qslots)]
    int qslots = 0;
    float *hpos = nullptr;              // device staging for regularize_host
    // reordering buffers (grown on demand, outside graph capture)
    float2 *spos = nullptr;             // samples in pixel order
    uint32_t *rank = nullptr;           // rank of each sample within its pixel
    uint32_t *inv = nullptr;            // slot of each sample in spos
    int64_t sort_cap = 0;
    uint32_t *cursor = nullptr;         // N*N exclusive prefix of the counts
    uint32_t *partials = nullptr;       // <= 1024 chunk sums
    int64_t hpos_cap = 0;
    int64_t scratch_bytes = 0;
    // regularize_adaptive: AdaptState, then cv[cap], move_px[cap] (double),
    // then dmax[cap] (float bits); the bodies of the conditional iterations
    // are captured on cap_stream2
    void *adapt = nullptr;
    int adapt_cap = 0;
    cudaStream_t cap_stream2 = nullptr;
    // the reordering's branch beside the first iteration's grid passes:
    // forked from and joined back to the iteration stream by these events
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // set by regularize_host around a run on the caller's host memory: the
    // first splat copies the samples into hpos and the reordering's scatter
    // reads that copy, so the host array is read over the link once
    bool copy_first = false;
    // layout_metrics scratch: lattice coordinates of both layouts, query terms
    uint32_t *lq = nullptr;
    int64_t lq_cap = 0;
    long long *lterms = nullptr;
    int64_t lterms_cap = 0;
    // warp_texture coverage scratch (uint32 per output pixel)
    uint32_t *wcover = nullptr;
    int64_t wcover_cap = 0;

    int64_t n_last = -1;                // n of the last splat
    bool have_disp = false;

    std::vector<dc::GraphEntry> graphs;
    cudaEvent_t prof_ev[2] = {};
};
