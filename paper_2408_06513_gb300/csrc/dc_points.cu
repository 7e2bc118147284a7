// Per-sample kernels: splat (Sec. 4.1), advection (Sec. 4.2) and the
// Sec. 6.2 quality reduction over the count grid.
#include <atomic>

#include "dc_internal.cuh"

namespace dc {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float clamp01(float v)
{
    // fmaxf(NaN, 0) = 0, so NaN counts as 0
    return fminf(fmaxf(v, 0.0f), 1.0f);
}

// Single-pixel accumulation (Sec. 4.1, Sec. 4.3 step 1).  Pixel index
// floor(x N) of the clamped coordinate; x N is exact in float since N is a
// power of two.  Lanes of a warp that hit the same pixel are merged with
// __match_any_sync so that one atomic carries their common count: heavy
// clusters put many samples of a warp into the same pixel.
__global__ void __launch_bounds__(kThreads) splat_kernel(const float2 *__restrict__ pos, int64_t n,
                                                         uint32_t *__restrict__ counts, int log2N)
{
    pdl_wait();
    const int N = 1 << log2N;
    const float fN = (float)N;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t k = base + lane;
        int pix = -1 - lane;  // distinct per lane when out of range
        if (k < n) {
            const float2 z = pos[k];
            const int i = min((int)(clamp01(z.x) * fN), N - 1);
            const int j = min((int)(clamp01(z.y) * fN), N - 1);
            pix = (j << log2N) + i;
        }
        const unsigned m = __match_any_sync(0xffffffffu, pix);
        if (k < n && lane == __ffs(m) - 1) atomicAdd(&counts[pix], (uint32_t)__popc(m));
    }
}

// The same splat, also recording each sample's rank among the samples of its
// pixel (the counter value its atomic increment returned), for the
// reordering below.  Ranks of a pixel's samples are exactly 0 .. count - 1.
// One atomic a sample, without warp aggregation: the samples arrive in the
// caller's order, where lanes of a warp rarely share a pixel (the 512^2
// step measured 0.2275 against 0.2347 ms with __match_any_sync).
// copy_out (or null): every sample is also written there (a device copy of
// samples that live in host memory, for the reordering's scatter).
__device__ __forceinline__ void splat_rank_body(const float2 *__restrict__ pos, int64_t n,
                                                              uint32_t *__restrict__ counts, int log2N,
                                                              uint32_t *__restrict__ rank,
                                                              float2 *__restrict__ copy_out = nullptr)
{
    pdl_wait();
    const int N = 1 << log2N;
    const float fN = (float)N;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // kU warp-rows of samples a trip: loads, then the independent atomics
    constexpr int kU = 4;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += kU * stride) {
        int pix[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int64_t k = base + u * stride + lane;
            pix[u] = -1 - lane;
            if (k < n) {
                const float2 z = pos[k];
                if (copy_out) copy_out[k] = z;
                const int i = min((int)(clamp01(z.x) * fN), N - 1);
                const int j = min((int)(clamp01(z.y) * fN), N - 1);
                pix[u] = (j << log2N) + i;
            }
        }
        // one atomic a sample: its return value is the sample's rank (or,
        // without rank, a reduction whose value nobody waits for)
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int64_t k = base + u * stride + lane;
            if (k < n) {
                if (rank) rank[k] = atomicAdd(&counts[pix[u]], 1u);
                else atomicAdd(&counts[pix[u]], 1u);
            }
        }
    }
}
__global__ void __launch_bounds__(kThreads) splat_rank_kernel(const float2 *__restrict__ pos, int64_t n,
                                                              uint32_t *__restrict__ counts, int log2N,
                                                              uint32_t *__restrict__ rank,
                                                              float2 *__restrict__ copy_out)
{
    splat_rank_body(pos, n, counts, log2N, rank, copy_out);
}

// Bilinear advection (Sec. 4.2): p = x N (- 1/2 for pixel centres),
// i0 = floor(p), f = p - i0, corners clamped to the grid.  px is first
// limited to [-1, N], which leaves every clamped corner index and every
// interpolated value unchanged but keeps the integer conversion in range.
struct Moved {
    float2 z;
    int pix;
};

// floor(v) for -2^22 <= v < 2^22 on the FMA pipe: adding 1.5 * 2^23 with
// rounding toward -inf leaves floor(v) in the low mantissa bits; fl is
// floor(v) as a float (exact)
__device__ __forceinline__ int floor_fma(float v, float &fl)
{
    const float r = __fadd_rd(v, 12582912.0f);
    fl = r - 12582912.0f;
    return __float_as_int(r) - 0x4B400000;
}

__device__ __forceinline__ Moved advect_one(float2 z, const float2 *__restrict__ D, int log2N, float fN, float off,
                                            int clamp)
{
    const int N = 1 << log2N;
    const float px = fminf(fmaxf(z.x * fN - off, -1.0f), fN);
    const float py = fminf(fmaxf(z.y * fN - off, -1.0f), fN);
    float fx, fy;
    const int ix = floor_fma(px, fx), iy = floor_fma(py, fy);
    const float f = px - fx, h = py - fy;
    const int i0 = min(max(ix, 0), N - 1), i1 = min(max(ix + 1, 0), N - 1);
    const int j0 = min(max(iy, 0), N - 1), j1 = min(max(iy + 1, 0), N - 1);
    const float2 d00 = __ldg(&D[(j0 << log2N) + i0]);
    const float2 d01 = __ldg(&D[(j0 << log2N) + i1]);
    const float2 d10 = __ldg(&D[(j1 << log2N) + i0]);
    const float2 d11 = __ldg(&D[(j1 << log2N) + i1]);
    const float dx = (1.0f - h) * ((1.0f - f) * d00.x + f * d01.x) + h * ((1.0f - f) * d10.x + f * d11.x);
    const float dy = (1.0f - h) * ((1.0f - f) * d00.y + f * d01.y) + h * ((1.0f - f) * d10.y + f * d11.y);
    z.x += dx;
    z.y += dy;
    if (clamp) {
        z.x = clamp01(z.x);
        z.y = clamp01(z.y);
    }
    // pixel of the moved sample for the next iteration's splat (Sec. 4.1 rule)
    float unused;
    const int si = min(floor_fma(clamp01(z.x) * fN, unused), N - 1);
    const int sj = min(floor_fma(clamp01(z.y) * fN, unused), N - 1);
    return {z, (sj << log2N) + si};
}

// Position loads that bypass L1 (each float4 is read once).
__device__ __forceinline__ float4 ldg_stream(const float4 *p)
{
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

// Splat one sample per lane with warp aggregation: lanes holding the same
// pixel are merged and their leader adds the group's size.  All 32 lanes
// must call this together; lanes with valid = false add nothing.
__device__ __forceinline__ void splat_warp(uint32_t *__restrict__ counts, int pix, bool valid)
{
    const int lane = threadIdx.x & 31;
    const int key = valid ? pix : -1 - lane;
    const unsigned m = __match_any_sync(0xffffffffu, key);
    if (valid && lane == __ffs(m) - 1) atomicAdd(&counts[pix], (uint32_t)__popc(m));
}

// Runs over the warp's 64 samples of one row of pairs: lane L holds samples
// 2L (pixel p0) and 2L + 1 (pixel p1), so in sample order the keys are
// p0(0), p1(0), p0(1), p1(1), ...  A sample starts a run when its key
// differs from the one before it; the run's first sample adds the run's
// length (the distance to the next start, or to the end of the row).  One
// shuffle and two ballots a row, no __match_any_sync (whose issue rate
// limited the kernel at 16M samples); after the reordering by pixel nearly
// every duplicate is a neighbour.  All 32 lanes must call this together;
// lanes with valid = false add nothing.
__device__ __forceinline__ void splat_pair_runs(uint32_t *__restrict__ counts, int p0, int p1, bool valid)
{
    const int lane = threadIdx.x & 31;
    const int k0 = valid ? p0 : -1 - 2 * lane;  // distinct negative keys for empty lanes
    const int k1 = valid ? p1 : -2 - 2 * lane;
    const int prev = __shfl_up_sync(0xffffffffu, k1, 1);
    const bool h0 = lane == 0 || k0 != prev;
    const bool h1 = k1 != k0;
    const unsigned b0 = __ballot_sync(0xffffffffu, h0), b1 = __ballot_sync(0xffffffffu, h1);
    const unsigned above = ~((2u << lane) - 1u);  // lanes after this one (lane 31: none)
    const unsigned a0 = b0 & above, a1 = b1 & above;
    const int s0 = a0 ? 2 * (__ffs(a0) - 1) : 64;
    const int s1 = a1 ? 2 * (__ffs(a1) - 1) + 1 : 64;
    const int next = min(s0, s1);  // first run start after this lane's pair
    if (valid && h0) atomicAdd(&counts[p0], (uint32_t)(h1 ? 1 : next - 2 * lane));
    if (valid && h1) atomicAdd(&counts[p1], (uint32_t)(next - 2 * lane - 1));
}

// Samples are processed in aligned pairs (one float4 = two samples), two
// pairs per thread and loop trip, so that all eight corner gathers of a trip
// are independent.  The loop runs warp-uniformly so that, with counts_next
// set, the moved samples can be splatted into the next iteration's count
// grid (which must be zero) with warp aggregation: after the reordering by
// pixel, neighbouring lanes mostly hold samples of the same pixel.  A sample
// before the first 16-byte boundary and one left after the last pair are
// handled by thread 0 of block 0.
// Squared length of a sample's move (domain units); lanes that hold no
// sample give 0.
__device__ __forceinline__ float move2(float2 a, float2 b, bool valid)
{
    const float dx = b.x - a.x, dy = b.y - a.y;
    return valid ? dx * dx + dy * dy : 0.0f;
}

// MAXD: the largest squared move of a sample is atomically maxed into
// *dmax as float bits (non-negative floats order like their bit patterns),
// one atomic per warp and trip: the impact of the iteration (Sec. 4.3 step 4).
template <bool RUNS, bool MAXD = false>
__device__ __forceinline__ void advect_body(float2 *__restrict__ pos, int64_t n, const float2 *__restrict__ D,
                                            int log2N, float off, int clamp, uint32_t *__restrict__ counts_next,
                                            unsigned *__restrict__ dmax = nullptr)
{
    pdl_wait();
    const float fN = (float)(1 << log2N);
    const int lane = threadIdx.x & 31;
    const int64_t head = (reinterpret_cast<uintptr_t>(pos) & 15) ? 1 : 0;
    const int64_t npairs = (n - head) / 2;
    float4 *pp = reinterpret_cast<float4 *>(pos + head);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // the next trip's two pairs are loaded before this trip's gathers
    int64_t qb = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    float4 na = zero4, nb = zero4;
    if (qb < npairs) {
        if (qb + lane < npairs) na = ldg_stream(pp + qb + lane);
        if (qb + lane + stride < npairs) nb = ldg_stream(pp + qb + lane + stride);
    }
    for (; qb < npairs; qb += 2 * stride) {
        const int64_t q1 = qb + lane, q2 = q1 + stride;
        const bool v1 = q1 < npairs, v2 = q2 < npairs;
        const float4 a = na, b = nb;
        const int64_t qn = qb + 2 * stride;
        na = zero4;
        nb = zero4;
        if (qn < npairs) {
            if (qn + lane < npairs) na = ldg_stream(pp + qn + lane);
            if (qn + lane + stride < npairs) nb = ldg_stream(pp + qn + lane + stride);
        }
        const Moved m0 = advect_one(make_float2(a.x, a.y), D, log2N, fN, off, clamp);
        const Moved m1 = advect_one(make_float2(a.z, a.w), D, log2N, fN, off, clamp);
        const Moved m2 = advect_one(make_float2(b.x, b.y), D, log2N, fN, off, clamp);
        const Moved m3 = advect_one(make_float2(b.z, b.w), D, log2N, fN, off, clamp);
        if (v1) pp[q1] = make_float4(m0.z.x, m0.z.y, m1.z.x, m1.z.y);
        if (v2) pp[q2] = make_float4(m2.z.x, m2.z.y, m3.z.x, m3.z.y);
        if constexpr (MAXD) {
            const float d = fmaxf(fmaxf(move2(make_float2(a.x, a.y), m0.z, v1), move2(make_float2(a.z, a.w), m1.z, v1)),
                                  fmaxf(move2(make_float2(b.x, b.y), m2.z, v2), move2(make_float2(b.z, b.w), m3.z, v2)));
            const unsigned w = __reduce_max_sync(0xffffffffu, __float_as_uint(d));
            if (lane == 0 && w) atomicMax(dmax, w);
        }
        if (counts_next) {
            if constexpr (RUNS) {
                splat_pair_runs(counts_next, m0.pix, m1.pix, v1);
                splat_pair_runs(counts_next, m2.pix, m3.pix, v2);
            } else {
                splat_warp(counts_next, m0.pix, v1);
                splat_warp(counts_next, m1.pix, v1);
                splat_warp(counts_next, m2.pix, v2);
                splat_warp(counts_next, m3.pix, v2);
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int64_t singles[2] = {head ? 0 : -1, (n - head) & 1 ? n - 1 : -1};
        for (int s = 0; s < 2; ++s) {
            if (singles[s] < 0) continue;
            const float2 z0 = pos[singles[s]];
            const Moved m = advect_one(z0, D, log2N, fN, off, clamp);
            pos[singles[s]] = m.z;
            if (counts_next) atomicAdd(&counts_next[m.pix], 1u);
            if constexpr (MAXD) {
                const unsigned w = __float_as_uint(move2(z0, m.z, true));
                if (w) atomicMax(dmax, w);
            }
        }
    }
}
template <bool RUNS, bool MAXD>
__global__ void __launch_bounds__(kThreads) advect_kernel(float2 *__restrict__ pos, int64_t n,
                                                          const float2 *__restrict__ D, int log2N, float off,
                                                          int clamp, uint32_t *__restrict__ counts_next,
                                                          unsigned *__restrict__ dmax)
{
    advect_body<RUNS, MAXD>(pos, n, D, log2N, off, clamp, counts_next, dmax);
}

// ------------------------------------------------------------------------
// Reordering of the samples by pixel (a counting sort keyed by the splat
// pixel), so that the iterations touch the grids with spatial locality.
// The method itself does not depend on the order of the samples: counts are
// integer sums and every sample moves by the same field.
// ------------------------------------------------------------------------
constexpr int kScanThreads = 256;

__device__ __forceinline__ uint32_t block_sum_u32(uint32_t v, uint32_t *s_red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) s_red[w] = v;
    __syncthreads();
    uint32_t t = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s_red[k];
    __syncthreads();
    if (threadIdx.x == 0) s_red[0] = t;
    __syncthreads();
    return s_red[0];
}

// partials[b] = sum of counts[b * chunk, (b + 1) * chunk)
__device__ __forceinline__ void scan_partials_body(const uint32_t *__restrict__ counts, int64_t M,
                                                                     int64_t chunk, uint32_t *__restrict__ partials)
{
    __shared__ uint32_t s_red[kScanThreads / 32];
    pdl_wait();
    const int64_t beg = (int64_t)blockIdx.x * chunk;
    const int64_t end = min(M, beg + chunk);
    uint32_t v = 0;
    for (int64_t k = beg + 4 * threadIdx.x; k < end; k += 4 * kScanThreads) {
        const uint4 q = *reinterpret_cast<const uint4 *>(counts + k);
        v += q.x + q.y + q.z + q.w;
    }
    v = block_sum_u32(v, s_red);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
}
__global__ void __launch_bounds__(kScanThreads) scan_partials_kernel(const uint32_t *__restrict__ counts, int64_t M,
                                                                     int64_t chunk, uint32_t *__restrict__ partials)
{
    scan_partials_body(counts, M, chunk, partials);
}

// cursor[k] = sum of counts[0, k) (exclusive prefix in row-major order).
__device__ __forceinline__ void scan_apply_body(const uint32_t *__restrict__ counts, int64_t M,
                                                                  int64_t chunk, const uint32_t *__restrict__ partials,
                                                                  uint32_t *__restrict__ cursor)
{
    __shared__ uint32_t s_red[kScanThreads / 32];
    __shared__ uint32_t s_w[kScanThreads / 32];
    pdl_wait();
    uint32_t pre = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += kScanThreads) pre += partials[b];
    uint32_t carry = block_sum_u32(pre, s_red);
    const int64_t beg = (int64_t)blockIdx.x * chunk;
    const int64_t end = min(M, beg + chunk);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t t0 = beg; t0 < end; t0 += 4 * kScanThreads) {
        const int64_t k = t0 + 4 * threadIdx.x;
        uint4 q = make_uint4(0, 0, 0, 0);
        if (k < end) q = *reinterpret_cast<const uint4 *>(counts + k);
        const uint32_t tsum = q.x + q.y + q.z + q.w;
        uint32_t x = tsum;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        __syncthreads();
        if (lane == 31) s_w[w] = x;
        __syncthreads();
        uint32_t wpre = 0, tile = 0;
        for (int k2 = 0; k2 < kScanThreads / 32; ++k2) {
            if (k2 < w) wpre += s_w[k2];
            tile += s_w[k2];
        }
        uint32_t e = carry + wpre + (x - tsum);
        if (k < end) {
            uint4 o;
            o.x = e; e += q.x;
            o.y = e; e += q.y;
            o.z = e; e += q.z;
            o.w = e;
            *reinterpret_cast<uint4 *>(cursor + k) = o;
        }
        carry += tile;
    }
}
__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const uint32_t *__restrict__ counts, int64_t M,
                                                                  int64_t chunk, const uint32_t *__restrict__ partials,
                                                                  uint32_t *__restrict__ cursor)
{
    scan_apply_body(counts, M, chunk, partials, cursor);
}

__device__ __forceinline__ int sample_pixel(float2 z, int log2N, float fN)
{
    const int N = 1 << log2N;
    const int i = min((int)(clamp01(z.x) * fN), N - 1);
    const int j = min((int)(clamp01(z.y) * fN), N - 1);
    return (j << log2N) + i;
}

// spos[slot] = pos[k] and inv[k] = slot, with slot = cursor[pixel] + rank[k]
// (cursor: exclusive prefix of the counts), or, without ranks, the value an
// atomic increment of cursor[pixel] returns.  The slots of pixel p are
// [prefix(p), prefix(p) + counts(p)), so every slot < n when cursor and rank
// come from the splat of these same samples; a slot out of range sets
// DC_ERR_RANGE in the status word and is skipped.
//
// Only slots in [lo, hi) are written by one launch: the sorted array is
// filled in windows small enough to stay in L2, so that the 8-byte writes
// to random slots of a window merge there into whole sectors before they
// reach DRAM (a sector written piecemeal after eviction costs a DRAM
// read-modify-write per sample).  The first window's launch (first = 1)
// computes the slots and stores them in inv; the later ones read them back.
// Sources are read with the streaming (evict-first) hint to spare the
// window's lines.
__device__ __forceinline__ void reorder_scatter_body(const float2 *__restrict__ pos, int64_t n,
                                                                   int log2N, uint32_t *__restrict__ cursor,
                                                                   const uint32_t *__restrict__ rank,
                                                                   float2 *__restrict__ spos,
                                                                   uint32_t *__restrict__ inv,
                                                                   unsigned *__restrict__ status, int64_t lo,
                                                                   int64_t hi, int first)
{
    pdl_wait();
    const float fN = (float)(1 << log2N);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const float2 z = __ldcs(pos + k);
        uint32_t slot;
        if (first) {
            // without ranks the sample claims the next slot of its pixel
            slot = rank ? __ldg(&cursor[sample_pixel(z, log2N, fN)]) + __ldcs(rank + k)
                        : atomicAdd(&cursor[sample_pixel(z, log2N, fN)], 1u);
            if ((int64_t)slot >= n) {
                inv[k] = 0xffffffffu;
                atomicOr(status, (unsigned)DC_ERR_RANGE);
                continue;
            }
            inv[k] = slot;
        } else {
            slot = __ldcs(inv + k);
            if ((int64_t)slot >= n) continue;  // reported by the first launch
        }
        if ((int64_t)slot >= lo && (int64_t)slot < hi) spos[slot] = z;
    }
}
__global__ void __launch_bounds__(kThreads) reorder_scatter_kernel(const float2 *__restrict__ pos, int64_t n,
                                                                   int log2N, uint32_t *__restrict__ cursor,
                                                                   const uint32_t *__restrict__ rank,
                                                                   float2 *__restrict__ spos,
                                                                   uint32_t *__restrict__ inv,
                                                                   unsigned *__restrict__ status, int64_t lo,
                                                                   int64_t hi, int first)
{
    reorder_scatter_body(pos, n, log2N, cursor, rank, spos, inv, status, lo, hi, first);
}

// pos[k] = spos[inv[k]]
__device__ __forceinline__ void reorder_gather_back_body(const float2 *__restrict__ spos,
                                                                       const uint32_t *__restrict__ inv, int64_t n,
                                                                       float2 *__restrict__ pos,
                                                                       unsigned *__restrict__ status)
{
    pdl_wait();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const uint32_t s = inv[k];
        if ((int64_t)s < n) pos[k] = spos[s];
        else atomicOr(status, (unsigned)DC_ERR_RANGE);
    }
}
__global__ void __launch_bounds__(kThreads) reorder_gather_back_kernel(const float2 *__restrict__ spos,
                                                                       const uint32_t *__restrict__ inv, int64_t n,
                                                                       float2 *__restrict__ pos,
                                                                       unsigned *__restrict__ status)
{
    reorder_gather_back_body(spos, inv, n, pos, status);
}

// Sec. 6.2: sum of squared 4x4-bin counts and number of occupied pixels.
// acc[0] += sum of b^2 over bins, acc[1] += occupied pixels, acc[2] += sum b.
__device__ __forceinline__ void quality_body(const uint32_t *__restrict__ counts, int log2N,
                                                           unsigned long long *__restrict__ acc)
{
    pdl_wait();
    const int N = 1 << log2N;
    const int B = N >> 2;
    const int nbins = B * B;
    unsigned long long ss = 0, occ = 0, tot = 0;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += gridDim.x * blockDim.x) {
        const int bi = b % B, bj = b / B;
        unsigned long long s = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint4 q = *reinterpret_cast<const uint4 *>(&counts[((size_t)(4 * bj + r) << log2N) + 4 * bi]);
            s += (unsigned long long)q.x + q.y + q.z + q.w;
            occ += (q.x != 0) + (q.y != 0) + (q.z != 0) + (q.w != 0);
        }
        ss += s * s;
        tot += s;
    }
    for (int o = 16; o > 0; o >>= 1) {
        ss += __shfl_down_sync(0xffffffffu, ss, o);
        occ += __shfl_down_sync(0xffffffffu, occ, o);
        tot += __shfl_down_sync(0xffffffffu, tot, o);
    }
    __shared__ unsigned long long red[3][kThreads / 32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        red[0][w] = ss;
        red[1][w] = occ;
        red[2][w] = tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = 0, c = 0, t = 0;
        for (int k = 0; k < kThreads / 32; ++k) {
            a += red[0][k];
            c += red[1][k];
            t += red[2][k];
        }
        atomicAdd(&acc[0], a);
        atomicAdd(&acc[1], c);
        atomicAdd(&acc[2], t);
    }
}
__global__ void __launch_bounds__(kThreads) quality_kernel(const uint32_t *__restrict__ counts, int log2N,
                                                           unsigned long long *__restrict__ acc)
{
    quality_body(counts, log2N, acc);
}

int grid_for(int64_t n, int per_block, int max_blocks)
{
    int64_t b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

// CTAs of the advection kernel resident on the whole GPU at once, per device
// (set by prepare_kernels): its grid is at most one wave, the grid-stride
// loop with the next trip's samples prefetched covering the rest (1.6 waves
// of one trip each measured slower at 1M samples).
constexpr int kMaxDevices = 64;
std::atomic<int> g_advect_wave[kMaxDevices];

int advect_wave()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return device_sms() * 4;
    }
    const int w = g_advect_wave[dev].load(std::memory_order_relaxed);
    return w > 0 ? w : device_sms() * 4;
}

}  // namespace

cudaError_t prepare_point_kernels()
{
    int dev = 0, sms = 0, p0 = 0, p1 = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p0, advect_kernel<false, false>, kThreads, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p1, advect_kernel<true, false>, kThreads, 0);
    if (e == cudaSuccess && dev >= 0 && dev < kMaxDevices && sms > 0 && p0 > 0 && p1 > 0)
        g_advect_wave[dev].store((p0 < p1 ? p0 : p1) * sms, std::memory_order_relaxed);
    return e;
}

cudaError_t launch_splat(cudaStream_t s, const float2 *pos, int64_t n, uint32_t *counts, int log2N)
{
    if (n <= 0) return cudaSuccess;
    return launch_kernel(splat_kernel, dim3(grid_for(n, kThreads, device_sms() * 16)), dim3(kThreads), 0, s, pos, n, counts,
                         log2N);
}

cudaError_t launch_advect(cudaStream_t s, float2 *pos, int64_t n, const float2 *disp, int log2N,
                          int pixel_center, int clamp, uint32_t *counts_next, bool sorted, unsigned *dmax)
{
    if (n <= 0) return cudaSuccess;
    // two pairs (four samples) per thread and trip, at most one wave; run
    // aggregation for samples in pixel order
    const dim3 grid(grid_for((n + 3) / 4, kThreads, advect_wave()));
    const float off = pixel_center ? 0.5f : 0.0f;
    const bool runs = sorted;
    if (dmax) {
        if (runs)
            return launch_kernel(advect_kernel<true, true>, grid, dim3(kThreads), 0, s, pos, n, disp, log2N, off,
                                 clamp, counts_next, dmax);
        return launch_kernel(advect_kernel<false, true>, grid, dim3(kThreads), 0, s, pos, n, disp, log2N, off, clamp,
                             counts_next, dmax);
    }
    if (runs)
        return launch_kernel(advect_kernel<true, false>, grid, dim3(kThreads), 0, s, pos, n, disp, log2N, off, clamp,
                             counts_next, (unsigned *)nullptr);
    return launch_kernel(advect_kernel<false, false>, grid, dim3(kThreads), 0, s, pos, n, disp, log2N, off, clamp,
                         counts_next, (unsigned *)nullptr);
}

int64_t reorder_scan_chunk(int log2N)
{
    const int64_t M = (int64_t)1 << (2 * log2N);
    int64_t chunk = 4096;
    while (M / chunk > 1024) chunk *= 2;
    return chunk;
}

cudaError_t launch_reorder_scan(cudaStream_t s, const uint32_t *counts, int log2N, uint32_t *partials,
                                uint32_t *cursor)
{
    const int64_t M = (int64_t)1 << (2 * log2N);
    const int64_t chunk = reorder_scan_chunk(log2N);
    const int blocks = (int)((M + chunk - 1) / chunk);
    cudaError_t e = launch_kernel(scan_partials_kernel, dim3(blocks), dim3(kScanThreads), 0, s, counts, M, chunk,
                                  partials);
    if (e != cudaSuccess) return e;
    return launch_kernel(scan_apply_kernel, dim3(blocks), dim3(kScanThreads), 0, s, counts, M, chunk,
                         (const uint32_t *)partials, cursor);
}

cudaError_t launch_splat_rank(cudaStream_t s, const float2 *pos, int64_t n, uint32_t *counts, int log2N,
                              uint32_t *rank, float2 *copy_out)
{
    if (n <= 0) return cudaSuccess;
    return launch_kernel(splat_rank_kernel, dim3(grid_for(n, kThreads, device_sms() * 16)), dim3(kThreads), 0, s, pos, n,
                         counts, log2N, rank, copy_out);
}

// Slots a scatter window holds: 64 MB of samples, half the L2 (16M samples:
// two passes, 0.45 ms for the reordering against 0.49 ms with four passes of
// 32 MB and 0.6 ms with one pass).
constexpr int64_t kScatterWindow = (int64_t)(64 << 20) / sizeof(float2);

cudaError_t launch_reorder_scatter(cudaStream_t s, const float2 *pos, int64_t n, int log2N, uint32_t *cursor,
                                   const uint32_t *rank, float2 *spos, uint32_t *inv, unsigned *status)
{
    if (n <= 0) return cudaSuccess;
    const int64_t passes = (n + kScatterWindow - 1) / kScatterWindow;
    const int64_t win = (n + passes - 1) / passes;
    const dim3 grid(grid_for(n, kThreads, device_sms() * 8));
    cudaError_t e = cudaSuccess;
    for (int64_t p = 0; p < passes && e == cudaSuccess; ++p)
        e = launch_kernel(reorder_scatter_kernel, grid, dim3(kThreads), 0, s, pos, n, log2N, cursor, rank, spos, inv,
                          status, p * win, p + 1 == passes ? n : (p + 1) * win, p == 0 ? 1 : 0);
    return e;
}

cudaError_t launch_reorder_back(cudaStream_t s, const float2 *spos, const uint32_t *inv, int64_t n, float2 *pos,
                                unsigned *status)
{
    if (n <= 0) return cudaSuccess;
    return launch_kernel(reorder_gather_back_kernel, dim3(grid_for(n, kThreads, device_sms() * 8)), dim3(kThreads), 0, s,
                         spos, inv, n, pos, status);
}

cudaError_t launch_quality(cudaStream_t s, const uint32_t *counts, int log2N, unsigned long long *acc)
{
    const int B = (1 << log2N) >> 2;
    return launch_kernel(quality_kernel, dim3(grid_for((int64_t)B * B, kThreads, device_sms() * 4)), dim3(kThreads), 0, s,
                         counts, log2N, acc);
}

// ------------------------------------------------------------------------
// Batched wrappers: panel blockIdx.y of a PanelDesc table
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) zero_batched_kernel(const PanelDesc *__restrict__ tab, int log2N,
                                                                int which, int qacc_words)
{
    pdl_wait();
    const PanelDesc &d = tab[blockIdx.y];
    const int64_t M4 = ((int64_t)1 << (2 * log2N)) / 4;
    uint4 *c = reinterpret_cast<uint4 *>(d.counts[which]);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < M4; k += (int64_t)gridDim.x * blockDim.x)
        c[k] = make_uint4(0u, 0u, 0u, 0u);
    if (blockIdx.x == 0)
        for (int k = threadIdx.x; k < qacc_words; k += blockDim.x) d.qacc[k] = 0ull;
}
__global__ void __launch_bounds__(kThreads) splat_rank_batched_kernel(const PanelDesc *__restrict__ tab, int log2N)
{
    const PanelDesc &d = tab[blockIdx.y];
    splat_rank_body(d.pos, d.n, d.counts[0], log2N, d.rank);
}
__global__ void __launch_bounds__(kScanThreads) scan_partials_batched_kernel(const PanelDesc *__restrict__ tab,
                                                                             int64_t M, int64_t chunk)
{
    pdl_wait();  // before the early return (see pdl_wait)
    const PanelDesc &d = tab[blockIdx.y];
    if (d.n <= 0) return;  // no samples: no sort buffers, nothing to reorder
    scan_partials_body(d.counts[0], M, chunk, d.partials);
}
__global__ void __launch_bounds__(kScanThreads) scan_apply_batched_kernel(const PanelDesc *__restrict__ tab,
                                                                          int64_t M, int64_t chunk)
{
    pdl_wait();
    const PanelDesc &d = tab[blockIdx.y];
    if (d.n <= 0) return;
    scan_apply_body(d.counts[0], M, chunk, d.partials, d.cursor);
}
__global__ void __launch_bounds__(kThreads) scatter_batched_kernel(const PanelDesc *__restrict__ tab, int log2N)
{
    const PanelDesc &d = tab[blockIdx.y];
    reorder_scatter_body(d.pos, d.n, log2N, d.cursor, d.rank, d.spos, d.inv, d.status, 0, d.n, 1);
}
template <bool RUNS>
__global__ void __launch_bounds__(kThreads) advect_batched_kernel(const PanelDesc *__restrict__ tab, int log2N,
                                                                  float off, int clamp, int nxt)
{
    const PanelDesc &d = tab[blockIdx.y];
    advect_body<RUNS>(d.spos, d.n, d.disp, log2N, off, clamp, nxt >= 0 ? d.counts[nxt] : nullptr);
}
__global__ void __launch_bounds__(kThreads) quality_batched_kernel(const PanelDesc *__restrict__ tab, int log2N,
                                                                   int which, int slot)
{
    const PanelDesc &d = tab[blockIdx.y];
    quality_body(d.counts[which], log2N, d.qacc + 3 * slot);
}
__global__ void __launch_bounds__(kThreads) back_batched_kernel(const PanelDesc *__restrict__ tab)
{
    const PanelDesc &d = tab[blockIdx.y];
    reorder_gather_back_body(d.spos, d.inv, d.n, d.pos, d.status);
}



cudaError_t launch_zero_batched(cudaStream_t s, const PanelDesc *tab, int P, int log2N, int which, int qacc_words)
{
    const int64_t M4 = ((int64_t)1 << (2 * log2N)) / 4;
    return launch_kernel(zero_batched_kernel, dim3(grid_for(M4, kThreads, 64), P), dim3(kThreads), 0, s, tab, log2N,
                         which, qacc_words);
}

cudaError_t launch_splat_rank_batched(cudaStream_t s, const PanelDesc *tab, int P, int64_t max_n, int log2N)
{
    if (max_n <= 0) return cudaSuccess;
    return launch_kernel(splat_rank_batched_kernel, dim3(grid_for(max_n, kThreads, device_sms() * 16), P), dim3(kThreads), 0,
                         s, tab, log2N);
}

cudaError_t launch_reorder_batched(cudaStream_t s, const PanelDesc *tab, int P, int64_t max_n, int log2N)
{
    if (max_n <= 0) return cudaSuccess;
    const int64_t M = (int64_t)1 << (2 * log2N);
    const int64_t chunk = reorder_scan_chunk(log2N);
    const unsigned nch = (unsigned)((M + chunk - 1) / chunk);
    cudaError_t e = launch_kernel(scan_partials_batched_kernel, dim3(nch, P), dim3(kScanThreads), 0, s, tab, M, chunk);
    if (e == cudaSuccess)
        e = launch_kernel(scan_apply_batched_kernel, dim3(nch, P), dim3(kScanThreads), 0, s, tab, M, chunk);
    if (e == cudaSuccess)
        e = launch_kernel(scatter_batched_kernel, dim3(grid_for(max_n, kThreads, device_sms() * 8), P), dim3(kThreads), 0, s,
                          tab, log2N);
    return e;
}

cudaError_t launch_advect_batched(cudaStream_t s, const PanelDesc *tab, int P, int64_t max_n, int log2N,
                                  int pixel_center, int clamp, int nxt, bool sorted)
{
    if (max_n <= 0) return cudaSuccess;
    const dim3 grid(grid_for((max_n + 3) / 4, kThreads, device_sms() * 8), P);
    if (sorted)
        return launch_kernel(advect_batched_kernel<true>, grid, dim3(kThreads), 0, s, tab, log2N,
                             pixel_center ? 0.5f : 0.0f, clamp, nxt);
    return launch_kernel(advect_batched_kernel<false>, grid, dim3(kThreads), 0, s, tab, log2N,
                         pixel_center ? 0.5f : 0.0f, clamp, nxt);
}

cudaError_t launch_quality_batched(cudaStream_t s, const PanelDesc *tab, int P, int log2N, int which, int slot)
{
    const int B = 1 << (log2N - 2);
    return launch_kernel(quality_batched_kernel, dim3(grid_for((int64_t)B * B, kThreads, device_sms() * 4), P), dim3(kThreads),
                         0, s, tab, log2N, which, slot);
}

cudaError_t launch_back_batched(cudaStream_t s, const PanelDesc *tab, int P, int64_t max_n)
{
    if (max_n <= 0) return cudaSuccess;
    return launch_kernel(back_batched_kernel, dim3(grid_for(max_n, kThreads, device_sms() * 8), P), dim3(kThreads), 0, s, tab);
}

}  // namespace dc
