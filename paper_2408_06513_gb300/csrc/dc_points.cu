// Per-sample kernels: splat (Sec. 4.1), advection (Sec. 4.2) and the
// Sec. 6.2 quality reduction over the count grid.
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

// Bilinear advection (Sec. 4.2): p = x N (- 1/2 for pixel centres),
// i0 = floor(p), f = p - i0, corners clamped to the grid.  px is first
// limited to [-1, N], which leaves every clamped corner index and every
// interpolated value unchanged but keeps the integer conversion in range.
__global__ void __launch_bounds__(kThreads) advect_kernel(float2 *__restrict__ pos, int64_t n,
                                                          const float2 *__restrict__ D, int log2N,
                                                          float off, int clamp)
{
    const int N = 1 << log2N;
    const float fN = (float)N;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        float2 z = pos[k];
        float px = fminf(fmaxf(z.x * fN - off, -1.0f), fN);
        float py = fminf(fmaxf(z.y * fN - off, -1.0f), fN);
        const float fx = floorf(px), fy = floorf(py);
        const float f = px - fx, h = py - fy;
        const int ix = (int)fx, iy = (int)fy;
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
        pos[k] = z;
    }
}

// Sec. 6.2: sum of squared 4x4-bin counts and number of occupied pixels.
// acc[0] += sum of b^2 over bins, acc[1] += occupied pixels, acc[2] += sum b.
__global__ void __launch_bounds__(kThreads) quality_kernel(const uint32_t *__restrict__ counts, int log2N,
                                                           unsigned long long *__restrict__ acc)
{
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

int grid_for(int64_t n, int per_block, int max_blocks)
{
    int64_t b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

}  // namespace

cudaError_t launch_splat(cudaStream_t s, const float2 *pos, int64_t n, uint32_t *counts, int log2N)
{
    if (n <= 0) return cudaSuccess;
    splat_kernel<<<grid_for(n, kThreads, 152 * 16), kThreads, 0, s>>>(pos, n, counts, log2N);
    return cudaGetLastError();
}

cudaError_t launch_advect(cudaStream_t s, float2 *pos, int64_t n, const float2 *disp, int log2N,
                          int pixel_center, int clamp)
{
    if (n <= 0) return cudaSuccess;
    advect_kernel<<<grid_for(n, kThreads, 152 * 16), kThreads, 0, s>>>(pos, n, disp, log2N,
                                                                         pixel_center ? 0.5f : 0.0f, clamp);
    return cudaGetLastError();
}

cudaError_t launch_quality(cudaStream_t s, const uint32_t *counts, int log2N, unsigned long long *acc)
{
    const int B = (1 << log2N) >> 2;
    quality_kernel<<<grid_for((int64_t)B * B, kThreads, 152 * 4), kThreads, 0, s>>>(counts, log2N, acc);
    return cudaGetLastError();
}

}  // namespace dc
