// The density background texture of Sec. 5: the original density drawn on
// the mesh of pixel nodes after the nodes have been moved by the method's
// mapping (e.g. as tracers of regularize_tracers), then mapped to colours by
// a transfer function.  A plain two-pass rasteriser in CUDA: (1) one thread
// per triangle of the deformed mesh (the whole warp for a triangle the
// mapping expanded) marks the output pixels whose centres it covers
// (fixed-point vertices with 8 sub-pixel bits, exact integer edge
// functions, a fill rule that gives a point on a shared edge or vertex to
// exactly one triangle, the lowest triangle index winning where triangles
// overlap); (2) one thread per output pixel takes the texture at the source
// point with the pixel centre's barycentric coordinates in its triangle
// (bilinear lookup between nodes), optionally times the undeformed over the
// deformed area (the push-forward density).
#include "dc_internal.cuh"

namespace dc {

namespace {

constexpr int kThreads = 256;
constexpr int kSub = 8;  // sub-pixel bits
constexpr uint32_t kNone = 0xffffffffu;

struct Fx {
    long long x, y;
};

// Fixed-point vertex: rint(float32(x * 2^(log2M + 8))) of x clamped to
// [-1, 2] (NaN -> -1); the product is exact (a power of two).
__device__ __forceinline__ Fx fixed_vertex(float2 z, float scale)
{
    const float x = fminf(fmaxf(z.x, -1.0f), 2.0f), y = fminf(fmaxf(z.y, -1.0f), 2.0f);
    return {__float2ll_rn(x * scale), __float2ll_rn(y * scale)};
}

// Node indices of triangle t of the mesh: cell c = t / 2 = j (N - 1) + i;
// t even: (i, j), (i+1, j), (i+1, j+1); t odd: (i, j), (i+1, j+1), (i, j+1).
__device__ __forceinline__ void tri_nodes(uint32_t t, int N, int (&ni)[3], int (&nj)[3])
{
    const uint32_t c = t >> 1;
    const int i = (int)(c % (uint32_t)(N - 1)), j = (int)(c / (uint32_t)(N - 1));
    ni[0] = i;
    nj[0] = j;
    if (t & 1) {
        ni[1] = i + 1; nj[1] = j + 1;
        ni[2] = i;     nj[2] = j + 1;
    } else {
        ni[1] = i + 1; nj[1] = j;
        ni[2] = i + 1; nj[2] = j + 1;
    }
}

__device__ __forceinline__ long long edge(Fx u, Fx v, long long px, long long py)
{
    return (v.x - u.x) * (py - u.y) - (v.y - u.y) * (px - u.x);
}

// A point exactly on edge u -> v (of a triangle of positive orientation)
// belongs to the triangle when the edge runs up, or level and to the right.
__device__ __forceinline__ bool owns(Fx u, Fx v)
{
    const long long dy = v.y - u.y, dx = v.x - u.x;
    return dy < 0 || (dy == 0 && dx > 0);
}

__global__ void __launch_bounds__(kThreads) clear_u32_kernel(uint32_t *__restrict__ p, int64_t count, uint32_t v)
{
    pdl_wait();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += stride) p[k] = v;
}

// Triangles whose bounding box holds at most kSmallBox pixel centres are
// covered by their own thread; larger ones (cells the mapping expanded) by
// the whole warp, one triangle after another, the lanes striding over its
// box, so that one expanded cell does not hold up its warp.
constexpr long long kSmallBox = 64;

__global__ void __launch_bounds__(kThreads) warp_raster_kernel(const float2 *__restrict__ nodes, int N, int log2M,
                                                               uint32_t *__restrict__ cover)
{
    pdl_wait();
    const uint32_t ntri = 2u * (uint32_t)(N - 1) * (uint32_t)(N - 1);
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int M = 1 << log2M;
    const float scale = (float)(1 << (log2M + kSub));
    const long long half = 1ll << (kSub - 1), one = 1ll << kSub;
    Fx a{0, 0}, b{0, 0}, c{0, 0};
    long long p0 = 0, p1 = -1, q0 = 0, q1 = -1;
    if (t < ntri) {
        int ni[3], nj[3];
        tri_nodes(t, N, ni, nj);
        a = fixed_vertex(nodes[nj[0] * N + ni[0]], scale);
        b = fixed_vertex(nodes[nj[1] * N + ni[1]], scale);
        c = fixed_vertex(nodes[nj[2] * N + ni[2]], scale);
        const long long area = (b.x - a.x) * (c.y - a.y) - (b.y - a.y) * (c.x - a.x);
        if (area < 0) {  // orient positively
            const Fx s = b;
            b = c;
            c = s;
        }
        if (area != 0) {  // a degenerate triangle covers nothing: empty box
            const long long mnx = min(a.x, min(b.x, c.x)), mxx = max(a.x, max(b.x, c.x));
            const long long mny = min(a.y, min(b.y, c.y)), mxy = max(a.y, max(b.y, c.y));
            p0 = max(0ll, (mnx - half + one - 1) >> kSub);
            p1 = min((long long)M - 1, (mxx - half) >> kSub);
            q0 = max(0ll, (mny - half + one - 1) >> kSub);
            q1 = min((long long)M - 1, (mxy - half) >> kSub);
        }
    }
    const long long box = (p1 >= p0 && q1 >= q0) ? (p1 - p0 + 1) * (q1 - q0 + 1) : 0;
    auto cover_pixel = [&](const Fx &ta, const Fx &tb, const Fx &tc, uint32_t tri, long long p, long long q) {
        const long long px = (p << kSub) + half, py = (q << kSub) + half;
        const long long e0 = edge(ta, tb, px, py), e1 = edge(tb, tc, px, py), e2 = edge(tc, ta, px, py);
        const bool in = (e0 > 0 || (e0 == 0 && owns(ta, tb))) && (e1 > 0 || (e1 == 0 && owns(tb, tc))) &&
                        (e2 > 0 || (e2 == 0 && owns(tc, ta)));
        if (in) atomicMin(&cover[(q << log2M) + p], tri);
    };
    if (box > 0 && box <= kSmallBox)
        for (long long q = q0; q <= q1; ++q)
            for (long long p = p0; p <= p1; ++p) cover_pixel(a, b, c, t, p, q);
    unsigned big = __ballot_sync(0xffffffffu, box > kSmallBox);
    while (big) {
        const int src = __ffs(big) - 1;
        big &= big - 1;
        const Fx ta{__shfl_sync(0xffffffffu, a.x, src), __shfl_sync(0xffffffffu, a.y, src)};
        const Fx tb{__shfl_sync(0xffffffffu, b.x, src), __shfl_sync(0xffffffffu, b.y, src)};
        const Fx tc{__shfl_sync(0xffffffffu, c.x, src), __shfl_sync(0xffffffffu, c.y, src)};
        const long long bp0 = __shfl_sync(0xffffffffu, p0, src), bq0 = __shfl_sync(0xffffffffu, q0, src);
        const long long bw = __shfl_sync(0xffffffffu, p1, src) - bp0 + 1;
        const long long bbox = __shfl_sync(0xffffffffu, box, src);
        const uint32_t tri = __shfl_sync(0xffffffffu, t, src);
        for (long long k = lane; k < bbox; k += 32) cover_pixel(ta, tb, tc, tri, bp0 + k % bw, bq0 + k / bw);
    }
}

__global__ void __launch_bounds__(kThreads) warp_shade_kernel(const float2 *__restrict__ nodes,
                                                              const float *__restrict__ tex, int N, int log2M,
                                                              int mass, const uint32_t *__restrict__ cover,
                                                              float *__restrict__ out)
{
    pdl_wait();
    const int M = 1 << log2M;
    const int64_t MM = (int64_t)M * M;
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= MM) return;
    const uint32_t t = cover[pix];
    if (t == kNone) {
        out[pix] = 0.0f;
        return;
    }
    const float scale = (float)(1 << (log2M + kSub));
    int ni[3], nj[3];
    tri_nodes(t, N, ni, nj);
    const Fx a = fixed_vertex(nodes[nj[0] * N + ni[0]], scale);
    const Fx b = fixed_vertex(nodes[nj[1] * N + ni[1]], scale);
    const Fx c = fixed_vertex(nodes[nj[2] * N + ni[2]], scale);
    const long long area = (b.x - a.x) * (c.y - a.y) - (b.y - a.y) * (c.x - a.x);  // != 0: it covers pixels
    const long long half = 1ll << (kSub - 1);
    const long long px = ((pix & (M - 1)) << kSub) + half, py = ((pix >> log2M) << kSub) + half;
    // barycentric weights of b and c (a takes the rest)
    const long long eb = (px - a.x) * (c.y - a.y) - (py - a.y) * (c.x - a.x);
    const long long ec = (b.x - a.x) * (py - a.y) - (b.y - a.y) * (px - a.x);
    const float fa = (float)area;
    const float lb = (float)eb / fa, lc = (float)ec / fa;
    const float la = 1.0f - lb - lc;
    float si = la * ni[0] + lb * ni[1] + lc * ni[2];
    float sj = la * nj[0] + lb * nj[1] + lc * nj[2];
    si = fminf(fmaxf(si, 0.0f), (float)(N - 1));
    sj = fminf(fmaxf(sj, 0.0f), (float)(N - 1));
    const int x0 = min((int)floorf(si), N - 2), y0 = min((int)floorf(sj), N - 2);
    const float fx = si - x0, fy = sj - y0;
    const float *r0 = tex + (size_t)y0 * N + x0;
    const float *r1 = r0 + N;
    float v = (1.0f - fy) * ((1.0f - fx) * __ldg(r0) + fx * __ldg(r0 + 1)) +
              fy * ((1.0f - fx) * __ldg(r1) + fx * __ldg(r1 + 1));
    if (mass) {
        const float cell = (float)M * (float)(1 << kSub) / (float)N;
        v *= cell * cell / fabsf(fa);  // undeformed over deformed edge cross product
    }
    out[pix] = v;
}

// Transfer function: value -> RGBA8 colour of a 256-entry table, index
// rint((v - lo) * 255 / (hi - lo)) clamped to 0..255 (float32, in that order).
__global__ void __launch_bounds__(kThreads) transfer_kernel(const float *__restrict__ v, int64_t count, float lo,
                                                            float scale, const uint32_t *__restrict__ lut,
                                                            uint32_t *__restrict__ rgba)
{
    pdl_wait();
    __shared__ uint32_t s_lut[256];
    s_lut[threadIdx.x] = lut[threadIdx.x];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += stride) {
        const float x = __fmul_rn(__fsub_rn(v[k], lo), scale);
        const float c = fminf(fmaxf(rintf(x), 0.0f), 255.0f);  // NaN -> 0
        rgba[k] = s_lut[(int)c];
    }
}

int blocks_for(int64_t n, int cap)
{
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

}  // namespace

cudaError_t launch_warp_texture(cudaStream_t s, const float2 *nodes, const float *tex, int log2N, int log2M,
                                int mass, uint32_t *cover, float *out)
{
    const int N = 1 << log2N;
    const int64_t MM = (int64_t)1 << (2 * log2M);
    cudaError_t e = launch_kernel(clear_u32_kernel, dim3(blocks_for(MM, device_sms() * 8)), dim3(kThreads), 0, s, cover,
                                  MM, kNone);
    if (e != cudaSuccess) return e;
    const int64_t ntri = 2ll * (N - 1) * (N - 1);
    e = launch_kernel(warp_raster_kernel, dim3((unsigned)((ntri + kThreads - 1) / kThreads)), dim3(kThreads), 0, s,
                      nodes, N, log2M, cover);
    if (e != cudaSuccess) return e;
    return launch_kernel(warp_shade_kernel, dim3((unsigned)((MM + kThreads - 1) / kThreads)), dim3(kThreads), 0, s,
                         nodes, tex, N, log2M, mass, (const uint32_t *)cover, out);
}

cudaError_t launch_transfer(cudaStream_t s, const float *v, int64_t count, float lo, float hi, const uint32_t *lut,
                            uint32_t *rgba)
{
    if (count <= 0) return cudaSuccess;
    const float scale = 255.0f / (hi - lo);
    return launch_kernel(transfer_kernel, dim3(blocks_for(count, device_sms() * 8)), dim3(256), 0, s, v, count, lo,
                         scale, lut, rgba);
}

}  // namespace dc
