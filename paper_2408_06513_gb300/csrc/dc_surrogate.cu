// Learned surrogate of the iteration: a convolutional encoder-decoder that
// maps a density grid to the displacement field composed over several plain
// iterations (not in the paper).  Forward and backward passes run on the BF16
// tensor-core implicit GEMM of dc_sg_gemm.cuh; training is plain Adam.
//
// Network (levels L, widths c_l = c0 * 2^l), tensors [batch][y][x][channel]
// in bf16, channels padded to multiples of 8:
//   encoder l = 0..L-1:  ya = relu(conv(h)); yb = relu(conv(ya)); skip_l = yb;
//                        h = avgpool2(yb) for l < L-1
//   decoder l = L-2..0:  u = upsample2(h); yu = relu(conv(u)); s = yu + skip_l;
//                        h = relu(conv(s))
//   head:                out = conv(h), 2 channels, FP32
// conv: 3x3 cross-correlation with zero padding and bias; weights
// [out][3][3][in]; loss 0.5 * mean((out - target)^2).
#include <cuda_bf16.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dc_internal.cuh"
#include "dc_sg_gemm.cuh"
#include "dc_sg_umma.cuh"

using namespace dc;
using namespace dc::sg;
typedef __nv_bfloat16 bf16;

namespace {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
        else
            cudaGetLastError();
    }
    return fn;
}

// Tensor map of the K-contiguous weights W[N][K] (bf16) with boxes of 64 k x
// N rows in the 128-byte swizzle; false (stage with cp.async instead) when
// the encoder is unavailable or refuses.  Out-of-range k reads as zero.
bool weights_map(CUtensorMap *m, const void *W, int N, int K)
{
    std::memset(m, 0, sizeof(*m));
    EncodeTiledFn fn = encode_tiled();
    if (!fn || (reinterpret_cast<uintptr_t>(W) & 15) || ((size_t)K * 2) % 16 != 0 || N > 256) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)N};
    const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    const cuuint32_t box[2] = {(cuuint32_t)UM_TK, (cuuint32_t)N};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(W), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct Layer {
    std::string name;
    int cin = 0, cout = 0, cin_p = 0, cout_p = 0;
    int log2H = 0;          // spatial size 2^log2H x 2^log2H
    size_t woff = 0;        // offset in the padded weight arrays
    size_t boff = 0;        // offset in the padded bias arrays
    size_t wsize() const { return (size_t)cout_p * 9 * cin_p; }
};

int round8(int c) { return (c + 7) & ~7; }

// ------------------------------------------------------------------------
// Convolution problems for the implicit GEMM
// ------------------------------------------------------------------------
// Input pixel (yy, xx) of a 2^log2H grid; with up, the input is stored at
// half resolution and read through nearest 2x upsampling.
__device__ __forceinline__ const bf16 *conv_in(const bf16 *X, int b, int yy, int xx, int log2H, int up, int cin_p,
                                               int ci)
{
    const int lg = log2H - up;
    yy >>= up;
    xx >>= up;
    return X + ((((size_t)b << lg) + yy) << lg) * cin_p + (size_t)xx * cin_p + ci;
}

// Epilogue of a convolution output pair (n, n + 1) of row m: bias, ReLU,
// bf16 store, the decoder's skip sum S = bf16(Y + skip), fp32 head output.
struct ConvOut {
    int cout_p, out_ch, relu;
    const float *bias;
    bf16 *Y;            // bf16 output [M][cout_p] or null
    const bf16 *skip;   // with S: S = bf16(bf16(out) + skip)
    bf16 *S;
    float *Yf;          // fp32 output [M][out_ch] or null
    __device__ void store(int m, int n, float v0, float v1) const
    {
        v0 += bias[n];
        v1 += bias[n + 1];
        if (relu) {
            v0 = fmaxf(v0, 0.f);
            v1 = fmaxf(v1, 0.f);
        }
        const __nv_bfloat162 y = __floats2bfloat162_rn(v0, v1);
        if (Y) *reinterpret_cast<__nv_bfloat162 *>(Y + (size_t)m * cout_p + n) = y;
        if (S) {
            const float2 a = __bfloat1622float2(y);
            const float2 k = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(skip + (size_t)m * cout_p + n));
            *reinterpret_cast<__nv_bfloat162 *>(S + (size_t)m * cout_p + n) = __floats2bfloat162_rn(a.x + k.x, a.y + k.y);
        }
        if (Yf) {
            if (n < out_ch) Yf[(size_t)m * out_ch + n] = v0;
            if (n + 1 < out_ch) Yf[(size_t)m * out_ch + n + 1] = v1;
        }
    }
};

struct ConvFwd {
    static constexpr int ALAYOUT = K_CONTIG, BLAYOUT = K_CONTIG;
    int M, N, K;
    int log2H, cin_p, cout_p;
    int lg_cin;     // log2(cin_p): cin_p is a power of two (8 .. 256)
    int up;         // input at half resolution, upsampled on the fly
    const bf16 *X;
    const bf16 *W;
    ConvOut out;
    float *acc;     // split-K: fp32 partial sums [M][cout_p] (atomic), epilogue later
    __device__ const void *base() const { return W; }
    __device__ const void *a_chunk(int m, int k) const
    {
        const int tap = k >> lg_cin, ci = k & (cin_p - 1);
        const int dy = (tap * 11) >> 5, dx = tap - 3 * dy;  // tap / 3 for tap < 9
        const int H = 1 << log2H;
        const int x = m & (H - 1), y = (m >> log2H) & (H - 1), b = m >> (2 * log2H);
        const int yy = y + dy - 1, xx = x + dx - 1;
        if (yy < 0 || yy >= H || xx < 0 || xx >= H) return nullptr;
        return conv_in(X, b, yy, xx, log2H, up, cin_p, ci);
    }
    __device__ const void *b_chunk(int k, int n) const { return W + (size_t)n * K + k; }
    __device__ void epilogue(int m, int n, float v0, float v1) const
    {
        if (acc) {
            atomicAdd(&acc[(size_t)m * cout_p + n], v0);
            atomicAdd(&acc[(size_t)m * cout_p + n + 1], v1);
        } else {
            out.store(m, n, v0, v1);
        }
    }
};

// dX[q][ci] = sum_{tap, co} dZ[q - (dy - 1, dx - 1)][co] W[co][tap][ci]
struct ConvBwdData {
    static constexpr int ALAYOUT = K_CONTIG, BLAYOUT = MN_CONTIG;
    int M, N, K;
    int log2H, cin_p, cout_p;
    const bf16 *dZ;
    const bf16 *W;
    float *dX;  // fp32 [M][cin_p]
    __device__ const void *base() const { return W; }
    __device__ const void *a_chunk(int m, int k) const
    {
        const int tap = k / cout_p, co = k - tap * cout_p;
        const int dy = tap / 3, dx = tap - 3 * dy;
        const int H = 1 << log2H;
        const int x = m & (H - 1), y = (m >> log2H) & (H - 1), b = m >> (2 * log2H);
        const int yy = y - dy + 1, xx = x - dx + 1;
        if (yy < 0 || yy >= H || xx < 0 || xx >= H) return nullptr;
        return dZ + ((((size_t)b << log2H) + yy) << log2H) * cout_p + (size_t)xx * cout_p + co;
    }
    __device__ const void *b_chunk(int k, int n) const
    {
        const int tap = k / cout_p, co = k - tap * cout_p;
        return W + ((size_t)co * 9 + tap) * cin_p + n;
    }
    __device__ void epilogue(int m, int n, float v0, float v1) const
    {
        *reinterpret_cast<float2 *>(dX + (size_t)m * cin_p + n) = make_float2(v0, v1);
    }
};

// dW[co][tap][ci] += sum_p dZ[p][co] X[p + (dy - 1, dx - 1)][ci]  (split over p)
struct ConvWgrad {
    static constexpr int ALAYOUT = MN_CONTIG, BLAYOUT = MN_CONTIG;
    int M, N, K;
    int log2H, cin_p, cout_p;
    int up;         // X at half resolution, read upsampled
    const bf16 *dZ;
    const bf16 *X;
    float *dW;  // fp32 [cout_p][9 * cin_p]
    __device__ const void *base() const { return dZ; }
    __device__ const void *a_chunk(int m, int k) const { return dZ + (size_t)k * cout_p + m; }
    __device__ const void *b_chunk(int k, int n) const
    {
        const int tap = n / cin_p, ci = n - tap * cin_p;
        const int dy = tap / 3, dx = tap - 3 * dy;
        const int H = 1 << log2H;
        const int x = k & (H - 1), y = (k >> log2H) & (H - 1), b = k >> (2 * log2H);
        const int yy = y + dy - 1, xx = x + dx - 1;
        if (yy < 0 || yy >= H || xx < 0 || xx >= H) return nullptr;
        return conv_in(X, b, yy, xx, log2H, up, cin_p, ci);
    }
    __device__ void epilogue(int m, int n, float v0, float v1) const
    {
        atomicAdd(&dW[(size_t)m * N + n], v0);
        atomicAdd(&dW[(size_t)m * N + n + 1], v1);
    }
};

template <class P>
cudaError_t run_gemm(cudaStream_t s, const P &p, int splits = 1)
{
    int kps = (p.K + splits - 1) / splits;
    kps = (kps + BK - 1) / BK * BK;
    splits = (p.K + kps - 1) / kps;
    if (p.N <= 32) {  // narrow layers: 64 x 32 tiles
        dim3 grid((p.M + BM - 1) / BM, (p.N + 31) / 32, splits);
        return launch_kernel(gemm_kernel<P, 32>, grid, dim3(GEMM_THREADS), 0, s, p, kps);
    }
    dim3 grid((p.M + BM - 1) / BM, (p.N + BN - 1) / BN, splits);
    return launch_kernel(gemm_kernel<P, BN>, grid, dim3(GEMM_THREADS), 0, s, p, kps);
}

// ------------------------------------------------------------------------
// Elementwise kernels (grid-stride)
// ------------------------------------------------------------------------
#define GRID_STRIDE(i, n) for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
                               i += (int64_t)gridDim.x * blockDim.x)

// x[p][0] = bf16(dens[p] * scales[p / HW]) (scales null: 1); with field,
// x[p][1..2] = bf16(field[p][0..1]); the other channels up to 8 zero
__global__ void pack_input_kernel(const float *__restrict__ dens, const float *__restrict__ scales,
                                  const float *__restrict__ field, int log2HW, int64_t P, bf16 *__restrict__ x)
{
    pdl_wait();
    GRID_STRIDE(i, P * 8) {
        const int64_t p = i >> 3;
        const int c = (int)(i & 7);
        float v = 0.f;
        if (c == 0) v = dens[p] * (scales ? scales[p >> log2HW] : 1.f);
        else if (c < 3 && field) v = field[2 * p + (c - 1)];
        x[i] = __float2bfloat16_rn(v);
    }
}

// split-K epilogue: ConvOut of the summed partials, pairs of columns
__global__ void conv_finalize_kernel(const float *__restrict__ acc, int64_t M, int cout_p, ConvOut o)
{
    pdl_wait();
    GRID_STRIDE(i, M * (cout_p / 2)) {
        const int64_t m = i / (cout_p / 2);
        const int n = 2 * (int)(i - m * (cout_p / 2));
        o.store((int)m, n, acc[m * cout_p + n], acc[m * cout_p + n + 1]);
    }
}

__global__ void set_value_kernel(float *p, float v)
{
    pdl_wait();
    *p = v;
}

// out[p][c] += kappa * field[p][c]
__global__ void add_skip_kernel(float *__restrict__ out, const float *__restrict__ field, float kappa, int64_t n)
{
    pdl_wait();
    GRID_STRIDE(i, n) out[i] += kappa * field[i];
}

// field[p] = disp[p] * N (domain units to pixels)
__global__ void disp_to_field_kernel(const float2 *__restrict__ disp, int64_t P, float N, float *__restrict__ field)
{
    pdl_wait();
    GRID_STRIDE(p, P) {
        const float2 d = disp[p];
        field[2 * p] = d.x * N;
        field[2 * p + 1] = d.y * N;
    }
}

// out[b][y][x][c] = bf16(mean of the 2x2 block)
__global__ void avgpool_kernel(const bf16 *__restrict__ in, int log2H_out, int C, int64_t total, bf16 *__restrict__ out)
{
    pdl_wait();
    GRID_STRIDE(i, total) {
        const int c = (int)(i % C);
        const int64_t p = i / C;
        const int Ho = 1 << log2H_out;
        const int x = (int)(p & (Ho - 1)), y = (int)((p >> log2H_out) & (Ho - 1));
        const int64_t b = p >> (2 * log2H_out);
        const int Hi = 2 * Ho;
        const int64_t base = ((b * Hi + 2 * y) * Hi + 2 * x) * C + c;
        const float s = __bfloat162float(in[base]) + __bfloat162float(in[base + C]) +
                        __bfloat162float(in[base + (int64_t)Hi * C]) + __bfloat162float(in[base + (int64_t)Hi * C + C]);
        out[i] = __float2bfloat16_rn(0.25f * s);
    }
}

// loss += 0.5 (out - t)^2 over the 2 logical channels; g (8 channels) = bf16((out - t) / count)
__global__ void loss_kernel(const float *__restrict__ out, const float *__restrict__ target, int64_t P, float inv_count,
                            float *__restrict__ loss, bf16 *__restrict__ g)
{
    pdl_wait();
    float acc = 0.f;
    GRID_STRIDE(i, P * 8) {
        const int64_t p = i >> 3;
        const int c = (int)(i & 7);
        float gv = 0.f;
        if (c < 2) {
            const float d = out[p * 2 + c] - target[p * 2 + c];
            acc += 0.5f * d * d;
            gv = d * inv_count;
        }
        g[i] = __float2bfloat16_rn(gv);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc * inv_count);
}

// dz = bf16((g1 + g2) * [y > 0])   (g2 may be null)
__global__ void relu_grad_kernel(const float *__restrict__ g1, const float *__restrict__ g2, const bf16 *__restrict__ y,
                                 int64_t n, bf16 *__restrict__ dz)
{
    pdl_wait();
    GRID_STRIDE(i, n) {
        const float g = g1[i] + (g2 ? g2[i] : 0.f);
        dz[i] = __float2bfloat16_rn(__bfloat162float(y[i]) > 0.f ? g : 0.f);
    }
}

// dh (H) = sum over the 2x2 block of du (2H)
__global__ void upsample_bwd_kernel(const float *__restrict__ du, int log2H_out, int C, int64_t total,
                                    float *__restrict__ dh)
{
    pdl_wait();
    GRID_STRIDE(i, total) {
        const int c = (int)(i % C);
        const int64_t p = i / C;
        const int Ho = 1 << log2H_out;
        const int x = (int)(p & (Ho - 1)), y = (int)((p >> log2H_out) & (Ho - 1));
        const int64_t b = p >> (2 * log2H_out);
        const int Hi = 2 * Ho;
        const int64_t base = ((b * Hi + 2 * y) * Hi + 2 * x) * C + c;
        dh[i] = du[base] + du[base + C] + du[base + (int64_t)Hi * C] + du[base + (int64_t)Hi * C + C];
    }
}

// dh (2H) = dx (H) / 4 spread over each 2x2 block
__global__ void avgpool_bwd_kernel(const float *__restrict__ dx, int log2H_out, int C, int64_t total,
                                   float *__restrict__ dh)
{
    pdl_wait();
    GRID_STRIDE(i, total) {
        const int c = (int)(i % C);
        const int64_t p = i / C;
        const int Ho = 1 << log2H_out;
        const int x = (int)(p & (Ho - 1)), y = (int)((p >> log2H_out) & (Ho - 1));
        const int64_t b = p >> (2 * log2H_out);
        const int Hi = Ho / 2;
        dh[i] = 0.25f * dx[((b * Hi + y / 2) * Hi + x / 2) * C + c];
    }
}

// db[c] += sum over pixels of dz[p][c]; one thread per channel, blocks over pixel chunks
__global__ void bias_grad_kernel(const bf16 *__restrict__ dz, int64_t P, int C, int64_t chunk, float *__restrict__ db)
{
    pdl_wait();
    const int c = threadIdx.x;
    if (c >= C) return;
    const int64_t beg = (int64_t)blockIdx.x * chunk, end = min(P, beg + chunk);
    float s = 0.f;
    for (int64_t p = beg; p < end; ++p) s += __bfloat162float(dz[p * C + c]);
    atomicAdd(&db[c], s);
}

__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, bf16 *__restrict__ w16, int64_t n, float lr, float b1, float b2,
                            float eps, float bc1, float bc2)
{
    pdl_wait();
    GRID_STRIDE(i, n) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        w[i] = wi;
        if (w16) w16[i] = __float2bfloat16_rn(wi);
    }
}

__global__ void to_bf16_kernel(const float *__restrict__ a, int64_t n, bf16 *__restrict__ out)
{
    pdl_wait();
    GRID_STRIDE(i, n) out[i] = __float2bfloat16_rn(a[i]);
}

// disp (domain units, float2) = F (pixels) / N
__global__ void field_to_disp_kernel(const float *__restrict__ F, int64_t P, float invN, float2 *__restrict__ disp)
{
    pdl_wait();
    GRID_STRIDE(i, P) disp[i] = make_float2(F[2 * i] * invN, F[2 * i + 1] * invN);
}

int eb(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, (int64_t)device_sms() * 16); }

// host-side normal deviates (splitmix64 + Box-Muller), deterministic by seed
struct HostRng {
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double normal() { return std::sqrt(-2.0 * std::log(uniform())) * std::cos(6.283185307179586 * uniform()); }
};

dc_status sfail(dc_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return st;
}

#define SG_CUDA(call)                                                                             \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return sfail(DC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

struct dc_surrogate {
    int levels = 4, c0 = 32, log2H = 8, max_batch = 1;
    int in_channels = 1;
    float kappa = 0.f;                  // output skip kappa * field
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int tc_path = DC_SG_AUTO;           // tensor-core path of the forward convolutions (DC_SG_*)
                                        // (surrogate_set_tensor_path; measured slower at these sizes)
    unsigned *status = nullptr;         // DC_ERR_TIMEOUT from a bounded wait in a kernel
    cudaEvent_t ev[2] = {nullptr, nullptr};  // stream ordering with a context in surrogate_apply
    // surrogate_apply's forward pass + field conversion as one CUDA graph,
    // captured on a private stream for the context buffers it was made for
    cudaStream_t cap = nullptr;
    cudaGraphExec_t apply_exec = nullptr;
    const void *apply_key[2] = {nullptr, nullptr};
    std::vector<Layer> layers;
    size_t nw = 0, nb = 0;   // padded parameter counts
    float *w32 = nullptr, *b32 = nullptr, *gw = nullptr, *gb = nullptr;
    float *mw = nullptr, *vw = nullptr, *mb = nullptr, *vb = nullptr;
    bf16 *w16 = nullptr;
    int64_t step = 0;
    // activations (bf16) and gradients (fp32), sized for max_batch
    std::vector<void *> bufs;
    bf16 *xin = nullptr;
    std::vector<bf16 *> ya, yb, pool, yu, sadd, yc;
    float *acc = nullptr;               // split-K partial sums of the forward convolutions
    float *out = nullptr;
    float *loss = nullptr;
    float *scale1 = nullptr;            // input scale of surrogate_apply
    float *field1 = nullptr;            // one iteration's field (pixels) in surrogate_apply
    bf16 *ghead = nullptr;
    float *g1 = nullptr, *g2 = nullptr, *g3 = nullptr;  // fp32 gradient scratch (largest tensor)
    std::vector<float *> dskip;
    bf16 *dz = nullptr;
    int64_t cap_elems = 0;   // elements of the largest activation tensor per batch entry
};

namespace {

int find_layer(const dc_surrogate *s, const std::string &name)
{
    for (size_t k = 0; k < s->layers.size(); ++k)
        if (s->layers[k].name == name) return (int)k;
    return -1;
}

// Split-K workspace of the forward convolutions (fp32 partial sums): layers
// whose output has at most this many elements may split K.
constexpr size_t kSplitAccElems = (size_t)320 * BM * BN;

// y = act(conv(x) + bias) (bf16), optionally the decoder skip sum
// sadd = bf16(y + skip) and the fp32 head output yf.  up: x at half
// resolution, upsampled in the loader.  Layers with fewer than two CTA tiles
// per SM split K and finish in conv_finalize_kernel.
cudaError_t conv_forward(dc_surrogate *s, const Layer &L, const bf16 *x, int B, bf16 *y, float *yf, int relu,
                         int up = 0, const bf16 *skip = nullptr, bf16 *sadd = nullptr)
{
    ConvFwd p;
    p.M = B << (2 * L.log2H);
    p.N = L.cout_p;
    p.K = 9 * L.cin_p;
    p.log2H = L.log2H;
    p.cin_p = L.cin_p;
    p.cout_p = L.cout_p;
    p.lg_cin = 31 - __builtin_clz((unsigned)L.cin_p);
    p.up = up;
    p.X = x;
    p.W = s->w16 + L.woff;
    p.out.cout_p = L.cout_p;
    p.out.out_ch = L.cout;
    p.out.relu = relu;
    p.out.bias = s->b32 + L.boff;
    p.out.Y = y;
    p.out.skip = skip;
    p.out.S = sadd;
    p.out.Yf = yf;
    p.acc = nullptr;
    // tcgen05 for 64..256 output channels (DC_SG_AUTO: in batches of two or
    // more samples, where it measured faster: 2.10 against 2.21 ms for the
    // forward at batch 16; mma.sync at batch 1, 0.29 against 0.30 ms); the
    // 32-channel full-resolution layers are loader-bound and faster on the
    // 64 x 32 mma.sync tiles
    const bool tc = s->tc_path == DC_SG_TCGEN05 || (s->tc_path == DC_SG_AUTO && B >= 2);
    const bool um = tc && (p.N == 64 || p.N == 128 || p.N == 256) && p.M % UM_TM == 0;
    const int tm = um ? UM_TM : BM, tk = um ? UM_TK : BK;
    const int tiles = ((p.M + tm - 1) / tm) * (um ? 1 : (p.N + BN - 1) / BN);
    const int ksteps = (p.K + tk - 1) / tk;
    const int min_steps = um ? 2 : 8;  // k-steps a split at least
    int splits = 1;
    const int sms = device_sms();
    if (tiles < 2 * sms && (size_t)p.M * p.N <= kSplitAccElems) {
        splits = (2 * sms + tiles - 1) / tiles;
        if (splits > ksteps / min_steps) splits = ksteps / min_steps;
        if (splits < 1) splits = 1;
    }
    cudaError_t e = cudaSuccess;
    if (splits > 1) {
        e = cudaMemsetAsync(s->acc, 0, (size_t)p.M * p.N * sizeof(float), s->stream);
        if (e != cudaSuccess) return e;
        p.acc = s->acc;
    }
    if (um) {
        int kps = (p.K + splits - 1) / splits;
        kps = (kps + UM_TK - 1) / UM_TK * UM_TK;
        const int sp = (p.K + kps - 1) / kps;
        CUtensorMap tmB;
        const int use_tma = weights_map(&tmB, p.W, p.N, p.K) ? 1 : 0;
        e = launch_kernel(umma_gemm_kernel<ConvFwd>, dim3(p.M / UM_TM, 1, sp), dim3(UM_THREADS), umma_smem_bytes(p.N),
                          s->stream, p, kps, s->status, tmB, use_tma);
    } else {
        e = run_gemm(s->stream, p, splits);
    }
    if (e != cudaSuccess || splits <= 1) return e;
    const int64_t pairs = (int64_t)p.M * (p.N / 2);
    return launch_kernel(conv_finalize_kernel, dim3(eb(pairs)), dim3(256), 0, s->stream, (const float *)s->acc,
                         (int64_t)p.M, p.N, p.out);
}

cudaError_t conv_backward(dc_surrogate *s, const Layer &L, const bf16 *x, const bf16 *dz, int B, float *dx,
                          int up = 0)
{
    const int64_t P = (int64_t)B << (2 * L.log2H);
    ConvWgrad w;
    w.M = L.cout_p;
    w.N = 9 * L.cin_p;
    w.K = (int)P;
    w.log2H = L.log2H;
    w.cin_p = L.cin_p;
    w.cout_p = L.cout_p;
    w.up = up;
    w.dZ = dz;
    w.X = x;
    w.dW = s->gw + L.woff;
    // the reduction over P pixels is split to ~8 CTAs a SM (7 fit at 68
    // registers and 18 KB): the tiles are few and each k-step is latency-bound
    // (2 a SM measured 8.97 ms a training step at batch 16, 8 a SM 7.55 ms)
    const int tiles = ((w.M + BM - 1) / BM) * ((w.N + BN - 1) / BN);
    int splits = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)8 * device_sms() + tiles - 1) / tiles, P / (4 * BK)));
    cudaError_t e = run_gemm(s->stream, w, splits);
    if (e != cudaSuccess) return e;
    const int64_t chunk = 256;
    e = launch_kernel(bias_grad_kernel, dim3((unsigned)((P + chunk - 1) / chunk)), dim3(L.cout_p), 0, s->stream, dz, P,
                      L.cout_p, chunk, s->gb + L.boff);
    if (e != cudaSuccess || !dx) return e;
    ConvBwdData d;
    d.M = (int)P;
    d.N = L.cin_p;
    d.K = 9 * L.cout_p;
    d.log2H = L.log2H;
    d.cin_p = L.cin_p;
    d.cout_p = L.cout_p;
    d.dZ = dz;
    d.W = s->w16 + L.woff;
    d.dX = dx;
    return run_gemm(s->stream, d);
}

cudaError_t forward_pass(dc_surrogate *s, const float *dens, const float *scales, const float *field, int B)
{
    const int L = s->levels;
    const int64_t P0 = (int64_t)B << (2 * s->log2H);
    if (s->in_channels < 3) field = nullptr;
    cudaError_t e = launch_kernel(pack_input_kernel, dim3(eb(P0 * 8)), dim3(256), 0, s->stream, dens, scales, field,
                                  2 * s->log2H, P0, s->xin);
    const bf16 *h = s->xin;
    for (int l = 0; l < L && e == cudaSuccess; ++l) {
        const Layer &La = s->layers[find_layer(s, "enc" + std::to_string(l) + "a")];
        const Layer &Lb = s->layers[find_layer(s, "enc" + std::to_string(l) + "b")];
        e = conv_forward(s, La, h, B, s->ya[l], nullptr, 1);
        if (e == cudaSuccess) e = conv_forward(s, Lb, s->ya[l], B, s->yb[l], nullptr, 1);
        if (e == cudaSuccess && l < L - 1) {
            const int64_t tot = ((int64_t)B << (2 * (La.log2H - 1))) * La.cout_p;
            e = launch_kernel(avgpool_kernel, dim3(eb(tot)), dim3(256), 0, s->stream, (const bf16 *)s->yb[l],
                              La.log2H - 1, La.cout_p, tot, s->pool[l]);
            h = s->pool[l];
        }
    }
    h = s->yb[L - 1];
    for (int l = L - 2; l >= 0 && e == cudaSuccess; --l) {
        const Layer &Lu = s->layers[find_layer(s, "dec" + std::to_string(l) + "up")];
        const Layer &Lc = s->layers[find_layer(s, "dec" + std::to_string(l) + "c")];
        // conv of the upsampled coarser output; the epilogue also forms the
        // skip sum yu + yb[l] that the next convolution reads
        e = conv_forward(s, Lu, h, B, s->yu[l], nullptr, 1, 1, s->yb[l], s->sadd[l]);
        if (e == cudaSuccess) e = conv_forward(s, Lc, s->sadd[l], B, s->yc[l], nullptr, 1);
        h = s->yc[l];
    }
    if (e == cudaSuccess) e = conv_forward(s, s->layers.back(), h, B, nullptr, s->out, 0);
    if (e == cudaSuccess && field && s->kappa != 0.f)
        e = launch_kernel(add_skip_kernel, dim3(eb(P0 * 2)), dim3(256), 0, s->stream, s->out, field, s->kappa, P0 * 2);
    return e;
}

cudaError_t backward_pass(dc_surrogate *s, const float *target, int B)
{
    const int L = s->levels;
    const int64_t P0 = (int64_t)B << (2 * s->log2H);
    cudaError_t e = cudaMemsetAsync(s->gw, 0, s->nw * sizeof(float), s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->gb, 0, s->nb * sizeof(float), s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->loss, 0, sizeof(float), s->stream);
    if (e == cudaSuccess)
        e = launch_kernel(loss_kernel, dim3(eb(P0 * 8)), dim3(256), 0, s->stream, (const float *)s->out, target, P0,
                          1.0f / (float)(P0 * 2), s->loss, s->ghead);
    // head
    const Layer &Lh = s->layers.back();
    const bf16 *head_in = L >= 2 ? s->yc[0] : s->yb[0];
    float *dh = s->g1;
    if (e == cudaSuccess) e = conv_backward(s, Lh, head_in, s->ghead, B, dh);
    // decoder, in reverse order of the forward pass
    for (int l = 0; l <= L - 2 && e == cudaSuccess; ++l) {
        const Layer &Lu = s->layers[find_layer(s, "dec" + std::to_string(l) + "up")];
        const Layer &Lc = s->layers[find_layer(s, "dec" + std::to_string(l) + "c")];
        const int64_t nc = ((int64_t)B << (2 * Lc.log2H)) * Lc.cout_p;
        e = launch_kernel(relu_grad_kernel, dim3(eb(nc)), dim3(256), 0, s->stream, (const float *)dh,
                          (const float *)nullptr, (const bf16 *)s->yc[l], nc, s->dz);
        if (e == cudaSuccess) e = conv_backward(s, Lc, s->sadd[l], s->dz, B, s->dskip[l]);
        if (e == cudaSuccess)
            e = launch_kernel(relu_grad_kernel, dim3(eb(nc)), dim3(256), 0, s->stream, (const float *)s->dskip[l],
                              (const float *)nullptr, (const bf16 *)s->yu[l], nc, s->dz);
        float *du = s->g2;
        const bf16 *coarse = l == L - 2 ? s->yb[L - 1] : s->yc[l + 1];  // dec{l}up's input, before upsampling
        if (e == cudaSuccess) e = conv_backward(s, Lu, coarse, s->dz, B, du, 1);
        const int64_t tot = ((int64_t)B << (2 * (Lu.log2H - 1))) * Lu.cin_p;
        if (e == cudaSuccess)
            e = launch_kernel(upsample_bwd_kernel, dim3(eb(tot)), dim3(256), 0, s->stream, (const float *)du,
                              Lu.log2H - 1, Lu.cin_p, tot, s->g1);
        dh = s->g1;
    }
    // encoder
    for (int l = L - 1; l >= 0 && e == cudaSuccess; --l) {
        const Layer &La = s->layers[find_layer(s, "enc" + std::to_string(l) + "a")];
        const Layer &Lb = s->layers[find_layer(s, "enc" + std::to_string(l) + "b")];
        const int64_t nb_ = ((int64_t)B << (2 * Lb.log2H)) * Lb.cout_p;
        e = launch_kernel(relu_grad_kernel, dim3(eb(nb_)), dim3(256), 0, s->stream, (const float *)dh,
                          (const float *)(l <= L - 2 ? s->dskip[l] : nullptr), (const bf16 *)s->yb[l], nb_, s->dz);
        float *dya = s->g2;
        if (e == cudaSuccess) e = conv_backward(s, Lb, s->ya[l], s->dz, B, dya);
        if (e == cudaSuccess)
            e = launch_kernel(relu_grad_kernel, dim3(eb(nb_)), dim3(256), 0, s->stream, (const float *)dya,
                              (const float *)nullptr, (const bf16 *)s->ya[l], nb_, s->dz);
        const bf16 *in = l == 0 ? s->xin : s->pool[l - 1];
        float *dx = l > 0 ? s->g3 : nullptr;
        if (e == cudaSuccess) e = conv_backward(s, La, in, s->dz, B, dx);
        if (e == cudaSuccess && l > 0) {
            const int64_t tot = ((int64_t)B << (2 * (La.log2H + 1))) * La.cin_p;
            e = launch_kernel(avgpool_bwd_kernel, dim3(eb(tot)), dim3(256), 0, s->stream, (const float *)s->g3,
                              La.log2H + 1, La.cin_p, tot, s->g1);
            dh = s->g1;
        }
    }
    return e;
}

dc_status check_sg(const dc_surrogate *s)
{
    if (!s) return sfail(DC_ERR_INVALID_ARG, "null surrogate");
    return DC_OK;
}

struct SgGuard {
    int prev = -1;
    bool changed = false;
    explicit SgGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
    }
    ~SgGuard()
    {
        if (changed) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

dc_status surrogate_create(int32_t log2_res, int32_t levels, int32_t base_channels, int32_t in_channels,
                           int32_t max_batch, uint64_t seed, int device, void *cuda_stream, dc_surrogate **out)
{
    if (!out) return sfail(DC_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    if (in_channels != 1 && in_channels != 3) return sfail(DC_ERR_INVALID_ARG, "in_channels = %d", in_channels);
    if (levels < 1 || levels > 6 || base_channels < 8 || base_channels > 256 || (base_channels & 7))
        return sfail(DC_ERR_INVALID_ARG, "levels = %d, base_channels = %d", levels, base_channels);
    if (log2_res < levels + 2 || log2_res > 11) return sfail(DC_ERR_INVALID_ARG, "log2_res = %d", log2_res);
    if (max_batch < 1 || max_batch > 256) return sfail(DC_ERR_INVALID_ARG, "max_batch = %d", max_batch);
    SgGuard guard(device);
    dc_surrogate *s = new dc_surrogate();
    s->levels = levels;
    s->c0 = base_channels;
    s->in_channels = in_channels;
    s->tc_path = DC_SG_AUTO;
    s->log2H = log2_res;
    s->max_batch = max_batch;
    s->device = device;
    auto bail = [&](dc_status st) {
        surrogate_destroy(s);
        return st;
    };
    if (cuda_stream) {
        s->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreate(&s->stream) != cudaSuccess) return bail(sfail(DC_ERR_CUDA, "cudaStreamCreate"));
        s->own_stream = true;
    }
    for (cudaEvent_t &ev : s->ev)
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
            return bail(sfail(DC_ERR_CUDA, "cudaEventCreate"));
    // layers, in the order of the oracle's layer list
    std::vector<int> ch(levels);
    for (int l = 0; l < levels; ++l) ch[l] = base_channels << l;
    auto add = [&](const std::string &name, int co, int ci, int lg) {
        Layer L;
        L.name = name;
        L.cout = co;
        L.cin = ci;
        L.cout_p = round8(co);
        L.cin_p = round8(ci);
        L.log2H = lg;
        L.woff = s->nw;
        L.boff = s->nb;
        s->nw += L.wsize();
        s->nb += L.cout_p;
        s->layers.push_back(L);
    };
    int cin = in_channels;
    for (int l = 0; l < levels; ++l) {
        add("enc" + std::to_string(l) + "a", ch[l], cin, log2_res - l);
        add("enc" + std::to_string(l) + "b", ch[l], ch[l], log2_res - l);
        cin = ch[l];
    }
    for (int l = levels - 2; l >= 0; --l) {
        add("dec" + std::to_string(l) + "up", ch[l], ch[l + 1], log2_res - l);
        add("dec" + std::to_string(l) + "c", ch[l], ch[l], log2_res - l);
    }
    add("head", 2, ch[0], log2_res);
    // parameters: He-normal weights (head scaled by 0.1), zero biases, zero padding
    std::vector<float> w(s->nw, 0.f), b(s->nb, 0.f);
    HostRng rng{seed};
    for (const Layer &L : s->layers) {
        const double std_ = std::sqrt(2.0 / (9.0 * L.cin)) * (L.name == "head" ? 0.1 : 1.0);
        for (int o = 0; o < L.cout; ++o)
            for (int t = 0; t < 9; ++t)
                for (int i = 0; i < L.cin; ++i) w[L.woff + ((size_t)o * 9 + t) * L.cin_p + i] = (float)(std_ * rng.normal());
    }
    const size_t B = (size_t)max_batch;
    const size_t P0 = B << (2 * log2_res);
    auto alloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        s->bufs.push_back(p);
        return p;
    };
    bool ok = true;
    auto A = [&](size_t bytes) {
        void *p = alloc(bytes);
        ok = ok && p;
        return p;
    };
    s->w32 = (float *)A(s->nw * 4);
    s->gw = (float *)A(s->nw * 4);
    s->mw = (float *)A(s->nw * 4);
    s->vw = (float *)A(s->nw * 4);
    s->w16 = (bf16 *)A(s->nw * 2);
    s->b32 = (float *)A(s->nb * 4);
    s->gb = (float *)A(s->nb * 4);
    s->mb = (float *)A(s->nb * 4);
    s->vb = (float *)A(s->nb * 4);
    s->xin = (bf16 *)A(P0 * 8 * 2);
    s->ya.resize(levels);
    s->yb.resize(levels);
    s->pool.resize(levels);
    s->yu.resize(levels);
    s->sadd.resize(levels);
    s->yc.resize(levels);
    s->dskip.resize(levels);
    size_t maxe = P0 * 8;
    for (int l = 0; l < levels; ++l) {
        const size_t Pl = B << (2 * (log2_res - l));
        const size_t e = Pl * (size_t)round8(ch[l]);
        s->ya[l] = (bf16 *)A(e * 2);
        s->yb[l] = (bf16 *)A(e * 2);
        if (l < levels - 1) {
            s->pool[l] = (bf16 *)A(e / 4 * 2);
            s->yu[l] = (bf16 *)A(e * 2);
            s->sadd[l] = (bf16 *)A(e * 2);
            s->yc[l] = (bf16 *)A(e * 2);
            s->dskip[l] = (float *)A(e * 4);
            maxe = std::max(maxe, Pl * (size_t)round8(ch[l + 1]));
        }
        maxe = std::max(maxe, e);
    }
    s->out = (float *)A(P0 * 2 * 4);
    s->acc = (float *)A(kSplitAccElems * 4);
    s->status = (unsigned *)A(4);
    s->loss = (float *)A(4);
    s->scale1 = (float *)A(4);
    s->field1 = (float *)A(((size_t)8 << (2 * log2_res)));
    s->ghead = (bf16 *)A(P0 * 8 * 2);
    s->g1 = (float *)A(maxe * 4);
    s->g2 = (float *)A(maxe * 4);
    s->g3 = (float *)A(maxe * 4);
    s->dz = (bf16 *)A(maxe * 2);
    if (!ok) return bail(sfail(DC_ERR_OOM, "surrogate buffers"));
    if (cudaMemcpy(s->w32, w.data(), s->nw * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(s->b32, b.data(), s->nb * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(s->mw, 0, s->nw * 4) != cudaSuccess || cudaMemset(s->vw, 0, s->nw * 4) != cudaSuccess ||
        cudaMemset(s->mb, 0, s->nb * 4) != cudaSuccess || cudaMemset(s->vb, 0, s->nb * 4) != cudaSuccess ||
        cudaMemset(s->status, 0, 4) != cudaSuccess)
        return bail(sfail(DC_ERR_CUDA, "parameter upload"));
    if (cudaFuncSetAttribute(umma_gemm_kernel<ConvFwd>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)umma_smem_bytes(256)) != cudaSuccess)
        return bail(sfail(DC_ERR_CUDA, "kernel attributes"));
    if (launch_kernel(to_bf16_kernel, dim3(eb((int64_t)s->nw)), dim3(256), 0, s->stream, (const float *)s->w32,
                      (int64_t)s->nw, s->w16) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return bail(sfail(DC_ERR_CUDA, "weight conversion"));
    *out = s;
    return DC_OK;
}

dc_status surrogate_destroy(dc_surrogate *s)
{
    if (!s) return DC_OK;
    SgGuard guard(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (void *p : s->bufs) cudaFree(p);
    for (cudaEvent_t &ev : s->ev)
        if (ev) cudaEventDestroy(ev);
    if (s->apply_exec) cudaGraphExecDestroy(s->apply_exec);
    if (s->cap) cudaStreamDestroy(s->cap);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return DC_OK;
}

// Parameters in the unpadded layout of the oracle: for each layer in order,
// weights [cout][3][3][cin] then, separately, biases [cout].
dc_status surrogate_num_params(const dc_surrogate *s, int64_t *weights, int64_t *biases)
{
    if (dc_status st = check_sg(s)) return st;
    int64_t nw = 0, nb = 0;
    for (const Layer &L : s->layers) {
        nw += (int64_t)L.cout * 9 * L.cin;
        nb += L.cout;
    }
    if (weights) *weights = nw;
    if (biases) *biases = nb;
    return DC_OK;
}

static dc_status copy_params(dc_surrogate *s, float *w_host, float *b_host, const float *wsrc_dev,
                             const float *bsrc_dev)
{
    std::vector<float> w(s->nw), b(s->nb);
    SG_CUDA(cudaStreamSynchronize(s->stream));
    SG_CUDA(cudaMemcpy(w.data(), wsrc_dev, s->nw * 4, cudaMemcpyDeviceToHost));
    SG_CUDA(cudaMemcpy(b.data(), bsrc_dev, s->nb * 4, cudaMemcpyDeviceToHost));
    size_t ow = 0, ob = 0;
    for (const Layer &L : s->layers) {
        for (int o = 0; o < L.cout; ++o)
            for (int t = 0; t < 9; ++t)
                for (int i = 0; i < L.cin; ++i)
                    if (w_host) w_host[ow++] = w[L.woff + ((size_t)o * 9 + t) * L.cin_p + i];
        for (int o = 0; o < L.cout; ++o)
            if (b_host) b_host[ob++] = b[L.boff + o];
    }
    return DC_OK;
}

dc_status surrogate_get_params(dc_surrogate *s, float *w_host, float *b_host)
{
    if (dc_status st = check_sg(s)) return st;
    SgGuard guard(s->device);
    return copy_params(s, w_host, b_host, s->w32, s->b32);
}

dc_status surrogate_get_grads(dc_surrogate *s, float *gw_host, float *gb_host)
{
    if (dc_status st = check_sg(s)) return st;
    SgGuard guard(s->device);
    return copy_params(s, gw_host, gb_host, s->gw, s->gb);
}

dc_status surrogate_set_params(dc_surrogate *s, const float *w_host, const float *b_host)
{
    if (dc_status st = check_sg(s)) return st;
    if (!w_host || !b_host) return sfail(DC_ERR_INVALID_ARG, "null parameters");
    SgGuard guard(s->device);
    std::vector<float> w(s->nw, 0.f), b(s->nb, 0.f);
    size_t ow = 0, ob = 0;
    for (const Layer &L : s->layers) {
        for (int o = 0; o < L.cout; ++o)
            for (int t = 0; t < 9; ++t)
                for (int i = 0; i < L.cin; ++i) w[L.woff + ((size_t)o * 9 + t) * L.cin_p + i] = w_host[ow++];
        for (int o = 0; o < L.cout; ++o) b[L.boff + o] = b_host[ob++];
    }
    SG_CUDA(cudaStreamSynchronize(s->stream));
    SG_CUDA(cudaMemcpy(s->w32, w.data(), s->nw * 4, cudaMemcpyHostToDevice));
    SG_CUDA(cudaMemcpy(s->b32, b.data(), s->nb * 4, cudaMemcpyHostToDevice));
    SG_CUDA(launch_kernel(to_bf16_kernel, dim3(eb((int64_t)s->nw)), dim3(256), 0, s->stream, (const float *)s->w32,
                          (int64_t)s->nw, s->w16));
    s->step = 0;
    SG_CUDA(cudaMemsetAsync(s->mw, 0, s->nw * 4, s->stream));
    SG_CUDA(cudaMemsetAsync(s->vw, 0, s->nw * 4, s->stream));
    SG_CUDA(cudaMemsetAsync(s->mb, 0, s->nb * 4, s->stream));
    SG_CUDA(cudaMemsetAsync(s->vb, 0, s->nb * 4, s->stream));
    return DC_OK;
}

// after a synchronisation: DC_ERR_TIMEOUT if a kernel's bounded wait expired
static dc_status sg_status(dc_surrogate *s)
{
    unsigned st = 0;
    if (cudaMemcpy(&st, s->status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
        return sfail(DC_ERR_CUDA, "status read");
    if (st) {
        cudaMemset(s->status, 0, sizeof(unsigned));
        return sfail((dc_status)st, "device status %u", st);
    }
    return DC_OK;
}

dc_status surrogate_set_skip(dc_surrogate *s, float kappa)
{
    if (dc_status st = check_sg(s)) return st;
    if (!(kappa == kappa)) return sfail(DC_ERR_INVALID_ARG, "kappa is NaN");
    if (kappa != s->kappa && s->apply_exec) {  // the captured forward holds kappa
        SgGuard guard(s->device);
        cudaGraphExecDestroy(s->apply_exec);
        s->apply_exec = nullptr;
    }
    s->kappa = kappa;
    return DC_OK;
}

dc_status surrogate_set_tensor_path(dc_surrogate *sg, int32_t path)
{
    if (dc_status st = check_sg(sg)) return st;
    if (path != DC_SG_MMA_SYNC && path != DC_SG_TCGEN05 && path != DC_SG_AUTO)
        return sfail(DC_ERR_INVALID_ARG, "path = %d", path);
    if (path != sg->tc_path && sg->apply_exec) {  // the captured forward holds the old kernels
        SgGuard guard(sg->device);
        cudaStreamSynchronize(sg->stream);
        cudaGraphExecDestroy(sg->apply_exec);
        sg->apply_exec = nullptr;
    }
    sg->tc_path = path;
    return DC_OK;
}

dc_status surrogate_forward(dc_surrogate *s, const float *density, const float *scales, const float *field,
                            int32_t batch, float *out)
{
    if (dc_status st = check_sg(s)) return st;
    if (!density || batch < 1 || batch > s->max_batch) return sfail(DC_ERR_INVALID_ARG, "density / batch");
    if (s->in_channels == 3 && !field) return sfail(DC_ERR_INVALID_ARG, "field required (in_channels = 3)");
    SgGuard guard(s->device);
    SG_CUDA(forward_pass(s, density, scales, field, batch));
    if (out)
        SG_CUDA(cudaMemcpyAsync(out, s->out, sizeof(float) * 2 * ((size_t)batch << (2 * s->log2H)),
                                cudaMemcpyDeviceToDevice, s->stream));
    return DC_OK;
}

dc_status surrogate_loss_grad(dc_surrogate *s, const float *density, const float *scales, const float *field,
                              const float *target, int32_t batch, float *loss_out)
{
    if (dc_status st = check_sg(s)) return st;
    if (!density || !target || batch < 1 || batch > s->max_batch) return sfail(DC_ERR_INVALID_ARG, "arguments");
    if (s->in_channels == 3 && !field) return sfail(DC_ERR_INVALID_ARG, "field required (in_channels = 3)");
    SgGuard guard(s->device);
    SG_CUDA(forward_pass(s, density, scales, field, batch));
    SG_CUDA(backward_pass(s, target, batch));
    if (loss_out) {
        SG_CUDA(cudaMemcpyAsync(loss_out, s->loss, sizeof(float), cudaMemcpyDeviceToHost, s->stream));
        SG_CUDA(cudaStreamSynchronize(s->stream));
        return sg_status(s);
    }
    return DC_OK;
}

dc_status surrogate_train_step(dc_surrogate *s, const float *density, const float *scales, const float *field,
                               const float *target, int32_t batch, float lr, float *loss_out)
{
    if (dc_status st = surrogate_loss_grad(s, density, scales, field, target, batch, nullptr)) return st;
    SgGuard guard(s->device);
    s->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float bc1 = 1.f - std::pow(b1, (float)s->step), bc2 = 1.f - std::pow(b2, (float)s->step);
    SG_CUDA(launch_kernel(adam_kernel, dim3(eb((int64_t)s->nw)), dim3(256), 0, s->stream, s->w32, (const float *)s->gw,
                          s->mw, s->vw, s->w16, (int64_t)s->nw, lr, b1, b2, eps, bc1, bc2));
    SG_CUDA(launch_kernel(adam_kernel, dim3(eb((int64_t)s->nb)), dim3(256), 0, s->stream, s->b32, (const float *)s->gb,
                          s->mb, s->vb, (bf16 *)nullptr, (int64_t)s->nb, lr, b1, b2, eps, bc1, bc2));
    if (loss_out) {
        SG_CUDA(cudaMemcpyAsync(loss_out, s->loss, sizeof(float), cudaMemcpyDeviceToHost, s->stream));
        SG_CUDA(cudaStreamSynchronize(s->stream));
        return sg_status(s);
    }
    return DC_OK;
}

// Apply the surrogate to samples: density of the samples (the context's
// splat and smoothing), one forward pass, one bilinear move of every sample
// by the predicted field; then plain iterations while the Sec. 6.2 bin
// coefficient of variation is above target_cv (at most max_plain_iters).
dc_status surrogate_apply(dc_ctx *ctx, dc_surrogate *s, float *pos_xy, int64_t n, float target_cv,
                          int32_t max_plain_iters, int32_t *plain_iters_out, double *cv_out)
{
    if (dc_status st = check_sg(s)) return st;
    if (!ctx || (int)ctx->p.log2_res != s->log2H) return sfail(DC_ERR_INVALID_ARG, "context resolution");
    if (n <= 0 || !pos_xy) return sfail(DC_ERR_INVALID_ARG, "samples");
    if (max_plain_iters < 0 || max_plain_iters > 1024) return sfail(DC_ERR_INVALID_ARG, "max_plain_iters (0..1024)");
    if (!(target_cv >= 0.f) || !std::isfinite(target_cv)) return sfail(DC_ERR_INVALID_ARG, "target_cv");
    if (ctx->mode != MODE_FLOAT) return sfail(DC_ERR_INVALID_ARG, "the surrogate takes a smoothed density");
    SgGuard guard(s->device);
    // no host synchronisation until the quality measure: the context's
    // stream and the network's are ordered by events
    if (dc_status st = splat_density(ctx, pos_xy, n, nullptr, nullptr)) return st;
    const int N = 1 << s->log2H;
    if (s->in_channels == 3) {
        // the field of one plain iteration, in pixels
        if (dc_status st = displacement_field(ctx, nullptr)) return st;
        SG_CUDA(launch_kernel(disp_to_field_kernel, dim3(eb((int64_t)N * N)), dim3(256), 0, ctx->stream,
                              (const float2 *)ctx->disp, (int64_t)N * N, (float)N, s->field1));
    }
    SG_CUDA(launch_kernel(set_value_kernel, dim3(1), dim3(1), 0, ctx->stream, s->scale1,
                          (float)((double)N * N / (double)n)));
    SG_CUDA(cudaEventRecord(s->ev[0], ctx->stream));
    SG_CUDA(cudaStreamWaitEvent(s->stream, s->ev[0], 0));
    if (!s->apply_exec || s->apply_key[0] != ctx->dens || s->apply_key[1] != ctx->disp) {
        if (s->apply_exec) {
            cudaGraphExecDestroy(s->apply_exec);
            s->apply_exec = nullptr;
        }
        if (!s->cap) SG_CUDA(cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking));
        cudaStream_t keep = s->stream;
        s->stream = s->cap;
        SG_CUDA(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = forward_pass(s, ctx->dens, s->scale1, s->in_channels == 3 ? s->field1 : nullptr, 1);
        if (e == cudaSuccess)
            e = launch_kernel(field_to_disp_kernel, dim3(eb((int64_t)N * N)), dim3(256), 0, s->cap,
                              (const float *)s->out, (int64_t)N * N, 1.0f / N, ctx->disp);
        cudaGraph_t g = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(s->cap, &g);
        s->stream = keep;
        if (e == cudaSuccess) e = ee;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&s->apply_exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            s->apply_exec = nullptr;
            return sfail(DC_ERR_CUDA, "surrogate_apply graph: %s", cudaGetErrorString(e));
        }
        s->apply_key[0] = ctx->dens;
        s->apply_key[1] = ctx->disp;
    }
    SG_CUDA(cudaGraphLaunch(s->apply_exec, s->stream));
    SG_CUDA(cudaEventRecord(s->ev[1], s->stream));
    SG_CUDA(cudaStreamWaitEvent(ctx->stream, s->ev[1], 0));
    ctx->have_disp = true;
    if (dc_status st = advect_samples(ctx, pos_xy, n)) return st;
    int used = 0;
    double m[3] = {0, 0, 0};
    if (dc_status st = splat_density(ctx, pos_xy, n, nullptr, nullptr)) return st;
    if (dc_status st = quality_metrics(ctx, m)) return st;
    if (m[1] > target_cv && max_plain_iters > 0) {
        // the fallback iterations in one graph launch, stopped on the GPU
        // after the first iteration whose moved samples meet target_cv
        std::vector<double> cvs((size_t)max_plain_iters);
        int32_t done = 0;
        if (dc_status st = regularize_adaptive(ctx, pos_xy, n, max_plain_iters, target_cv > 0.f ? target_cv : 0.0,
                                               0.0, 0.0, &done, cvs.data(), nullptr))
            return st;
        used = done;
        m[1] = cvs[(size_t)done - 1];
    }
    if (plain_iters_out) *plain_iters_out = used;
    if (cv_out) *cv_out = m[1];
    if (dc_status st = declutter_sync(ctx)) return st;
    return sg_status(s);
}

}  // extern "C"
