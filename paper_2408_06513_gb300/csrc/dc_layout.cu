// Layout-level kernels around the iteration: the continuous transition
// between the original and the regularised scatterplot (Sec. 1) and the
// Sec. 6.2 neighbourhood measures of a regularised layout against the
// original one (trustworthiness after Venna and Kaski, orthogonal ordering
// after Misue et al.).
#include "dc_internal.cuh"

namespace dc {

namespace {

constexpr int kThreads = 256;

// out = (1 - s) a + s b, each operation rounded to float32 in that order
// (no contraction), so that s = 0 and s = 1 return a and b exactly.
__device__ __forceinline__ float blend(float a, float b, float one_minus_s, float s)
{
    return __fadd_rn(__fmul_rn(one_minus_s, a), __fmul_rn(s, b));
}

// vec: all three arrays are 16-byte aligned (float4 accesses)
__global__ void __launch_bounds__(kThreads) transition_kernel(const float *__restrict__ a, const float *__restrict__ b,
                                                              int64_t count, float s, float *__restrict__ out, int vec)
{
    pdl_wait();
    const float t = __fsub_rn(1.0f, s);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t c4 = vec ? count / 4 : 0;
    const float4 *a4 = reinterpret_cast<const float4 *>(a);
    const float4 *b4 = reinterpret_cast<const float4 *>(b);
    float4 *o4 = reinterpret_cast<float4 *>(out);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < c4; k += stride) {
        const float4 x = __ldg(a4 + k), y = __ldg(b4 + k);
        o4[k] = make_float4(blend(x.x, y.x, t, s), blend(x.y, y.y, t, s), blend(x.z, y.z, t, s),
                            blend(x.w, y.w, t, s));
    }
    for (int64_t k = 4 * c4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += stride)
        out[k] = blend(a[k], b[k], t, s);
}

// Lattice coordinates of the layout measures: X = rint(float32(x * 65535))
// of x clamped to [0, 1] (NaN -> 0), packed as X << 16 | Y.
__global__ void __launch_bounds__(kThreads) quantise_kernel(const float2 *__restrict__ a, const float2 *__restrict__ b,
                                                            int64_t n, uint32_t *__restrict__ qa,
                                                            uint32_t *__restrict__ qb)
{
    pdl_wait();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const float2 u = a[k], v = b[k];
        auto q = [](float x) {
            const float c = fminf(fmaxf(x, 0.0f), 1.0f);  // fmaxf(NaN, 0) = 0
            return (uint32_t)__float2int_rn(__fmul_rn(c, 65535.0f));
        };
        qa[k] = (q(u.x) << 16) | q(u.y);
        qb[k] = (q(v.x) << 16) | q(v.y);
    }
}

// Ordering key of sample j seen from the query: squared lattice distance,
// ties broken by the index (d2 < 2^33, j < 2^31: the key fits 64 bits).
__device__ __forceinline__ unsigned long long lkey(uint32_t qi, uint32_t qj, uint32_t j)
{
    const int dx = (int)(qi >> 16) - (int)(qj >> 16);
    const int dy = (int)(qi & 0xffffu) - (int)(qj & 0xffffu);
    const unsigned long long d2 = (unsigned long long)((long long)dx * dx) + (unsigned long long)((long long)dy * dy);
    return (d2 << 31) | j;
}

__device__ __forceinline__ int sgn(int v) { return (v > 0) - (v < 0); }

// Keeps the K smallest keys seen by this thread, ascending.
template <int K>
struct TopK {
    unsigned long long v[K];
    __device__ void init()
    {
#pragma unroll
        for (int t = 0; t < K; ++t) v[t] = ~0ull;
    }
    __device__ void push(unsigned long long c)
    {
        if (c >= v[K - 1]) return;
        v[K - 1] = c;
#pragma unroll
        for (int t = K - 1; t > 0; --t) {
            if (v[t] < v[t - 1]) {
                const unsigned long long x = v[t];
                v[t] = v[t - 1];
                v[t - 1] = x;
            }
        }
    }
    // remove the head (the thread's smallest)
    __device__ void pop()
    {
#pragma unroll
        for (int t = 0; t + 1 < K; ++t) v[t] = v[t + 1];
        v[K - 1] = ~0ull;
    }
};

__device__ __forceinline__ unsigned long long block_min_u64(unsigned long long x, unsigned long long *s_red)
{
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
        x = y < x ? y : x;
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) s_red[w] = x;
    __syncthreads();
    if (w == 0) {
        x = l < (int)(blockDim.x >> 5) ? s_red[l] : ~0ull;
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
            x = y < x ? y : x;
        }
        if (l == 0) s_red[32] = x;
    }
    __syncthreads();
    return s_red[32];
}

// The k smallest keys over all samples of one layout, ascending, into out[k]
// (k <= K): each thread keeps its K smallest, then k rounds of a block
// minimum over the threads' heads.
template <int K>
__device__ void knn_keys(const uint32_t *__restrict__ q, int64_t n, int64_t self, int k, unsigned long long *out,
                         unsigned long long *s_red)
{
    TopK<K> top;
    top.init();
    const uint32_t qi = q[self];
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x)
        if (j != self) top.push(lkey(qi, __ldg(q + j), (uint32_t)j));
    for (int r = 0; r < k; ++r) {
        const unsigned long long m = block_min_u64(top.v[0], s_red);
        if (top.v[0] == m && m != ~0ull) top.pop();  // keys are unique: one thread owns it
        if (threadIdx.x == 0) out[r] = m;
    }
    __syncthreads();
}

// One CTA per query sample i:
//   t_term = sum over the new layout's k nearest j that are not among the
//            original layout's k nearest of (rank of j in the original - k);
//   o_term = samples j whose orthogonal order relative to i changed.
template <int K>
__global__ void __launch_bounds__(kThreads) layout_terms_kernel(const uint32_t *__restrict__ qo,
                                                                const uint32_t *__restrict__ qn, int64_t n,
                                                                const uint32_t *__restrict__ queries, int k,
                                                                long long *__restrict__ terms)
{
    __shared__ unsigned long long s_red[33];
    __shared__ unsigned long long s_nn_new[K], s_nn_old[K], s_thr[K];
    __shared__ int s_nthr;
    pdl_wait();
    const int64_t i = queries ? (int64_t)queries[blockIdx.x] : (int64_t)blockIdx.x;
    if (i < 0 || i >= n) {  // checked on the host; never reached
        if (threadIdx.x == 0) terms[2 * blockIdx.x] = terms[2 * blockIdx.x + 1] = -1;
        return;
    }
    // orthogonal ordering (every j; j = i keeps its zero signs)
    const uint32_t oi = qo[i], ni = qn[i];
    const int oix = (int)(oi >> 16), oiy = (int)(oi & 0xffffu), nix = (int)(ni >> 16), niy = (int)(ni & 0xffffu);
    unsigned long long bad = 0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        const uint32_t a = __ldg(qo + j), b = __ldg(qn + j);
        const bool keep = sgn(oix - (int)(a >> 16)) == sgn(nix - (int)(b >> 16)) &&
                          sgn(oiy - (int)(a & 0xffffu)) == sgn(niy - (int)(b & 0xffffu));
        bad += keep ? 0 : 1;
    }
    // k nearest in both layouts
    knn_keys<K>(qn, n, i, k, s_nn_new, s_red);
    knn_keys<K>(qo, n, i, k, s_nn_old, s_red);
    if (threadIdx.x == 0) {
        // the new neighbours missing from the original neighbourhood, with
        // their original-layout keys as rank thresholds
        int m = 0;
        for (int r = 0; r < k; ++r) {
            const uint32_t j = (uint32_t)(s_nn_new[r] & 0x7fffffffu);
            bool found = false;
            for (int t = 0; t < k; ++t) found |= (uint32_t)(s_nn_old[t] & 0x7fffffffu) == j;
            if (!found) s_thr[m++] = lkey(oi, qo[j], j);
        }
        s_nthr = m;
    }
    __syncthreads();
    const int m = s_nthr;
    // rank - 1 of each threshold: the samples (other than i) with a smaller key
    unsigned long long below[K];
#pragma unroll
    for (int t = 0; t < K; ++t) below[t] = 0;
    if (m > 0) {
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
            if (j == i) continue;
            const unsigned long long kj = lkey(oi, __ldg(qo + j), (uint32_t)j);
#pragma unroll
            for (int t = 0; t < K; ++t)
                if (t < m && kj < s_thr[t]) ++below[t];
        }
    }
    long long tsum = 0;
#pragma unroll
    for (int t = 0; t < K; ++t) tsum += (long long)below[t];  // sum of (rank - 1) over the thresholds
    // block sums (warp shuffles, then shared memory)
    for (int o = 16; o > 0; o >>= 1) {
        tsum += __shfl_down_sync(0xffffffffu, tsum, o);
        bad += __shfl_down_sync(0xffffffffu, bad, o);
    }
    __shared__ long long s_t[kThreads / 32], s_b[kThreads / 32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        s_t[w] = tsum;
        s_b[w] = (long long)bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long T = 0, B = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            T += s_t[q];
            B += s_b[q];
        }
        // sum over thresholds of (rank - k) = sum of (rank - 1) - m (k - 1)
        terms[2 * blockIdx.x] = T - (long long)m * (k - 1);
        terms[2 * blockIdx.x + 1] = B;
    }
}

// ------------------------------------------------------------------------
// Stopping criteria of Sec. 4.3 step 4 inside one graph launch
// ------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void adapt_start_kernel(AdaptState *st)
{
    pdl_wait();
    st->t0 = global_ns();
    st->iters = 0;
}

// One thread.  The Sec. 6.2 measure from the accumulators of the grid the
// iteration splatted its moved samples into (the same double arithmetic as
// the host's read-back), the largest move in pixels, the elapsed time; the
// next iteration runs only while no criterion holds.
__global__ void adapt_check_kernel(const unsigned long long *qacc, const unsigned *dmax, AdaptState *st, double *cv,
                                   double *move_px, int it, int log2N, cudaGraphConditionalHandle next, int has_next)
{
    pdl_wait();
    const double B = (double)((1 << log2N) / 4);
    const double nbins = B * B;
    const double n = (double)qacc[2];
    const double mean = n / nbins;
    double var = (double)qacc[0] / nbins - mean * mean;
    if (var < 0.0) var = 0.0;
    const double sd = sqrt(var);
    const double c = mean > 0.0 ? sd / mean : 0.0;
    const double mv = (double)sqrtf(__uint_as_float(dmax[it])) * (double)(1 << log2N);
    cv[it] = c;
    move_px[it] = mv;
    st->iters = it + 1;
    const double el = (double)(global_ns() - st->t0);
    const bool stop = (st->target_cv > 0.0 && c <= st->target_cv) || (st->min_move_px > 0.0 && mv <= st->min_move_px) ||
                      (st->max_ns > 0.0 && el >= st->max_ns);
    if (has_next) cudaGraphSetConditional(next, stop ? 0u : 1u);
}

int grid_for(int64_t n, int max_blocks)
{
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

}  // namespace

cudaError_t launch_transition(cudaStream_t s, const float *a, const float *b, int64_t count, float t, float *out)
{
    if (count <= 0) return cudaSuccess;
    const int vec = ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) |
                      reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    return launch_kernel(transition_kernel, dim3(grid_for((count + 3) / 4, device_sms() * 8)), dim3(kThreads), 0, s,
                         a, b, count, t, out, vec);
}

cudaError_t launch_adapt_start(cudaStream_t s, AdaptState *st)
{
    return launch_kernel(adapt_start_kernel, dim3(1), dim3(1), 0, s, st);
}

cudaError_t launch_adapt_check(cudaStream_t s, const unsigned long long *qacc, const unsigned *dmax, AdaptState *st,
                               double *cv, double *move_px, int it, int log2N, cudaGraphConditionalHandle next,
                               int has_next)
{
    return launch_kernel(adapt_check_kernel, dim3(1), dim3(1), 0, s, qacc, dmax, st, cv, move_px, it, log2N, next,
                         has_next);
}

cudaError_t launch_layout_terms(cudaStream_t s, const float2 *orig, const float2 *reg, int64_t n,
                                const uint32_t *queries, int n_queries, int k, uint32_t *qo, uint32_t *qn,
                                long long *terms)
{
    cudaError_t e = launch_kernel(quantise_kernel, dim3(grid_for(n, device_sms() * 8)), dim3(kThreads), 0, s, orig,
                                  reg, n, qo, qn);
    if (e != cudaSuccess) return e;
    const dim3 grid(n_queries);
    if (k <= 8)
        return launch_kernel(layout_terms_kernel<8>, grid, dim3(kThreads), 0, s, (const uint32_t *)qo,
                             (const uint32_t *)qn, n, queries, k, terms);
    if (k <= 16)
        return launch_kernel(layout_terms_kernel<16>, grid, dim3(kThreads), 0, s, (const uint32_t *)qo,
                             (const uint32_t *)qn, n, queries, k, terms);
    return launch_kernel(layout_terms_kernel<32>, grid, dim3(kThreads), 0, s, (const uint32_t *)qo,
                         (const uint32_t *)qn, n, queries, k, terms);
}

}  // namespace dc
