// Grid kernels: Gaussian smoothing (Sec. 4.1), the integral images of
// Sec. 3.1 and the defect-corrected displacement of eq. (map_res).
//
// Integral images by full-width row bands.  With P(j, c) the row prefix of
// row j (P(j, -1) = 0, P(j, c >= N) = row total), every quantity the mapping
// needs is a running sum of P down one of three line families:
//   alpha(i, j) = sum_{j' <= j} P(j', i)                    (vertical)
//   U(i, j)     = sum_{j' <= j} P(j', i + j - j')           (anti-diagonal)
//   V(i, j)     = sum_{j' <= j} P(j', i - j + j' - 1)       (diagonal)
//   alpha_t = U - V  (the clipped upward cone, Sec. 3.1).
// Inside a band each of the three is a one-row recurrence
//   a(i, j) = a(i, j-1) + P(j, i)
//   U(i, j) = U(i+1, j-1) + P(j, i)
//   V(i, j) = V(i-1, j-1) + P(j, i-1)
// and the rows above the band enter as carries, one value per line: the band
// kernels are run twice (aggregate, then final), with an exclusive scan of
// the per-band aggregates over bands in between.  A band's aggregate along
// every line follows from the recurrence state at its last row plus one value
// per row at its left and right edges (compact form, 3N + 2T + 1 values).
//
// The marginals R(i) = alpha(i, N-1), Cc(j) = alpha(N-1, j),
// A(u) = sum over i'+j' <= u, B(v) = sum over i'-j' >= v and the total C give
// beta, gamma, delta and their tilted versions from alpha and alpha_t
// (Sec. 3.1 partition identities; Fig. 2 caption).
#include "dc_internal.cuh"

namespace dc {

BandGeom make_band_geom(int log2N, int band_rows, int sms)
{
    BandGeom g;
    g.log2N = log2N;
    g.N = 1 << log2N;
    g.sms = sms > 0 ? sms : 1;
    int T = band_rows;
    if (T <= 0) {
        // from 1024^2 one band for each SM (the last one shorter); below,
        // N / 256 rows (2 at 512^2: measured 2.6 % faster than 4)
        T = g.N >= 1024 ? (g.N + g.sms - 1) / g.sms : g.N / 256;
        if (T < 1) T = 1;
        if (T > 64) T = 64;
    }
    g.T = T;
    g.nb = (g.N + T - 1) / T;  // band b: rows [b T, min(N, b T + T))
    // at most 512 threads per band CTA (128 registers a thread)
    g.CPT = g.N >= 128 ? (g.N / 512 > 4 ? g.N / 512 : 4) : 1;
    g.NT = g.N / g.CPT;
    if (g.NT < 32) g.NT = 32;
    g.agg_stride = (3 * g.N + 2 * T + 2 + 3) & ~3;  // + the 64-bit-band flag
    g.lanes = 5 * g.N;
    return g;
}

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Carry layout: band b < nb keeps the lanes its final pass reads, at
// b * carry_stride: [vertical N][anti-diagonal window N + T - 1]
// [diagonal window N + T - 1], the windows starting at lines u = j0 and
// v = -(j0 + T - 1); row nb (at nb * carry_stride) keeps all 5N lanes of
// the totals (the marginals).
__host__ __device__ __forceinline__ int carry_stride(int N, int T) { return (3 * N + 2 * T - 2 + 3) & ~3; }

// shared memory the fused smoothing-aggregate kernel may use
constexpr size_t kSmoothAggSmemMax = 200 * 1024;

// ------------------------------------------------------------------------
// Smoothing: one 2D tile per CTA with a halo of r on each side, vertical
// then horizontal pass in shared memory; reflect border (-1 -> 0, N -> N-1).
// ------------------------------------------------------------------------
__device__ __forceinline__ int reflect_index(int k, int N)
{
    return k < 0 ? -1 - k : (k >= N ? 2 * N - 1 - k : k);
}

__global__ void __launch_bounds__(256) smooth_kernel(const uint32_t *__restrict__ counts,
                                                     float *__restrict__ dens, int log2N, GaussW w,
                                                     uint32_t *__restrict__ zero_out)
{
    extern __shared__ float s_sm[];
    const int N = 1 << log2N;
    const int TW = N < 32 ? N : 32;
    const int r = w.r;
    const int W = TW + 2 * r;
    float *s_in = s_sm;          // W x W
    float *s_mid = s_sm + W * W; // TW x W
    const int ox = blockIdx.x * TW, oy = blockIdx.y * TW;
    const int tid = threadIdx.x;
    pdl_wait();
    for (int idx = tid; idx < W * W; idx += blockDim.x) {
        const int yy = idx / W, xx = idx - yy * W;
        const int gy = reflect_index(oy + yy - r, N), gx = reflect_index(ox + xx - r, N);
        s_in[idx] = (float)counts[((size_t)gy << log2N) + gx];
    }
    __syncthreads();
    for (int idx = tid; idx < TW * W; idx += blockDim.x) {
        const int y = idx / W, xx = idx - y * W;
        float s = 0.0f;
        for (int k = 0; k <= 2 * r; ++k) s += w.g[k] * s_in[(y + k) * W + xx];
        s_mid[idx] = s;
    }
    __syncthreads();
    for (int idx = tid; idx < TW * TW; idx += blockDim.x) {
        const int y = idx / TW, x = idx - y * TW;
        float s = 0.0f;
        for (int k = 0; k <= 2 * r; ++k) s += w.g[k] * s_mid[y * W + x + k];
        dens[((size_t)(oy + y) << log2N) + ox + x] = s;
        if (zero_out) zero_out[((size_t)(oy + y) << log2N) + ox + x] = 0u;
    }
}

// R consecutive outputs of a 1-D Gaussian pass: acc[k] = sum over taps t
// (ascending) of g[t] x(k + t), one fused multiply-add each, x(i) = load(i)
// for i in [0, R + 2r).  RAD >= 0 is the radius known at compile time: the
// taps are fully unrolled, each weight an operand straight from the kernel
// parameters and every input loaded once into registers; RAD < 0 slides a
// register window through a loop over the runtime radius r.  Both sum in
// the same order, so they give identical results.
template <int R, int RAD, typename Load>
__device__ __forceinline__ void gauss_window(const GaussW &w, int r, Load load, float (&acc)[R])
{
#pragma unroll
    for (int k = 0; k < R; ++k) acc[k] = 0.0f;
    if constexpr (RAD >= 0) {
        float x[R + 2 * RAD];
#pragma unroll
        for (int i = 0; i < R + 2 * RAD; ++i) x[i] = load(i);
#pragma unroll
        for (int t = 0; t <= 2 * RAD; ++t)
#pragma unroll
            for (int k = 0; k < R; ++k) acc[k] = fmaf(w.g[t], x[k + t], acc[k]);
    } else {
        float win[R];
#pragma unroll
        for (int k = 0; k + 1 < R; ++k) win[k + 1] = load(k);
#pragma unroll R
        for (int t = 0; t <= 2 * r; ++t) {
#pragma unroll
            for (int k = 0; k + 1 < R; ++k) win[k] = win[k + 1];
            win[R - 1] = load(t + R - 1);
            const float g = w.g[t];
#pragma unroll
            for (int k = 0; k < R; ++k) acc[k] = fmaf(g, win[k], acc[k]);
        }
    }
}

// The same smoothing with register sliding windows: each thread computes R
// consecutive outputs of a column (vertical pass) or of a row (horizontal
// pass), loading R + 2r values instead of R (2r + 1).  Taps are summed in
// the same order as smooth_kernel, one fused multiply-add each, so the two
// kernels give identical results.  TS x TS outputs per CTA; the vertical
// pass's output rows are padded to an odd stride so that the horizontal
// pass's lanes (one row each) read conflict-free.
template <int TS, int R, int RAD>
__device__ __forceinline__ void smooth_win_body(const uint32_t *__restrict__ counts, float *__restrict__ dens,
                                                int log2N, const GaussW &w, uint32_t *__restrict__ zero_out)
{
    extern __shared__ float s_sm[];
    const int N = 1 << log2N;
    const int r = w.r;
    const int W = TS + 2 * r;
    const int Wp = W | 1;
    float *s_in = s_sm;           // W x W
    float *s_mid = s_sm + W * W;  // TS x Wp
    const int ox = blockIdx.x * TS, oy = blockIdx.y * TS;
    const int tid = threadIdx.x;
    pdl_wait();
    {
        const int lane = tid & 31, nwarp = blockDim.x >> 5;
        for (int yy = tid >> 5; yy < W; yy += nwarp) {
            const uint32_t *crow = counts + ((size_t)reflect_index(oy + yy - r, N) << log2N);
            for (int xx = lane; xx < W; xx += 32) s_in[yy * W + xx] = (float)crow[reflect_index(ox + xx - r, N)];
        }
    }
    if (zero_out) {
        for (int idx = tid; idx < TS * TS / 4; idx += blockDim.x) {
            const int y = idx / (TS / 4), x4 = idx - y * (TS / 4);
            *reinterpret_cast<uint4 *>(zero_out + ((size_t)(oy + y) << log2N) + ox + 4 * x4) =
                make_uint4(0u, 0u, 0u, 0u);
        }
    }
    __syncthreads();
    // vertical: s_mid[y][xx] = sum_t g[t] s_in[y + t][xx], lanes along xx
    for (int item = tid; item < (TS / R) * W; item += blockDim.x) {
        const int seg = item / W, xx = item - seg * W;
        const int y0 = seg * R;
        const float *col = s_in + y0 * W + xx;
        float acc[R];
        gauss_window<R, RAD>(w, r, [&](int i) { return col[i * W]; }, acc);
#pragma unroll
        for (int k = 0; k < R; ++k) s_mid[(y0 + k) * Wp + xx] = acc[k];
    }
    __syncthreads();
    // horizontal: out[y][x] = sum_t g[t] s_mid[y][x + t], lanes along y
    for (int item = tid; item < TS * (TS / R); item += blockDim.x) {
        const int seg = item / TS, y = item - seg * TS;
        const int x0 = seg * R;
        const float *row = s_mid + y * Wp + x0;
        float acc[R];
        gauss_window<R, RAD>(w, r, [&](int i) { return row[i]; }, acc);
        float *o = dens + ((size_t)(oy + y) << log2N) + ox + x0;
#pragma unroll
        for (int k = 0; k < R; k += 4)
            *reinterpret_cast<float4 *>(o + k) = make_float4(acc[k], acc[k + 1], acc[k + 2], acc[k + 3]);
    }
}
template <int TS, int R, int RAD>
__global__ void __launch_bounds__(256) smooth_win_kernel(const uint32_t *__restrict__ counts,
                                                         float *__restrict__ dens, int log2N, GaussW w,
                                                         uint32_t *__restrict__ zero_out)
{
    smooth_win_body<TS, R, RAD>(counts, dens, log2N, w, zero_out);
}

// ------------------------------------------------------------------------
// Band kernels.
// ------------------------------------------------------------------------
template <int MODE> struct ModeT;
template <> struct ModeT<MODE_COUNT> { using Acc = uint32_t; using In = uint32_t; };
template <> struct ModeT<MODE_FLOAT> { using Acc = float; using In = float; };
template <> struct ModeT<MODE_GRID64> { using Acc = unsigned long long; using In = uint32_t; };

template <int MODE, int CPT>
__device__ __forceinline__ void load_row(const void *src, int log2N, int j, int c0,
                                         float mu, typename ModeT<MODE>::Acc (&v)[CPT])
{
    using Acc = typename ModeT<MODE>::Acc;
    using In = typename ModeT<MODE>::In;
    const int N = 1 << log2N;
    const In *row = static_cast<const In *>(src) + ((size_t)j << log2N);
    In x[CPT];
    if constexpr (CPT % 4 == 0) {
#pragma unroll
        for (int q = 0; q < CPT / 4; ++q) {
            if constexpr (MODE == MODE_FLOAT) {
                const float4 f = *reinterpret_cast<const float4 *>(row + c0 + 4 * q);
                x[4 * q] = f.x; x[4 * q + 1] = f.y; x[4 * q + 2] = f.z; x[4 * q + 3] = f.w;
            } else {
                const uint4 f = *reinterpret_cast<const uint4 *>(row + c0 + 4 * q);
                x[4 * q] = f.x; x[4 * q + 1] = f.y; x[4 * q + 2] = f.z; x[4 * q + 3] = f.w;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < CPT; ++k) x[k] = (c0 + k < N) ? row[c0 + k] : In(0);
    }
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        if constexpr (MODE == MODE_FLOAT) v[k] = (c0 + k < N) ? x[k] - mu : 0.0f;
        else v[k] = (Acc)x[k];
    }
}

// Two-sum accumulation of a float pair (hi, lo) for the compensated carries.
struct F2 { float hi, lo; };
__device__ __forceinline__ F2 f2_add(F2 a, float b)
{
    const float s = a.hi + b;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b - bb);
    return {s, a.lo + e};
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b)
{
    F2 r = f2_add(a, b.hi);
    r.lo += b.lo;
    return r;
}

// Anchor numerators of eq. (map) at grid scale S (position = numerator / S):
// order alpha, beta, gamma, delta, alpha_t, beta_t, gamma_t, delta_t with
// anchors q1, q2, q3, q4, (x,1), (1,y), (x,0), (0,y).  Ties as printed:
// y < x and x + y < 1 tested on the integer numerators.
__device__ __forceinline__ void anchors(int a, int b, int S, int (&qx)[8], int (&qy)[8])
{
    if (b < a) { qx[0] = S; qy[0] = S + b - a; qx[2] = a - b; qy[2] = 0; }
    else       { qx[0] = S - b + a; qy[0] = S; qx[2] = 0; qy[2] = b - a; }
    if (a + b < S) { qx[1] = a + b; qy[1] = 0; qx[3] = 0; qy[3] = a + b; }
    else           { qx[1] = S; qy[1] = a + b - S; qx[3] = a + b - S; qy[3] = S; }
    qx[4] = a; qy[4] = S;
    qx[5] = S; qy[5] = b;
    qx[6] = a; qy[6] = 0;
    qx[7] = 0; qy[7] = b;
}

// Pixel counts of the eight regions for the constant texture 1 (the defect
// t(x, y; d0) of Sec. 4.2 is this mapping, which does not depend on d0).
__device__ __forceinline__ int lattice_A(int u, int N)
{
    return u <= N - 1 ? (u + 1) * (u + 2) / 2 : N * N - (2 * N - 2 - u) * (2 * N - 1 - u) / 2;
}
__device__ __forceinline__ int tri(int m) { return m > 0 ? m * (m + 1) / 2 : 0; }
__device__ __forceinline__ void lattice_counts(int c, int j, int N, int (&w0)[8])
{
    w0[0] = (c + 1) * (j + 1);
    w0[1] = (c + 1) * (N - 1 - j);
    w0[2] = (N - 1 - c) * (N - 1 - j);
    w0[3] = (j + 1) * (N - 1 - c);
    const int at = (j + 1) * (j + 1) - tri(j - (N - 1 - c)) - tri(j - c);
    const int A = lattice_A(c + j, N);
    const int B = lattice_A(N - 1 - c + j, N);
    w0[4] = at;
    w0[5] = A - at;
    w0[6] = N * N - A - B + at;
    w0[7] = B - at;
}

__device__ __forceinline__ double u128_mag_to_double(unsigned long long hi, unsigned long long lo)
{
    return (double)hi * 18446744073709551616.0 + (double)lo;
}

// Exact-mode displacement: w = exact region sums of the counts, C = n.
// M = N^2 sum_k w_k Q_k - C sum_k w0_k Q_k is an exact integer (128 bits),
// D = M / (2 S N^2 (C + d0 N^2)) rounded once.
__device__ __forceinline__ float exact_component(long long A1, long long A0, int log2NN, long long C,
                                                 double inv_den)
{
    const __int128 M = ((__int128)A1 << log2NN) - (__int128)C * (__int128)A0;
    const bool neg = M < 0;
    const unsigned __int128 mag = neg ? (unsigned __int128)(-M) : (unsigned __int128)M;
    const double dm = u128_mag_to_double((unsigned long long)(mag >> 64), (unsigned long long)mag);
    return (float)((neg ? -dm : dm) * inv_den);
}

// Virtual-lens component t - x of eq. (map) at pixel numerator ai (scale S):
// t - x = (X(d - mu) + mu X(1) - 2 Call ai) / (2 S Call) with
// Call = C(d - mu) + mu N^2, i.e. (nx + mu E1 - 2 C(d - mu) ai) * scale where
// E1 = X(1) - 2 N^2 ai = sum_k w0_k q_k - 2 N^2 ai is formed exactly in
// integers: the O(1) pixel position cancels before any float rounding.
__device__ __forceinline__ float lens_component(float nx, const int (&w0)[8], const int (&q)[8], int ai, int log2NN,
                                                float mu, float Cex, float scale)
{
    long long x1 = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) x1 += (long long)w0[k] * q[k];
    const long long e1 = x1 - ((long long)ai << (log2NN + 1));
    return fmaf(-2.0f * Cex, (float)ai, fmaf(mu, (float)e1, nx)) * scale;
}

__device__ __forceinline__ unsigned bits32(float x) { return __float_as_uint(x); }
__device__ __forceinline__ unsigned bits32(uint32_t x) { return x; }

template <typename T, int CPT>
__device__ __forceinline__ void store_row(T *dst, const T (&v)[CPT], int c0, int N)
{
    if constexpr ((CPT * sizeof(T)) % 16 == 0) {
        constexpr int per = 16 / sizeof(T);
#pragma unroll
        for (int q = 0; q < CPT / per; ++q) {
            if constexpr (sizeof(T) == 4) {
                const uint4 f = make_uint4(bits32(v[per * q]), bits32(v[per * q + 1]), bits32(v[per * q + 2]),
                                           bits32(v[per * q + 3]));
                *reinterpret_cast<uint4 *>(dst + c0 + per * q) = f;
            } else {
                ulonglong2 f;
                f.x = (unsigned long long)v[per * q];
                f.y = (unsigned long long)v[per * q + 1];
                *reinterpret_cast<ulonglong2 *>(dst + c0 + per * q) = f;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < CPT; ++k)
            if (c0 + k < N) dst[c0 + k] = v[k];
    }
}

// One band per CTA, thread t owning the CPT contiguous columns
// [t CPT, t CPT + CPT), state in MODE's accumulator type (uint64 for
// MODE_GRID64).  Used for grids below 128 x 128 and, for MODE_GRID64, for
// bands whose sums may reach 2^32 (the interleaved kernels below keep
// band-local sums in 32 bits).  FINAL = false: write the band's compact
// aggregate.  FINAL = true: combine with the carries and evaluate the outputs.
// carry loads: L2 (coherent with stores of other CTAs earlier in the same
// launch, for the fused kernel) or the default cached path
template <bool COH, typename Acc>
__device__ __forceinline__ Acc ld_carry(const Acc *p)
{
    if constexpr (COH) return __ldcg(p);
    else return *p;
}

// A band row from shared memory (float mode, rows of N values, CPT a
// multiple of 4): the same values as load_row reads from the grid.
template <int CPT>
__device__ __forceinline__ void load_row_smem(const float *row, int c0, float mu, float (&v)[CPT])
{
#pragma unroll
    for (int q = 0; q < CPT / 4; ++q) {
        const float4 f = *reinterpret_cast<const float4 *>(row + c0 + 4 * q);
        v[4 * q] = f.x - mu;
        v[4 * q + 1] = f.y - mu;
        v[4 * q + 2] = f.z - mu;
        v[4 * q + 3] = f.w - mu;
    }
}

// Barrier of the threads running band_body: the whole CTA, or (NAMED) the
// first nt threads on barrier 1 while the CTA's other warps have left.
template <bool NAMED>
__device__ __forceinline__ void band_sync(int nt)
{
    if constexpr (NAMED) asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory");
    else __syncthreads();
}

// SROWS: the band's rows come from shared memory (srows, row r of the band at
// srows + r N) instead of a.src, and the first N / CPT threads of the CTA run
// the band (synchronising on barrier 1); float mode, CPT a multiple of 4.
template <int MODE, int CPT, bool FINAL, bool COH = false, bool SROWS = false>
__device__ __forceinline__ void band_body(const BandArgs &a, int log2N, int T, const float *srows = nullptr)
{
    static_assert(!SROWS || (MODE == MODE_FLOAT && CPT % 4 == 0), "shared-memory rows: float mode, CPT % 4 == 0");
    using Acc = typename ModeT<MODE>::Acc;
    const int N = 1 << log2N;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int nthr = SROWS ? N / CPT : (int)blockDim.x;
    const int nw = nthr >> 5;
    const int b = blockIdx.x;
    const int j0 = b * T;
    const int Tb = min(T, N - j0);  // rows of this band (the last one may be shorter)
    const int c0 = t * CPT;

    __shared__ Acc s_wt[2][32];
    __shared__ Acc s_uf[2][32];
    __shared__ Acc s_vl[2][32];
    __shared__ Acc s_U0[64], s_VN[64], s_RT[64];

    pdl_wait();
    Acc arun[CPT], Uo[CPT], Vo[CPT];
#pragma unroll
    for (int k = 0; k < CPT; ++k) { arun[k] = Acc(0); Uo[k] = Acc(0); Vo[k] = Acc(0); }
    Acc RTcum = Acc(0);

    // per-band constants of the final pass
    const Acc *cb = nullptr, *ce = nullptr;
    Acc cvb[CPT], Rk[CPT];
    Acc Ctot = Acc(0), CVbN = Acc(0);
    float kappa = 0.f, scale = 0.f;
    if constexpr (FINAL) {
        cb = static_cast<const Acc *>(a.carry) + (size_t)b * carry_stride(N, T);
        ce = static_cast<const Acc *>(a.carry) + (size_t)((N + T - 1) / T) * carry_stride(N, T);
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            const int c = min(c0 + k, N - 1);
            cvb[k] = ld_carry<COH>(cb + c);
            Rk[k] = ld_carry<COH>(ce + c);
        }
        Ctot = ld_carry<COH>(ce + N - 1);
        CVbN = ld_carry<COH>(cb + N - 1);
        if constexpr (MODE == MODE_FLOAT) {
            const float NN = (float)N * (float)N;
            // the defect's coefficient (the lens keeps t(x, y; d) itself and
            // uses lens_component instead)
            kappa = Ctot / NN;
            const float S = a.pixel_center ? 2.0f * N : (float)N;
            const float Call = Ctot + a.mu * NN + a.d0 * NN;
            scale = Call > 0.0f ? 1.0f / (2.0f * S * Call) : 0.0f;
            // eq. (map) has no value for a density without mass: the lens
            // then writes zero and reports an invalid argument
            if (a.lens && !(Call > 0.0f) && t == 0 && a.status) atomicOr(a.status, (unsigned)DC_ERR_INVALID_ARG);
        }
    }

    Acc vnext[CPT];
    if constexpr (SROWS) load_row_smem<CPT>(srows, c0, a.mu, vnext);
    else load_row<MODE, CPT>(a.src, log2N, j0, c0, a.mu, vnext);
    for (int r = 0; r < Tb; ++r) {
        const int j = j0 + r;
        const int par = r & 1;
        Acc v[CPT];
#pragma unroll
        for (int k = 0; k < CPT; ++k) v[k] = vnext[k];
        if (r + 1 < Tb) {  // prefetch
            if constexpr (SROWS) load_row_smem<CPT>(srows + ((size_t)(r + 1) << log2N), c0, a.mu, vnext);
            else load_row<MODE, CPT>(a.src, log2N, j + 1, c0, a.mu, vnext);
        }
        if constexpr (!FINAL) {
            if (a.zero_out) {
                uint32_t zz[CPT];
#pragma unroll
                for (int k = 0; k < CPT; ++k) zz[k] = 0u;
                store_row<uint32_t, CPT>(a.zero_out + ((size_t)j << log2N), zz, c0, N);
            }
        }

        // neighbour state of the previous row, exchanged before the scan's barrier
        Acc u_next = __shfl_down_sync(kFull, Uo[0], 1);
        Acc v_prev = __shfl_up_sync(kFull, Vo[CPT - 1], 1);
        if (lane == 0) s_uf[par][warp] = Uo[0];
        if (lane == 31) s_vl[par][warp] = Vo[CPT - 1];

        // row prefix P: thread-local, warp, then block
#pragma unroll
        for (int k = 1; k < CPT; ++k) v[k] = v[k] + v[k - 1];
        const Acc tsum = v[CPT - 1];
        Acc x = tsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const Acc y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x = x + y;
        }
        if (lane == 31) s_wt[par][warp] = x;
        band_sync<SROWS>(nthr);
        Acc wv = lane < nw ? s_wt[par][lane] : Acc(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const Acc y = __shfl_up_sync(kFull, wv, o);
            if (lane >= o) wv = wv + y;
        }
        const Acc wexcl = __shfl_sync(kFull, wv, (warp + 31) & 31);
        const Acc total = __shfl_sync(kFull, wv, nw - 1);
        const Acc off = (warp > 0 ? wexcl : Acc(0)) + (x - tsum);
#pragma unroll
        for (int k = 0; k < CPT; ++k) v[k] = v[k] + off;
        if (lane == 31) u_next = (warp + 1 < nw) ? s_uf[par][warp + 1] : Acc(0);
        if (lane == 0) v_prev = (warp > 0) ? s_vl[par][warp - 1] : Acc(0);

        // the three recurrences
        const Acc RTprev = RTcum;
        RTcum = RTcum + total;
        Acc Un[CPT], Vn[CPT];
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            const int c = c0 + k;
            Acc ur = (k + 1 < CPT) ? Uo[k + 1] : u_next;
            if (c == N - 1) ur = RTprev;              // U(N, j-1): row totals only
            Un[k] = ur + v[k];
            Acc vl = (k > 0) ? Vo[k - 1] : v_prev;
            if (c == 0) vl = Acc(0);                  // V(-1, j-1) = 0
            const Acc pm1 = (k > 0) ? v[k - 1] : off; // P(j, c-1)
            Vn[k] = vl + pm1;
            arun[k] = arun[k] + v[k];
        }

        if constexpr (!FINAL) {
            if (t == 0) {
                s_U0[r] = Un[0];
                s_RT[r] = total;
            }
#pragma unroll
            for (int k = 0; k < CPT; ++k)
                if (c0 + k == N - 1) s_VN[r] = Vn[k];
        } else {
            const Acc Ccj = CVbN + RTcum;
            float dxy[2 * CPT];
            Acc oal[CPT], oat[CPT];
            float fal[CPT], fat[CPT];
#pragma unroll
            for (int k = 0; k < CPT; ++k) {
                const int c = c0 + k;
                const int cc = min(c, N - 1);
                const int u = cc + j;
                const int vi = cc - j + N - 1;
                const Acc al = cvb[k] + arun[k];
                const Acc at = (ld_carry<COH>(cb + N + (u - j0)) + Un[k]) -
                               (ld_carry<COH>(cb + 2 * N + T - 1 + (vi - (N - j0 - Tb))) + Vn[k]);
                const Acc A = ld_carry<COH>(ce + N + u);
                const Acc Bv = Ctot - ld_carry<COH>(ce + 3 * N + vi);
                const Acc R = Rk[k];
                Acc w[8];
                w[0] = al;
                w[1] = R - al;
                w[2] = Ctot - R - Ccj + al;
                w[3] = Ccj - al;
                w[4] = at;
                w[5] = A - at;
                w[6] = Ctot - A - Bv + at;
                w[7] = Bv - at;
                oal[k] = al;
                oat[k] = at;
                if constexpr (MODE == MODE_GRID64) {
                    (void)w;
                } else {
                    const int S = a.pixel_center ? 2 * N : N;
                    const int ai = a.pixel_center ? 2 * cc + 1 : cc;
                    const int bj = a.pixel_center ? 2 * j + 1 : j;
                    int qx[8], qy[8], w0[8];
                    anchors(ai, bj, S, qx, qy);
                    lattice_counts(cc, j, N, w0);
                    if constexpr (MODE == MODE_FLOAT) {
                        float nx = 0.f, ny = 0.f, nx0 = 0.f, ny0 = 0.f;
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            nx = fmaf(w[q], (float)qx[q], nx);
                            ny = fmaf(w[q], (float)qy[q], ny);
                            nx0 = fmaf((float)w0[q], (float)qx[q], nx0);
                            ny0 = fmaf((float)w0[q], (float)qy[q], ny0);
                        }
                        if (a.lens) {  // uniform: a launch parameter
                            dxy[2 * k] = lens_component(nx, w0, qx, ai, 2 * log2N, a.mu, Ctot, scale);
                            dxy[2 * k + 1] = lens_component(ny, w0, qy, bj, 2 * log2N, a.mu, Ctot, scale);
                        } else {
                            dxy[2 * k] = fmaf(-kappa, nx0, nx) * scale;
                            dxy[2 * k + 1] = fmaf(-kappa, ny0, ny) * scale;
                        }
                        const float muf = a.mu;
                        fal[k] = al + muf * (float)w0[0];
                        fat[k] = at + muf * (float)w0[4];
                    } else {
                        long long A1x = 0, A1y = 0, A0x = 0, A0y = 0;
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const long long wq = (long long)(uint32_t)w[q];
                            A1x += wq * qx[q];
                            A1y += wq * qy[q];
                            A0x += (long long)w0[q] * qx[q];
                            A0y += (long long)w0[q] * qy[q];
                        }
                        const long long C = (long long)(uint32_t)Ctot;
                        dxy[2 * k] = exact_component(A1x, A0x, 2 * log2N, C, a.inv_den_exact);
                        dxy[2 * k + 1] = exact_component(A1y, A0y, 2 * log2N, C, a.inv_den_exact);
                    }
                }
            }
            const size_t rowoff = (size_t)j << log2N;
            if constexpr (MODE != MODE_GRID64) {
                if (a.disp) {
                    float *dd = reinterpret_cast<float *>(a.disp) + 2 * rowoff;
                    store_row<float, 2 * CPT>(dd, dxy, 2 * c0, 2 * N);
                }
            }
            if constexpr (MODE == MODE_FLOAT) {
                if (a.alpha_out) store_row<float, CPT>(static_cast<float *>(a.alpha_out) + rowoff, fal, c0, N);
                if (a.alpha_t_out) store_row<float, CPT>(static_cast<float *>(a.alpha_t_out) + rowoff, fat, c0, N);
            } else {
                unsigned long long o1[CPT], o2[CPT];
#pragma unroll
                for (int k = 0; k < CPT; ++k) {
                    o1[k] = (unsigned long long)oal[k];
                    o2[k] = (unsigned long long)oat[k];
                }
                if (a.alpha_out)
                    store_row<unsigned long long, CPT>(static_cast<unsigned long long *>(a.alpha_out) + rowoff, o1, c0, N);
                if (a.alpha_t_out)
                    store_row<unsigned long long, CPT>(static_cast<unsigned long long *>(a.alpha_t_out) + rowoff, o2, c0, N);
            }
        }
#pragma unroll
        for (int k = 0; k < CPT; ++k) { Uo[k] = Un[k]; Vo[k] = Vn[k]; }
    }

    if constexpr (!FINAL) {
        // compact aggregate [alpha N][U N][V N][U0 T][E T][S]:
        //   alpha, U, V: recurrence state at the band's last row;
        //   U0[r] = U(0, j0 + r); E[r] = V(N-1, j0 + r) + row totals below row r;
        //   S = band total.
        band_sync<SROWS>(nthr);
        Acc *ag = static_cast<Acc *>(a.agg) + (size_t)b * a.agg_stride;
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            const int c = c0 + k;
            if (c < N) {
                ag[c] = arun[k];
                ag[N + c] = Uo[k];
                ag[2 * N + c] = Vo[k];
            }
        }
        for (int rr = t; rr < Tb; rr += nthr) {
            Acc below = Acc(0);
            for (int q = rr + 1; q < Tb; ++q) below = below + s_RT[q];
            ag[3 * N + rr] = s_U0[rr];
            ag[3 * N + T + rr] = s_VN[rr] + below;
        }
        if (t == 0) ag[3 * N + 2 * T] = RTcum;
    }
}

template <int MODE, int CPT, bool FINAL>
__global__ void __launch_bounds__(CPT == 1 ? 64 : 512) band_kernel(BandArgs a, int log2N, int T)
{
    band_body<MODE, CPT, FINAL>(a, log2N, T);
}

// out-of-line copy for the 64-bit fallback of the interleaved kernels
template <int MODE, int CPT, bool FINAL>
__device__ __noinline__ void band_body_wide(BandArgs a, int log2N, int T)
{
    band_body<MODE, CPT, FINAL>(a, log2N, T);
}

// ------------------------------------------------------------------------
// Smoothing fused into the aggregate pass (float mode, 128^2 .. 1024^2).
// CTA b smooths the rows of its band from the counts (its rows plus r halo
// rows on each side, reflected at the border), writes them to dens for the
// final pass and aggregates the band from shared memory.  The taps are
// summed as in smooth_win_body (vertical, then horizontal, one fused
// multiply-add per tap in tap order), and band_body runs with the same CPT
// as band_kernel, so the densities and aggregates are bit-identical to the
// separate launches'.  The CTA has up to 4x the band's N / CPT threads: all
// of them load and smooth, then the band's threads aggregate while the
// others leave.  Windows of R outputs per thread in both passes; the
// vertical pass's rows are stored at x + x / 32 so that the horizontal
// pass's lanes (R columns apart) read distinct banks.
// ------------------------------------------------------------------------
__device__ __forceinline__ int swz32(int x) { return x + (x >> 5); }

template <int CPT, int R, int RAD>
__global__ void __launch_bounds__(1024) smooth_agg_kernel(BandArgs a, int log2N, int T, GaussW w,
                                                         const uint32_t *__restrict__ counts,
                                                         float *__restrict__ dens, uint32_t *__restrict__ zero_out)
{
    extern __shared__ __align__(16) float s_sa[];
    const int N = 1 << log2N;
    const int r = w.r;
    const int W = N + 2 * r;
    const int j0 = blockIdx.x * T;
    const int Tb = min(T, N - j0);
    const int nseg = (Tb + R - 1) / R;
    const int H = Tb + 2 * r;          // input rows with the halo
    const int Hal = nseg * R + 2 * r;  // rows the R-windows touch (>= H)
    const int Ws = swz32(W - 1) + 1;
    float *s_in = s_sa;                                                // Hal x W
    float *s_mid = s_sa + (size_t)((T + R - 1) / R * R + 2 * r) * W;  // Tb x Ws, swizzled columns
    float *s_rows = s_sa;  // Tb x N (reuses s_in after the vertical pass)
    const int tid = threadIdx.x, nthr = blockDim.x;
    pdl_wait();
    // input rows: the interior by 16-byte loads, eight in flight a thread,
    // the r reflected columns on each side, zeros below row H
    {
        const int q4 = log2N - 2;  // uint4 a row = N / 4
        const int total = Hal << q4;
        for (int base = 0; base < total; base += 8 * nthr) {
            uint4 v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int i = base + k * nthr + tid;
                const int yy = i >> q4;
                v[k] = make_uint4(0u, 0u, 0u, 0u);
                if (i < total && yy < H) {
                    const uint4 *crow = reinterpret_cast<const uint4 *>(
                        counts + ((size_t)reflect_index(j0 + yy - r, N) << log2N));
                    v[k] = crow[i & ((1 << q4) - 1)];
                }
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int i = base + k * nthr + tid;
                if (i < total) {
                    float *d = s_in + (size_t)(i >> q4) * W + r + 4 * (i & ((1 << q4) - 1));
                    d[0] = (float)v[k].x;
                    d[1] = (float)v[k].y;
                    d[2] = (float)v[k].z;
                    d[3] = (float)v[k].w;
                }
            }
        }
        for (int i = tid; i < Hal * 2 * r; i += nthr) {
            const int yy = i / (2 * r), e = i - yy * (2 * r);
            const int xx = e < r ? e : N + e;  // halo columns [0, r) and [N + r, N + 2r)
            float x = 0.0f;
            if (yy < H)
                x = (float)counts[((size_t)reflect_index(j0 + yy - r, N) << log2N) + reflect_index(xx - r, N)];
            s_in[(size_t)yy * W + xx] = x;
        }
    }
    if (zero_out) {
        uint4 *z = reinterpret_cast<uint4 *>(zero_out + ((size_t)j0 << log2N));
        for (int i = tid; i < (Tb << log2N) / 4; i += nthr) z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    // vertical: s_mid[y][xx] = sum_t g[t] s_in[y + t][xx]
    for (int item = tid; item < nseg * W; item += blockDim.x) {
        const int seg = item / W, xx = item - seg * W;
        const int y0 = seg * R;
        const float *col = s_in + (size_t)y0 * W + xx;
        float acc[R];
        gauss_window<R, RAD>(w, r, [&](int i) { return col[(size_t)i * W]; }, acc);
#pragma unroll
        for (int k = 0; k < R; ++k)
            if (y0 + k < Tb) s_mid[(size_t)(y0 + k) * Ws + swz32(xx)] = acc[k];
    }
    __syncthreads();
    // horizontal: d_r[y][x] = sum_t g[t] s_mid[y][x + t]
    const int segs = N / R;
    for (int item = tid; item < Tb * segs; item += blockDim.x) {
        const int y = item / segs, x0 = (item - y * segs) * R;
        const float *row = s_mid + (size_t)y * Ws;
        float acc[R];
        gauss_window<R, RAD>(w, r, [&](int i) { return row[swz32(x0 + i)]; }, acc);
        float *o = dens + ((size_t)(j0 + y) << log2N) + x0;
        float *so = s_rows + ((size_t)y << log2N) + x0;
#pragma unroll
        for (int k = 0; k < R; k += 4) {
            const float4 v = make_float4(acc[k], acc[k + 1], acc[k + 2], acc[k + 3]);
            *reinterpret_cast<float4 *>(o + k) = v;
            *reinterpret_cast<float4 *>(so + k) = v;
        }
    }
    __syncthreads();
    if (tid >= N / CPT) return;  // the band's N / CPT threads go on (barrier 1)
    band_body<MODE_FLOAT, CPT, false, false, true>(a, log2N, T, s_rows);
}

// ------------------------------------------------------------------------
// Band kernels for N >= 128, interleaved column layout.
//
// Thread t of NT = min(512, N / 4) owns G = N / (4 NT) chunks of four
// columns: chunk q covers columns 4 (q NT + t) .. 4 (q NT + t) + 3, so the
// 32 lanes of a warp load and store one chunk's row segment as one
// contiguous run (128- or 256-bit accesses).  The row prefix is a scan of G
// values per thread (one warp scan each, one block barrier per row).
// Rows are prefetched PD rows ahead into registers.
//
// The final pass stages, once per band, every carry and marginal lane the
// band touches into shared memory: the vertical lines [0, N) and the
// anti-diagonal / diagonal windows of N + T - 1 lines.  A window element
// i sits at (i & 3) * L4 + (i >> 2), so that the 32 lanes reading one
// (chunk, column) slot at any row shift hit 32 consecutive words.
//
// MODE_GRID64 keeps its band-local sums in 32 bits: every band-local
// quantity (row prefix, vertical, anti-diagonal and diagonal sums) is at
// most the band total, which is below 2^32 whenever max(grid) T N < 2^32.
// The aggregate pass checks that bound per band and runs the 64-bit body
// for a band that fails it, flagging it in its aggregate record; the final
// pass sends flagged bands to the 64-bit body too.  Carries are 64-bit.
// ------------------------------------------------------------------------
template <int MODE> struct Band2T;
template <> struct Band2T<MODE_COUNT> { using S = uint32_t; using C = uint32_t; };
template <> struct Band2T<MODE_FLOAT> { using S = float; using C = float; };
template <> struct Band2T<MODE_GRID64> { using S = uint32_t; using C = unsigned long long; };

__device__ __forceinline__ int wpos(int i, int L4) { return (i & 3) * L4 + (i >> 2); }

__device__ __forceinline__ uint4 ld_stream_v4(const void *p)
{
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p));
    return r;
}
__device__ __forceinline__ void st_v4_u64(void *p, unsigned long long a, unsigned long long b, unsigned long long c,
                                          unsigned long long d)
{
    asm volatile("st.global.v4.u64 [%0], {%1,%2,%3,%4};" ::"l"(p), "l"(a), "l"(b), "l"(c), "l"(d) : "memory");
}
__device__ __forceinline__ void st_v8_f32(void *p, const float (&v)[8])
{
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]),
                 "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                 : "memory");
}
// four consecutive uint64 at p (16-byte aligned; one 256-bit store when
// 32-byte aligned)
__device__ __forceinline__ void store4_u64(unsigned long long *p, unsigned long long a, unsigned long long b,
                                           unsigned long long c, unsigned long long d, bool al32)
{
    if (al32) {
        st_v4_u64(p, a, b, c, d);
    } else {
        reinterpret_cast<ulonglong2 *>(p)[0] = make_ulonglong2(a, b);
        reinterpret_cast<ulonglong2 *>(p)[1] = make_ulonglong2(c, d);
    }
}

// Row staging by the bulk-copy (TMA) engine: one thread copies a whole row
// into a ring slot of shared memory; the slot's mbarrier completes when the
// bytes have landed.
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long *m)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(m)) : "memory");
}
__device__ __forceinline__ void tma_row(void *dst, const void *src, unsigned bytes, unsigned long long *m)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(m))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long *m, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(m)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for a ring slot: false after one second.
__device__ __noinline__ bool mbar_wait_slow(unsigned long long *m, unsigned parity)
{
    const unsigned long long t0 = global_ns();
    while (!mbar_try(m, parity))
        if (global_ns() - t0 > 1000000000ull) return false;
    return true;
}
__device__ __forceinline__ bool mbar_wait(unsigned long long *m, unsigned parity)
{
    return mbar_try(m, parity) || mbar_wait_slow(m, parity);
}

// RING: rows arrive through a ring of `ring` shared-memory slots filled by
// bulk copies (placed before the carry windows); otherwise each thread
// prefetches its own chunks of the next row into registers.
template <int MODE, int NT, int G, bool FINAL, bool RING>
__global__ void __launch_bounds__(NT) band2_kernel(BandArgs a, int log2N, int T, int ring)
{
    using S = typename Band2T<MODE>::S;
    using C = typename Band2T<MODE>::C;
    constexpr int nw = NT / 32;
    const int N = 4 * NT * G;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int b = blockIdx.x;
    const int j0 = b * T;
    const int Tb = min(T, N - j0);  // rows of this band (the last one may be shorter)

    __shared__ S s_wt[2][G][16];
    __shared__ S s_uf[2][G][16];
    __shared__ S s_vl[2][G][16];
    __shared__ S s_U0[64], s_VN[64], s_RT[64];
    __shared__ unsigned long long s_mbar[8];
    extern __shared__ __align__(128) unsigned char s_dyn[];
    const unsigned rowbytes = 4u << log2N;
    unsigned char *ringp = s_dyn;

    pdl_wait();
    if constexpr (MODE == MODE_GRID64 && FINAL) {
        const unsigned long long *ag = static_cast<const unsigned long long *>(a.agg) + (size_t)b * a.agg_stride;
        if (ag[3 * N + 2 * T + 1]) {
            band_body_wide<MODE_GRID64, 4 * G, true>(a, log2N, T);
            return;
        }
    }

    const unsigned char *src = static_cast<const unsigned char *>(a.src);
    if constexpr (RING) {
        if (t == 0) {
            for (int k = 0; k < ring; ++k) mbar_init(&s_mbar[k]);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (t == 0)
            for (int k = 0; k < ring && k < Tb; ++k)
                tma_row(ringp + (size_t)k * rowbytes, src + (size_t)(j0 + k) * rowbytes, rowbytes, &s_mbar[k]);
    }

    // ---- final pass: stage the band's carry and marginal windows
    const int L4a = ((((N + 3) >> 2) + 23) >> 5 << 5) + 8;
    const int L4w = ((((N + T - 1 + 3) >> 2) + 23) >> 5 << 5) + 8;
    C *sA = nullptr, *sU = nullptr, *sV = nullptr, *sR = nullptr, *sAm = nullptr, *sBm = nullptr;
    C Ctot = C(0), CVbN = C(0);
    float kappa = 0.f, scale = 0.f;
    if constexpr (FINAL) {
        C *p = reinterpret_cast<C *>(s_dyn + (RING ? (size_t)ring * rowbytes : 0));
        sA = p; p += 4 * L4a;
        sU = p; p += 4 * L4w;
        sV = p; p += 4 * L4w;
        if constexpr (MODE != MODE_GRID64) {
            sR = p; p += 4 * L4a;
            sAm = p; p += 4 * L4w;
            sBm = p;
        }
        const C *cb = static_cast<const C *>(a.carry) + (size_t)b * carry_stride(N, T);
        const C *ce = static_cast<const C *>(a.carry) + (size_t)((N + T - 1) / T) * carry_stride(N, T);
        const int ubase = N + j0;               // marginal lane of window element 0: u = j0
        const int vbase = 3 * N + N - j0 - Tb;  // marginal lane of window element 0: v = -(j0 + Tb - 1)
        for (int i = t; i < N; i += NT) {
            sA[wpos(i, L4a)] = cb[i];
            if constexpr (MODE != MODE_GRID64) sR[wpos(i, L4a)] = ce[i];
        }
        for (int i = t; i < N + Tb - 1; i += NT) {
            sU[wpos(i, L4w)] = cb[N + i];
            sV[wpos(i, L4w)] = cb[2 * N + T - 1 + i];
            if constexpr (MODE != MODE_GRID64) {
                sAm[wpos(i, L4w)] = ce[ubase + i];
                sBm[wpos(i, L4w)] = ce[vbase + i];
            }
        }
        Ctot = ce[N - 1];
        CVbN = cb[N - 1];
        if constexpr (MODE == MODE_FLOAT) {
            const float NN = (float)N * (float)N;
            kappa = Ctot / NN;  // as in band_body
            const float Sg = a.pixel_center ? 2.0f * N : (float)N;
            const float Call = Ctot + a.mu * NN + a.d0 * NN;
            scale = Call > 0.0f ? 1.0f / (2.0f * Sg * Call) : 0.0f;
            if (a.lens && !(Call > 0.0f) && t == 0 && a.status) atomicOr(a.status, (unsigned)DC_ERR_INVALID_ARG);
        }
        // the first row's barrier orders these writes before any read
    }

    S arun[G][4], Uo[G][4], Vo[G][4];
#pragma unroll
    for (int q = 0; q < G; ++q)
#pragma unroll
        for (int e = 0; e < 4; ++e) { arun[q][e] = S(0); Uo[q][e] = S(0); Vo[q][e] = S(0); }
    S RTcum = S(0);
    uint32_t vmax = 0u;

    auto load = [&](int j, uint4 (&dst)[G]) {
#pragma unroll
        for (int q = 0; q < G; ++q)
            dst[q] = ld_stream_v4(src + 4 * (((size_t)j << log2N) + 4 * (q * NT + t)));
    };
    uint4 buf[G];
    if constexpr (!RING) load(j0, buf);
    int rslot = 0;
    unsigned rpar = 0;
    bool dead = false;  // a ring wait expired: stop waiting, report DC_ERR_TIMEOUT

    const bool out32 = ((reinterpret_cast<uintptr_t>(a.alpha_out) | reinterpret_cast<uintptr_t>(a.alpha_t_out)) & 31) == 0;

    for (int r = 0; r < Tb; ++r) {
        const int j = j0 + r;
        const int par = r & 1;
        uint4 cur[G];
        if constexpr (RING) {
            if (!dead && !mbar_wait(&s_mbar[rslot], rpar)) {
                dead = true;
                if (a.status) atomicOr(a.status, (unsigned)DC_ERR_TIMEOUT);
            }
            const unsigned char *rowp = ringp + (size_t)rslot * rowbytes;
#pragma unroll
            for (int q = 0; q < G; ++q) cur[q] = *reinterpret_cast<const uint4 *>(rowp + 16 * (q * NT + t));
        } else {
#pragma unroll
            for (int q = 0; q < G; ++q) cur[q] = buf[q];
            if (r + 1 < Tb) load(j + 1, buf);
        }

        if constexpr (!FINAL) {
            if (a.zero_out) {
#pragma unroll
                for (int q = 0; q < G; ++q)
                    *reinterpret_cast<uint4 *>(a.zero_out + ((size_t)j << log2N) + 4 * (q * NT + t)) =
                        make_uint4(0u, 0u, 0u, 0u);
            }
        }

        // row values and the in-chunk prefix
        S p[G][4];
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const uint32_t x[4] = {cur[q].x, cur[q].y, cur[q].z, cur[q].w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if constexpr (MODE == MODE_FLOAT) p[q][e] = __uint_as_float(x[e]) - a.mu;
                else p[q][e] = x[e];
                if constexpr (MODE == MODE_GRID64 && !FINAL) vmax = max(vmax, x[e]);
            }
#pragma unroll
            for (int e = 1; e < 4; ++e) p[q][e] = p[q][e] + p[q][e - 1];
        }

        // neighbour state of the previous row (before this row's barrier)
        S u_next[G], v_prev[G];
#pragma unroll
        for (int q = 0; q < G; ++q) {
            u_next[q] = __shfl_down_sync(kFull, Uo[q][0], 1);
            v_prev[q] = __shfl_up_sync(kFull, Vo[q][3], 1);
            if (lane == 0) s_uf[par][q][warp] = Uo[q][0];
            if (lane == 31) s_vl[par][q][warp] = Vo[q][3];
        }

        // warp scans of the chunk sums
        S incl[G];
#pragma unroll
        for (int q = 0; q < G; ++q) {
            S x = p[q][3];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const S y = __shfl_up_sync(kFull, x, o);
                if (lane >= o) x = x + y;
            }
            incl[q] = x;
            if (lane == 31) s_wt[par][q][warp] = x;
        }
        __syncthreads();
        if constexpr (RING) {
            // every thread has read this row's slot: refill it with row j + ring
            if (t == 0 && r + ring < Tb && !dead) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                tma_row(ringp + (size_t)rslot * rowbytes, src + (size_t)(j + ring) * rowbytes, rowbytes,
                        &s_mbar[rslot]);
            }
            if (++rslot == ring) {
                rslot = 0;
                rpar ^= 1u;
            }
        }

        // scan over warps, then over chunk groups
        S off[G];
        S gp = S(0);
#pragma unroll
        for (int q = 0; q < G; ++q) {
            S wv = lane < nw ? s_wt[par][q][lane] : S(0);
#pragma unroll
            for (int o = 1; o < 16; o <<= 1) {
                const S y = __shfl_up_sync(kFull, wv, o);
                if (lane >= o) wv = wv + y;
            }
            const S wex = __shfl_sync(kFull, wv, (warp + 31) & 31);
            const S tot = __shfl_sync(kFull, wv, nw - 1);
            off[q] = gp + (warp > 0 ? wex : S(0)) + (incl[q] - p[q][3]);
            gp = gp + tot;
        }
        const S total = gp;
#pragma unroll
        for (int q = 0; q < G; ++q) {
#pragma unroll
            for (int e = 0; e < 4; ++e) p[q][e] = p[q][e] + off[q];
        }
        // the grid's edges: U(N, j-1) is the row totals above (column N - 1
        // is element 3 of thread NT - 1's last chunk); V(-1, j-1) = 0
        // (column 0 is element 0 of thread 0's first chunk)
        const S RTprev = RTcum;
        RTcum = RTcum + total;
#pragma unroll
        for (int q = 0; q < G; ++q) {
            if (lane == 31)
                u_next[q] = warp + 1 < nw ? s_uf[par][q][warp + 1] : (q + 1 < G ? s_uf[par][q + 1][0] : RTprev);
            if (lane == 0) v_prev[q] = warp > 0 ? s_vl[par][q][warp - 1] : (q > 0 ? s_vl[par][q - 1][nw - 1] : S(0));
        }

        // the three recurrences, in place: U ascending, V descending
#pragma unroll
        for (int q = 0; q < G; ++q) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const S ur = e < 3 ? Uo[q][e + 1] : u_next[q];
                Uo[q][e] = ur + p[q][e];
                arun[q][e] = arun[q][e] + p[q][e];
            }
#pragma unroll
            for (int e = 3; e >= 0; --e) {
                const S vl = e > 0 ? Vo[q][e - 1] : v_prev[q];
                const S pm1 = e > 0 ? p[q][e - 1] : off[q];  // P(j, c-1)
                Vo[q][e] = vl + pm1;
            }
        }

        if constexpr (!FINAL) {
            if (t == 0) {
                s_U0[r] = Uo[0][0];
                s_RT[r] = total;
            }
            if (t == NT - 1) s_VN[r] = Vo[G - 1][3];
        } else {
            const size_t rowoff = (size_t)j << log2N;
            // window element of column 4 m + e at this row: wpos(4 m + e + r)
            // = offU[e] + m, wpos(4 m + e - r + T - 1) = offV[e] + m
            int offU[4], offV[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int iu = e + r, iv = e - r + Tb - 1;
                offU[e] = (iu & 3) * L4w + (iu >> 2) + t;
                offV[e] = (iv & 3) * L4w + (iv >> 2) + t;
            }
#pragma unroll
            for (int q = 0; q < G; ++q) {
                const int cq = 4 * (q * NT + t);
                if constexpr (MODE == MODE_GRID64) {
                    unsigned long long oal[4], oat[4];
#pragma unroll
                    // (window positions recomputed per column: fewer live
                    // registers than the per-row offsets, faster at G = 4)
                    for (int e = 0; e < 4; ++e) {
                        const int c = cq + e;
                        oal[e] = sA[wpos(c, L4a)] + (unsigned long long)arun[q][e];
                        oat[e] = (sU[wpos(c + r, L4w)] + (unsigned long long)Uo[q][e]) -
                                 (sV[wpos(c - r + Tb - 1, L4w)] + (unsigned long long)Vo[q][e]);
                    }
                    if (a.alpha_out)
                        store4_u64(static_cast<unsigned long long *>(a.alpha_out) + rowoff + cq, oal[0], oal[1],
                                   oal[2], oal[3], out32);
                    if (a.alpha_t_out)
                        store4_u64(static_cast<unsigned long long *>(a.alpha_t_out) + rowoff + cq, oat[0], oat[1],
                                   oat[2], oat[3], out32);
                } else {
                    const C Ccj = CVbN + RTcum;
                    float dxy[8];
                    C oal[4], oat[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int c = cq + e;
                        const int iu = offU[e] + q * NT, iv = offV[e] + q * NT, ia = e * L4a + q * NT + t;
                        const C al = sA[ia] + arun[q][e];
                        const C at = (sU[iu] + Uo[q][e]) - (sV[iv] + Vo[q][e]);
                        const C A = sAm[iu];
                        const C Bv = Ctot - sBm[iv];
                        const C R = sR[ia];
                        C w[8];
                        w[0] = al;
                        w[1] = R - al;
                        w[2] = Ctot - R - Ccj + al;
                        w[3] = Ccj - al;
                        w[4] = at;
                        w[5] = A - at;
                        w[6] = Ctot - A - Bv + at;
                        w[7] = Bv - at;
                        oal[e] = al;
                        oat[e] = at;
                        const int Sg = a.pixel_center ? 2 * N : N;
                        const int ai = a.pixel_center ? 2 * c + 1 : c;
                        const int bj = a.pixel_center ? 2 * j + 1 : j;
                        int qx[8], qy[8], w0[8];
                        anchors(ai, bj, Sg, qx, qy);
                        lattice_counts(c, j, N, w0);
                        if constexpr (MODE == MODE_FLOAT) {
                            float nx = 0.f, ny = 0.f, nx0 = 0.f, ny0 = 0.f;
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                nx = fmaf(w[k], (float)qx[k], nx);
                                ny = fmaf(w[k], (float)qy[k], ny);
                                nx0 = fmaf((float)w0[k], (float)qx[k], nx0);
                                ny0 = fmaf((float)w0[k], (float)qy[k], ny0);
                            }
                            if (a.lens) {  // uniform: a launch parameter
                                dxy[2 * e] = lens_component(nx, w0, qx, ai, 2 * log2N, a.mu, Ctot, scale);
                                dxy[2 * e + 1] = lens_component(ny, w0, qy, bj, 2 * log2N, a.mu, Ctot, scale);
                            } else {
                                dxy[2 * e] = fmaf(-kappa, nx0, nx) * scale;
                                dxy[2 * e + 1] = fmaf(-kappa, ny0, ny) * scale;
                            }
                            oal[e] = al + a.mu * (float)w0[0];
                            oat[e] = at + a.mu * (float)w0[4];
                        } else {
                            long long A1x = 0, A1y = 0, A0x = 0, A0y = 0;
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                const long long wq = (long long)(uint32_t)w[k];
                                A1x += wq * qx[k];
                                A1y += wq * qy[k];
                                A0x += (long long)w0[k] * qx[k];
                                A0y += (long long)w0[k] * qy[k];
                            }
                            const long long Cn = (long long)(uint32_t)Ctot;
                            dxy[2 * e] = exact_component(A1x, A0x, 2 * log2N, Cn, a.inv_den_exact);
                            dxy[2 * e + 1] = exact_component(A1y, A0y, 2 * log2N, Cn, a.inv_den_exact);
                        }
                    }
                    if (a.disp) st_v8_f32(reinterpret_cast<float *>(a.disp) + 2 * (rowoff + cq), dxy);
                    if constexpr (MODE == MODE_FLOAT) {
                        if (a.alpha_out)
                            *reinterpret_cast<float4 *>(static_cast<float *>(a.alpha_out) + rowoff + cq) =
                                make_float4(oal[0], oal[1], oal[2], oal[3]);
                        if (a.alpha_t_out)
                            *reinterpret_cast<float4 *>(static_cast<float *>(a.alpha_t_out) + rowoff + cq) =
                                make_float4(oat[0], oat[1], oat[2], oat[3]);
                    } else {
                        if (a.alpha_out)
                            store4_u64(static_cast<unsigned long long *>(a.alpha_out) + rowoff + cq, oal[0], oal[1],
                                       oal[2], oal[3], out32);
                        if (a.alpha_t_out)
                            store4_u64(static_cast<unsigned long long *>(a.alpha_t_out) + rowoff + cq, oat[0], oat[1],
                                       oat[2], oat[3], out32);
                    }
                }
            }
        }
    }

    if constexpr (!FINAL) {
        // compact aggregate [alpha N][U N][V N][U0 T][E T][S][flag], as in band_body
        __syncthreads();
        C *ag = static_cast<C *>(a.agg) + (size_t)b * a.agg_stride;
        if constexpr (MODE == MODE_GRID64) {
            const uint32_t lim = 0xffffffffu / (uint32_t)(T << log2N);
            if (__syncthreads_or(vmax > lim)) {
                band_body_wide<MODE_GRID64, 4 * G, false>(a, log2N, T);
                if (t == 0) ag[3 * N + 2 * T + 1] = 1ull;
                return;
            }
            if (t == 0) ag[3 * N + 2 * T + 1] = 0ull;
        }
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int cq = 4 * (q * NT + t);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                ag[cq + e] = C(arun[q][e]);
                ag[N + cq + e] = C(Uo[q][e]);
                ag[2 * N + cq + e] = C(Vo[q][e]);
            }
        }
        for (int rr = t; rr < Tb; rr += NT) {
            S below = S(0);
            for (int q = rr + 1; q < Tb; ++q) below = below + s_RT[q];
            ag[3 * N + rr] = C(s_U0[rr]);
            ag[3 * N + T + rr] = C(s_VN[rr] + below);
        }
        if (t == 0) ag[3 * N + 2 * T] = C(RTcum);
    }
}

// ------------------------------------------------------------------------
// Aggregate pass by projections (N >= 128).
//
// Every value of a band's compact aggregate is a prefix sum of one of three
// one-dimensional projections of the band (rows r' = 0 .. T-1 of the band,
// x its values, minus mu in MODE_FLOAT):
//   column sums        K_c  = sum_r' x(r', c)                c in [0, N)
//   anti-diagonal sums A_d  = sum_r' x(r', d - r')           d in [0, N + T - 1)
//   diagonal sums      D_e  = sum_r' x(r', e + r' - T + 1)   e in [0, N + T - 1)
// Unrolling the band-local recurrences of band_body gives, with inclusive
// prefixes PK, PA, PD:
//   alpha(i) = PK(i), U(i) = PA(i + T - 1), V(i) = PD(i - 1) (0 for i = 0),
//   U0[r] = PA(r), E[r] = PD(N + T - 3 - r), S = PK(N - 1).
// So the pass needs no per-row scan: rows arrive by bulk copy into a ring of
// shared-memory slots padded by T - 1 columns on both sides (zeros, or mu in
// MODE_FLOAT, so that the padding contributes nothing), each thread adds the
// shifted row values of the lines it owns, and three block scans at the end
// produce the record.  Thread t owns columns 4 (t + NT k) .. + 3 of the
// column sums and lines t + NT k (k < CPT) plus N + t and N + NT + t (below
// N + T - 1) of the diagonal projections, so that every shared-memory read
// of a warp is conflict-free.
// ------------------------------------------------------------------------
__device__ __forceinline__ int ring_pad(int T) { return ((T - 1) + 3) & ~3; }

// inclusive block scan, in place, of smem array v[0, L); NT threads
template <typename S>
__device__ void block_scan_inplace(S *v, int L, S *s_part)
{
    const int NT = blockDim.x, t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = NT >> 5;
    const int per = ((L + NT - 1) / NT) | 1;  // odd stride: conflict-free segments
    const int b0 = t * per, b1 = min(L, b0 + per);
    S acc = S(0);
    for (int i = b0; i < b1; ++i) acc = acc + v[i];
    S x = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const S y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x = x + y;
    }
    if (lane == 31) s_part[warp] = x;
    __syncthreads();
    S wv = lane < nw ? s_part[lane] : S(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const S y = __shfl_up_sync(kFull, wv, o);
        if (lane >= o) wv = wv + y;
    }
    const S wex = __shfl_sync(kFull, wv, (warp + 31) & 31);
    S run = (warp > 0 ? wex : S(0)) + (x - acc);
    for (int i = b0; i < b1; ++i) {
        run = run + v[i];
        v[i] = run;
    }
    __syncthreads();
}

template <int MODE, int NT, int CPT>
__global__ void __launch_bounds__(NT) agg_proj_kernel(BandArgs a, int log2N, int T, int ring)
{
    using S = typename Band2T<MODE>::S;
    using C = typename Band2T<MODE>::C;
    constexpr int G = CPT / 4;
    const int N = NT * CPT;
    const int t = threadIdx.x;
    const int b = blockIdx.x;
    const int j0 = b * T;
    const int Tb = min(T, N - j0);  // rows of this band (the last one may be shorter)
    const int P0 = ring_pad(T);
    const int slotw = N + 2 * P0;  // words per ring slot
    const unsigned rowbytes = 4u << log2N;

    __shared__ unsigned long long s_mbar[8];
    __shared__ S s_part[32];
    extern __shared__ __align__(128) unsigned char s_dyn[];
    S *ringw = reinterpret_cast<S *>(s_dyn);
    const unsigned char *src = static_cast<const unsigned char *>(a.src);

    pdl_wait();
    // padding columns of every slot (the bulk copies fill only the middle)
    const S padv = MODE == MODE_FLOAT ? S(a.mu) : S(0);
    for (int k = 0; k < ring; ++k)
        for (int i = t; i < 2 * P0; i += NT) ringw[k * slotw + (i < P0 ? i : N + i)] = padv;
    if (t == 0) {
        for (int k = 0; k < ring; ++k) mbar_init(&s_mbar[k]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (t == 0)
        for (int k = 0; k < ring && k < Tb; ++k)
            tma_row(ringw + k * slotw + P0, src + (size_t)(j0 + k) * rowbytes, rowbytes, &s_mbar[k]);

    S K[G][4], A[CPT + 2], D[CPT + 2];
#pragma unroll
    for (int q = 0; q < G; ++q)
#pragma unroll
        for (int e = 0; e < 4; ++e) K[q][e] = S(0);
#pragma unroll
    for (int k = 0; k < CPT + 2; ++k) { A[k] = S(0); D[k] = S(0); }
    // lines N + t and N + NT + t of the diagonal projections (T - 1 <= 63, NT >= 32)
    const bool extra = t < Tb - 1, extra2 = NT + t < Tb - 1;
    uint32_t vor = 0u;
    int rslot = 0;
    unsigned rpar = 0;
    bool dead = false;

    for (int r = 0; r < Tb; ++r) {
        const int j = j0 + r;
        if (!dead && !mbar_wait(&s_mbar[rslot], rpar)) {
            dead = true;
            if (a.status) atomicOr(a.status, (unsigned)DC_ERR_TIMEOUT);
        }
        const S *row = ringw + rslot * slotw + P0;  // row[c], c in [-P0, N + P0)
        if constexpr (MODE == MODE_COUNT) {
            if (a.zero_out) {
#pragma unroll
                for (int q = 0; q < G; ++q)
                    *reinterpret_cast<uint4 *>(a.zero_out + ((size_t)j << log2N) + 4 * (t + NT * q)) =
                        make_uint4(0u, 0u, 0u, 0u);
            }
        }
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const uint4 v = *reinterpret_cast<const uint4 *>(row + 4 * (t + NT * q));
            if constexpr (MODE == MODE_FLOAT) {
                K[q][0] = K[q][0] + (__uint_as_float(v.x) - a.mu);
                K[q][1] = K[q][1] + (__uint_as_float(v.y) - a.mu);
                K[q][2] = K[q][2] + (__uint_as_float(v.z) - a.mu);
                K[q][3] = K[q][3] + (__uint_as_float(v.w) - a.mu);
            } else {
                K[q][0] = K[q][0] + v.x;
                K[q][1] = K[q][1] + v.y;
                K[q][2] = K[q][2] + v.z;
                K[q][3] = K[q][3] + v.w;
                if constexpr (MODE == MODE_GRID64) vor |= v.x | v.y | v.z | v.w;
            }
        }
        const S *ra = row + t - r;            // A: column (t + NT k) - r
        const S *rd = row + t + r - (Tb - 1);  // D: column (t + NT k) + r - (Tb - 1)
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            if constexpr (MODE == MODE_FLOAT) {
                A[k] = A[k] + (ra[NT * k] - a.mu);
                D[k] = D[k] + (rd[NT * k] - a.mu);
            } else {
                A[k] = A[k] + ra[NT * k];
                D[k] = D[k] + rd[NT * k];
            }
        }
        if (extra) {
            if constexpr (MODE == MODE_FLOAT) {
                A[CPT] = A[CPT] + (ra[N] - a.mu);
                D[CPT] = D[CPT] + (rd[N] - a.mu);
            } else {
                A[CPT] = A[CPT] + ra[N];
                D[CPT] = D[CPT] + rd[N];
            }
        }
        if (extra2) {
            if constexpr (MODE == MODE_FLOAT) {
                A[CPT + 1] = A[CPT + 1] + (ra[N + NT] - a.mu);
                D[CPT + 1] = D[CPT + 1] + (rd[N + NT] - a.mu);
            } else {
                A[CPT + 1] = A[CPT + 1] + ra[N + NT];
                D[CPT + 1] = D[CPT + 1] + rd[N + NT];
            }
        }
        __syncthreads();
        if (t == 0 && r + ring < Tb && !dead) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tma_row(ringw + rslot * slotw + P0, src + (size_t)(j + ring) * rowbytes, rowbytes, &s_mbar[rslot]);
        }
        if (++rslot == ring) {
            rslot = 0;
            rpar ^= 1u;
        }
    }

    C *ag = static_cast<C *>(a.agg) + (size_t)b * a.agg_stride;
    if constexpr (MODE == MODE_GRID64) {
        // every band-local sum is at most the band total <= max(x) T N
        const uint32_t lim = 0xffffffffu / (uint32_t)(T << log2N);
        if (__syncthreads_or(vor > lim)) {
            band_body_wide<MODE_GRID64, CPT, false>(a, log2N, T);
            if (t == 0) ag[3 * N + 2 * T + 1] = 1ull;
            return;
        }
    }

    // projections into shared memory (the ring is no longer read), then scans
    const int L = N + Tb - 1;
    S *pk = ringw, *pa = ringw + N, *pd = ringw + N + L;
#pragma unroll
    for (int q = 0; q < G; ++q)
#pragma unroll
        for (int e = 0; e < 4; ++e) pk[4 * (t + NT * q) + e] = K[q][e];
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        pa[t + NT * k] = A[k];
        pd[t + NT * k] = D[k];
    }
    if (extra) {
        pa[N + t] = A[CPT];
        pd[N + t] = D[CPT];
    }
    if (extra2) {
        pa[N + NT + t] = A[CPT + 1];
        pd[N + NT + t] = D[CPT + 1];
    }
    __syncthreads();
    block_scan_inplace(pk, N, s_part);
    block_scan_inplace(pa, L, s_part);
    block_scan_inplace(pd, L, s_part);

    // compact aggregate [alpha N][U N][V N][U0 T][E T][S][flag]
    for (int i = t; i < N; i += NT) {
        ag[i] = C(pk[i]);
        ag[N + i] = C(pa[i + Tb - 1]);
        ag[2 * N + i] = i > 0 ? C(pd[i - 1]) : C(0);
    }
    for (int r = t; r < Tb; r += NT) {
        ag[3 * N + r] = C(pa[r]);
        ag[3 * N + T + r] = C(pd[N + Tb - 3 - r]);
    }
    if (t == 0) {
        ag[3 * N + 2 * T] = C(pk[N - 1]);
        if constexpr (MODE == MODE_GRID64) ag[3 * N + 2 * T + 1] = 0ull;
    }
}

// ------------------------------------------------------------------------
// Carries: exclusive scan over bands of every absolute line.
// Lanes [0, N): vertical line i.  [N, 3N): anti-diagonal u = lane - N.
// [3N, 5N): diagonal v = lane - 3N - (N - 1).  Row b of the output holds
// the sum over bands < b; row nb the total (the marginals).
// ------------------------------------------------------------------------
// Index in band b's compact aggregate of its contribution to line `lane`
// (-1: none).  Selects rather than branches; the lane family (vertical,
// anti-diagonal, diagonal) is uniform across a warp since N % 32 == 0.
__device__ __forceinline__ int contrib_index(int b, int lane, int N, int T)
{
    const int j0 = b * T, Tb = min(T, N - j0), jl = j0 + Tb - 1;
    const int S = 3 * N + 2 * T;  // band total
    if (lane < N) return lane;
    if (lane < 3 * N) {
        const int u = lane - N;
        return u < j0 ? -1 : (u < jl ? 3 * N + (u - j0) : (u <= jl + N - 1 ? N + (u - jl) : S));
    }
    const int v = lane - 3 * N - (N - 1);
    const int m = v - (N - 1 - jl);
    return v < -jl ? -1 : (m <= 0 ? 2 * N + (v + jl) : (m <= Tb - 1 ? 3 * N + T + (Tb - 1 - m) : S));
}

// Where band b's carry row keeps line `lane` (-1: outside its windows).
__device__ __forceinline__ int carry_slot(int b, int lane, int N, int T)
{
    if (lane < N) return lane;
    const int j0 = b * T, Tb = min(T, N - j0);
    const int o = lane < 3 * N ? lane - N - j0 : lane - 3 * N - (N - j0 - Tb);
    const int base = lane < 3 * N ? N : 2 * N + T - 1;
    return (o >= 0 && o < N + Tb - 1) ? base + o : -1;
}

template <typename Acc, bool COH = false>
__device__ __forceinline__ Acc band_contrib(const Acc *ab, int b, int lane, int N, int T)
{
    // COH: L2 loads, for the fused kernel (records written by other CTAs of
    // the same launch)
    const int i = contrib_index(b, lane, N, T);
    return i >= 0 ? ld_carry<COH>(ab + i) : Acc(0);
}

template <typename Acc> struct ScanSum {
    Acc s;
    __device__ void zero() { s = Acc(0); }
    __device__ void add(Acc x) { s = s + x; }
    __device__ void add(const ScanSum &o) { s = s + o.s; }
    __device__ Acc value() const { return s; }
    __device__ ScanSum shfl_up(int o) const { ScanSum r; r.s = __shfl_up_sync(kFull, s, o); return r; }
};
struct ScanF2 {
    F2 s;
    __device__ void zero() { s = {0.f, 0.f}; }
    __device__ void add(float x) { s = f2_add(s, x); }
    __device__ void add(const ScanF2 &o) { s = f2_add(s, o.s); }
    __device__ float value() const { return s.hi + s.lo; }
    __device__ ScanF2 shfl_up(int o) const
    {
        ScanF2 r;
        r.s.hi = __shfl_up_sync(kFull, s.hi, o);
        r.s.lo = __shfl_up_sync(kFull, s.lo, o);
        return r;
    }
};
struct ScanF64 {
    double s;
    __device__ void zero() { s = 0.0; }
    __device__ void add(float x) { s += (double)x; }
    __device__ void add(const ScanF64 &o) { s += o.s; }
    __device__ float value() const { return (float)s; }
    __device__ ScanF64 shfl_up(int o) const { ScanF64 r; r.s = __shfl_up_sync(kFull, s, o); return r; }
};

// One block: 32 lanes x ng groups of bands (ng warps); each thread sums its
// group's contributions (kept in registers when the group has at most
// kCarryCache bands), the groups' totals are scanned in shared memory, and
// each thread writes its group's exclusive prefixes into the bands whose
// windows hold the lane.
constexpr int kCarryCache = 16;

template <typename Acc, typename Sum>
__device__ __forceinline__ void carry_body(const Acc *__restrict__ agg, Acc *__restrict__ carry, int log2N, int T,
                                           int nb, int agg_stride)
{
    const int N = 1 << log2N;
    const int lanes = 5 * N;
    const int cs = carry_stride(N, T);
    const int lx = threadIdx.x & 31, g = threadIdx.x >> 5, ng = blockDim.x >> 5;
    const int lane = blockIdx.x * 32 + lx;
    const bool active = lane < lanes;
    const int bpg = (nb + ng - 1) / ng;
    const int b_beg = g * bpg;
    const int b_end = min(nb, b_beg + bpg);
    __shared__ Sum s_sum[32][33];
    pdl_wait();

    // 32-bit element offsets (records and carries stay below 2^31 elements)
    Acc cache[kCarryCache];
    Sum s;
    s.zero();
    if (active) {
        if (bpg <= kCarryCache) {
#pragma unroll
            for (int k = 0; k < kCarryCache; ++k) {
                const int b = b_beg + k;
                const int i = b < b_end ? contrib_index(b, lane, N, T) : -1;
                cache[k] = i >= 0 ? agg[b * agg_stride + i] : Acc(0);
            }
#pragma unroll
            for (int k = 0; k < kCarryCache; ++k)
                if (b_beg + k < b_end) s.add(cache[k]);
        } else {
            for (int b = b_beg; b < b_end; ++b) {
                const int i = contrib_index(b, lane, N, T);
                s.add(i >= 0 ? agg[b * agg_stride + i] : Acc(0));
            }
        }
    }
    s_sum[g][lx] = s;
    __syncthreads();
    // exclusive scan over the ng groups of each of the 32 lanes: warp w
    // scans lanes w, w + ng, ... (one group per warp lane)
    for (int col = g; col < 32; col += ng) {
        Sum x;
        if (lx < ng) x = s_sum[lx][col];
        else x.zero();
        Sum inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            Sum y = inc.shfl_up(o);
            if (lx >= o) inc.add(y);
        }
        Sum ex = inc.shfl_up(1);
        if (lx == 0) ex.zero();
        if (lx < ng) s_sum[lx][col] = ex;
    }
    __syncthreads();
    if (!active) return;
    Sum pre = s_sum[g][lx];

    if (bpg <= kCarryCache) {
#pragma unroll
        for (int k = 0; k < kCarryCache; ++k) {
            const int b = b_beg + k;
            if (b < b_end) {
                const int o = carry_slot(b, lane, N, T);
                if (o >= 0) carry[b * cs + o] = pre.value();
                pre.add(cache[k]);
            }
        }
    } else {
        for (int b = b_beg; b < b_end; ++b) {
            const int o = carry_slot(b, lane, N, T);
            if (o >= 0) carry[b * cs + o] = pre.value();
            const int i = contrib_index(b, lane, N, T);
            pre.add(i >= 0 ? agg[b * agg_stride + i] : Acc(0));
        }
    }
    if (b_beg < nb && b_end == nb) carry[nb * cs + lane] = pre.value();
}
template <typename Acc, typename Sum>
__global__ void __launch_bounds__(1024, 1) carry_kernel(const Acc *__restrict__ agg, Acc *__restrict__ carry,
                                                     int log2N, int T, int nb, int agg_stride)
{
    carry_body<Acc, Sum>(agg, carry, log2N, T, nb, agg_stride);
}

// ------------------------------------------------------------------------
// Aggregate, carries and final pass in one cooperative launch (grids below
// 2048^2, where the three launches are latency-bound).  One CTA per band as
// in band_kernel; between the phases a grid barrier (all CTAs are resident:
// cooperative launch); the carries are computed by the CTAs together, CTA c
// taking lanes [c LPC, c LPC + LPC) split into G = NT / LPC groups of bands.
// ------------------------------------------------------------------------

// Sense-reversing grid barrier on bar[0] (arrivals) and bar[1] (generation);
// reusable across barriers and launches without a reset.  Waits at most
// limit_ns (then DC_ERR_TIMEOUT in status, and the CTA goes on; the status
// reset of declutter_sync also clears both words).  nblocks is the number of
// arrivals that completes the barrier: the grid size, or more when a test
// makes every wait run to its limit.
__device__ __noinline__ void grid_barrier(unsigned *bar, unsigned nblocks, unsigned *status,
                                          unsigned long long limit_ns)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*gen == g0) {
                if (global_ns() - t0 > limit_ns) {
                    if (status) atomicOr(status, (unsigned)DC_ERR_TIMEOUT);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
}

template <typename Acc, typename Sum>
__device__ void carry_phase(const Acc *agg, Acc *carry, int N, int T, int nb, int agg_stride, Sum *s_part)
{
    const int NT = blockDim.x, t = threadIdx.x;
    const int lanes = 5 * N;
    const int cs = carry_stride(N, T);
    const int LPC = (lanes + gridDim.x - 1) / gridDim.x;  // <= NT (checked by the launcher)
    const int G = NT / LPC;
    const int li = t % LPC, g = t / LPC;
    const int lane = blockIdx.x * LPC + li;
    const bool active = g < G && lane < lanes;
    const int bpg = (nb + G - 1) / G;
    const int b_beg = g * bpg, b_end = min(nb, b_beg + bpg);
    // a group's contributions in registers (all loads in flight at once)
    constexpr int kCache = 32;
    Acc cache[kCache];
    const bool cached = b_end - b_beg <= kCache;
    Sum sm;
    sm.zero();
    if (active) {
        if (cached) {
#pragma unroll
            for (int k = 0; k < kCache; ++k)
                if (b_beg + k < b_end) cache[k] = band_contrib<Acc, true>(agg + (size_t)(b_beg + k) * agg_stride, b_beg + k, lane, N, T);
#pragma unroll
            for (int k = 0; k < kCache; ++k)
                if (b_beg + k < b_end) sm.add(cache[k]);
        } else {
            for (int b = b_beg; b < b_end; ++b) sm.add(band_contrib<Acc, true>(agg + (size_t)b * agg_stride, b, lane, N, T));
        }
    }
    if (g < G) s_part[t] = sm;
    __syncthreads();
    if (!active) return;
    Sum pre;
    pre.zero();
    for (int q = 0; q < g; ++q) pre.add(s_part[q * LPC + li]);
#pragma unroll
    for (int k = 0; k < kCache; ++k) {
        const int b = b_beg + k;
        if (!cached || b >= b_end) break;
        int o = -1;
        const int j0 = b * T, Tb = min(T, N - j0);
        if (lane < N) {
            o = lane;
        } else if (lane < 3 * N) {
            const int w = lane - N - j0;
            if (w >= 0 && w < N + Tb - 1) o = N + w;
        } else {
            const int w = lane - 3 * N - (N - j0 - Tb);
            if (w >= 0 && w < N + Tb - 1) o = 2 * N + T - 1 + w;
        }
        if (o >= 0) carry[(size_t)b * cs + o] = pre.value();
        pre.add(cache[k]);
    }
    for (int b = cached ? b_end : b_beg; b < b_end; ++b) {
        int o = -1;
        const int j0 = b * T, Tb = min(T, N - j0);
        if (lane < N) {
            o = lane;
        } else if (lane < 3 * N) {
            const int w = lane - N - j0;
            if (w >= 0 && w < N + Tb - 1) o = N + w;
        } else {
            const int w = lane - 3 * N - (N - j0 - Tb);
            if (w >= 0 && w < N + Tb - 1) o = 2 * N + T - 1 + w;
        }
        if (o >= 0) carry[(size_t)b * cs + o] = pre.value();
        pre.add(band_contrib<Acc, true>(agg + (size_t)b * agg_stride, b, lane, N, T));
    }
    if (b_beg < nb && b_end == nb) carry[(size_t)nb * cs + lane] = pre.value();
}

template <int MODE, int CPT, typename Sum>
__global__ void __launch_bounds__(CPT == 1 ? 64 : 512) band_fused_kernel(BandArgs aagg, BandArgs afin, int log2N, int T,
                                                                        unsigned *bar, unsigned long long limit_ns,
                                                                        unsigned extra_arrivals)
{
    using Acc = typename ModeT<MODE>::Acc;
    __shared__ Sum s_part[CPT == 1 ? 64 : 512];
    band_body<MODE, CPT, false>(aagg, log2N, T);
    grid_barrier(bar, gridDim.x + extra_arrivals, afin.status, limit_ns);
    const int N = 1 << log2N;
    carry_phase<Acc, Sum>(static_cast<const Acc *>(aagg.agg), static_cast<Acc *>(const_cast<void *>(afin.carry)), N,
                          T, (N + T - 1) / T, aagg.agg_stride, s_part);
    grid_barrier(bar, gridDim.x + extra_arrivals, afin.status, limit_ns);
    band_body<MODE, CPT, true, true>(afin, log2N, T);
}

// ------------------------------------------------------------------------
// Batched wrappers: panel blockIdx.y (blockIdx.z for the smoothing tiles) of
// a PanelDesc table
// ------------------------------------------------------------------------
template <int TS, int R, int RAD>
__global__ void __launch_bounds__(256) smooth_batched_kernel(const PanelDesc *__restrict__ tab, int log2N, GaussW w,
                                                             int cur, int zero_next)
{
    const PanelDesc &d = tab[blockIdx.z];
    smooth_win_body<TS, R, RAD>(d.counts[cur], d.dens, log2N, w, zero_next ? d.counts[cur ^ 1] : nullptr);
}

template <int MODE, int CPT, bool FINAL>
__global__ void __launch_bounds__(CPT == 1 ? 64 : 512) band_batched_kernel(const PanelDesc *__restrict__ tab,
                                                                          int log2N, int T, int cur, int zero_next)
{
    const PanelDesc &d = tab[blockIdx.y];
    BandArgs a = d.band;
    if constexpr (MODE == MODE_FLOAT) {
        a.src = d.dens;
        a.zero_out = nullptr;
    } else {
        a.src = d.counts[cur];
        a.zero_out = (!FINAL && zero_next) ? d.counts[cur ^ 1] : nullptr;
    }
    if constexpr (FINAL) a.zero_out = nullptr;
    band_body<MODE, CPT, FINAL>(a, log2N, T);
}

template <typename Acc, typename Sum>
__global__ void __launch_bounds__(1024, 1) carry_batched_kernel(const PanelDesc *__restrict__ tab, int log2N, int T,
                                                             int nb, int agg_stride)
{
    const PanelDesc &d = tab[blockIdx.y];
    carry_body<Acc, Sum>(static_cast<const Acc *>(d.band.agg), static_cast<Acc *>(const_cast<void *>(d.band.carry)),
                         log2N, T, nb, agg_stride);
}

}  // namespace

int smooth_smem_bytes(int r)
{
    const int TW = 32;
    const int W = TW + 2 * r;
    return (W * W + TW * W) * (int)sizeof(float);
}

// tile of the sliding-window smoothing: 64 x 64 outputs from 1024 x 1024
static int smooth_tile(int log2N) { return log2N >= 10 ? 64 : 32; }
static int smooth_win_smem_bytes(int TS, int r)
{
    const int W = TS + 2 * r;
    return (W * W + TS * (W | 1)) * (int)sizeof(float);
}

// Grids from 2048 x 2048 (1024 x 1024 for the exact 64-bit images) use the
// interleaved kernels; smaller ones (few rows per band, latency-bound) the
// per-thread-contiguous band_kernel, which measured faster there (512^2
// float mode: 3.5 vs 4.9 us aggregate, 5.3 vs 5.9 us final pass).
constexpr int interleaved_min_log2(int mode) { return mode == MODE_GRID64 ? 10 : 11; }

// dynamic shared memory of the interleaved final kernel: the carry windows
// (and, outside MODE_GRID64, the marginal windows)
static size_t band2_smem_bytes(int mode, int N, int T)
{
    auto l4 = [](int len) { return ((((len + 3) >> 2) + 23) >> 5 << 5) + 8; };
    const size_t per = 4 * (size_t)l4(N) + 8 * (size_t)l4(N + T - 1);
    return mode == MODE_GRID64 ? per * 8 : 2 * per * 4;
}

template <int MODE, int NT, int G>
static cudaError_t allow_band2_smem()
{
    // the most any launch asks for (carry windows plus ring, <= 200 KB)
    const int most = 204800;
    cudaError_t e = cudaFuncSetAttribute(agg_proj_kernel<MODE, NT, 4 * G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         most);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(band2_kernel<MODE, NT, G, true, (G < 4)>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 most);
    return e;
}
template <int MODE>
static cudaError_t allow_band2_smem_all()
{
    cudaError_t e = allow_band2_smem<MODE, 512, 1>();
    if constexpr (MODE == MODE_GRID64)
        if (e == cudaSuccess) e = allow_band2_smem<MODE, 256, 1>();
    if (e == cudaSuccess) e = allow_band2_smem<MODE, 512, 2>();
    if (e == cudaSuccess) e = allow_band2_smem<MODE, 512, 4>();
    return e;
}

// dynamic shared memory of the smoothing kernels of one radius instantiation
template <int RAD>
static cudaError_t allow_smooth_smem()
{
    const int rmax = RAD >= 0 ? RAD : 64;
    cudaError_t e = cudaFuncSetAttribute(smooth_win_kernel<64, 8, RAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smooth_win_smem_bytes(64, rmax));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(smooth_win_kernel<32, 8, RAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smooth_win_smem_bytes(32, rmax));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(smooth_batched_kernel<64, 8, RAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smooth_win_smem_bytes(64, rmax));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(smooth_batched_kernel<32, 8, RAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smooth_win_smem_bytes(32, rmax));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(smooth_agg_kernel<4, 4, RAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmoothAggSmemMax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(smooth_agg_kernel<4, 8, RAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmoothAggSmemMax);
    return e;
}

// F(RAD) for the smoothing instantiation of radius r
#define DC_RADIUS_DISPATCH(r, F)                                                                                      \
    switch (r) {                                                                                                     \
    case 2: F(2);                                                                                                    \
    case 4: F(4);                                                                                                    \
    case 8: F(8);                                                                                                    \
    case 16: F(16);                                                                                                  \
    case 32: F(32);                                                                                                  \
    default: F(-1);                                                                                                  \
    }

cudaError_t prepare_kernels()
{
    // dynamic shared memory of the smoothing tile for the largest radius
    cudaError_t e = cudaFuncSetAttribute(smooth_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smooth_smem_bytes(64));
    if (e == cudaSuccess) e = allow_smooth_smem<-1>();
    if (e == cudaSuccess) e = allow_smooth_smem<2>();
    if (e == cudaSuccess) e = allow_smooth_smem<4>();
    if (e == cudaSuccess) e = allow_smooth_smem<8>();
    if (e == cudaSuccess) e = allow_smooth_smem<16>();
    if (e == cudaSuccess) e = allow_smooth_smem<32>();
    if (e == cudaSuccess) e = allow_band2_smem_all<MODE_COUNT>();
    if (e == cudaSuccess) e = allow_band2_smem_all<MODE_FLOAT>();
    if (e == cudaSuccess) e = allow_band2_smem_all<MODE_GRID64>();
    if (e == cudaSuccess) e = prepare_point_kernels();
    return e;
}

cudaError_t launch_smooth(cudaStream_t s, const uint32_t *counts, float *dens, int log2N, const GaussW &w,
                          uint32_t *zero_out)
{
    const int N = 1 << log2N;
    if (N >= 32) {
        const int TS = smooth_tile(log2N);
        const size_t bytes = (size_t)smooth_win_smem_bytes(TS, w.r);
        const dim3 grid(N / TS, N / TS);
#define DC_LAUNCH_WIN(RAD)                                                                                            \
    return TS == 64 ? launch_kernel(smooth_win_kernel<64, 8, RAD>, grid, dim3(256), bytes, s, counts, dens, log2N, w,  \
                                    zero_out)                                                                         \
                    : launch_kernel(smooth_win_kernel<32, 8, RAD>, grid, dim3(256), bytes, s, counts, dens, log2N, w,  \
                                    zero_out)
        DC_RADIUS_DISPATCH(w.r, DC_LAUNCH_WIN)
#undef DC_LAUNCH_WIN
    }
    const int TW = N;
    const int bytes = smooth_smem_bytes(w.r);
    dim3 grid(N / TW, N / TW);
    return launch_kernel(smooth_kernel, grid, dim3(256), (size_t)bytes, s, counts, dens, log2N, w, zero_out);
}

// Smoothing fused into the aggregate pass: windows of 4 rows for bands of
// up to 4 rows, else 8; shared memory for the input rows (with halo and the
// windows' overrun) and the vertical pass's swizzled rows.
static int smooth_agg_R(int T) { return T <= 4 ? 4 : 8; }
static size_t smooth_agg_smem_bytes(const BandGeom &g, int r)
{
    const int R = smooth_agg_R(g.T);
    const int W = g.N + 2 * r;
    const int Ws = (W - 1) + ((W - 1) >> 5) + 1;
    return 4 * ((size_t)((g.T + R - 1) / R * R + 2 * r) * W + (size_t)g.T * Ws);
}
bool smooth_agg_available(const BandGeom &g, const GaussW &w)
{
    return g.N >= 128 && g.log2N < interleaved_min_log2(MODE_FLOAT) && g.CPT == 4 && w.r >= 1 &&
           smooth_agg_smem_bytes(g, w.r) <= kSmoothAggSmemMax;
}

cudaError_t launch_smooth_agg(cudaStream_t s, const BandGeom &g, const BandArgs &a, const GaussW &w,
                              const uint32_t *counts, float *dens, uint32_t *zero_out)
{
    if (!smooth_agg_available(g, w)) return cudaErrorInvalidValue;
    const size_t smem = smooth_agg_smem_bytes(g, w.r);
    const int nt = 4 * g.NT < 1024 ? 4 * g.NT : 1024;  // g.NT = N / 4 band threads
    const bool r4 = smooth_agg_R(g.T) == 4;
#define DC_LAUNCH_AGG(RAD)                                                                                            \
    return r4 ? launch_kernel(smooth_agg_kernel<4, 4, RAD>, dim3(g.nb), dim3(nt), smem, s, a, g.log2N, g.T, w, counts,  \
                              dens, zero_out)                                                                         \
              : launch_kernel(smooth_agg_kernel<4, 8, RAD>, dim3(g.nb), dim3(nt), smem, s, a, g.log2N, g.T, w, counts,  \
                              dens, zero_out)
    DC_RADIUS_DISPATCH(w.r, DC_LAUNCH_AGG)
#undef DC_LAUNCH_AGG
}

// Ring slots of the interleaved kernels: up to 128 KB of rows for the
// aggregate pass; for the final pass what is left of 200 KB after the carry
// windows (none at N = 8192, whose final pass prefetches into registers).
static int band2_ring(int mode, bool final_pass, int N, int T)
{
    const size_t row = 4 * (size_t)N;
    size_t room = 131072;
    if (final_pass) {
        const size_t win = band2_smem_bytes(mode, N, T);
        room = win < 204800 ? 204800 - win : 0;
    }
    int k = (int)(room / row);
    if (k > 8) k = 8;
    if (k > T) k = T < 2 ? 2 : T;
    return k >= 2 ? k : 0;
}

// Ring of the projection aggregate pass: up to 8 padded rows within 128 KB;
// the scans at the end reuse the same memory (3N + 2T words).
static int agg_ring(int N, int T)
{
    const int pad = ((T - 1) + 3) & ~3;
    const size_t slot = 4 * (size_t)(N + 2 * pad);
    int k = (int)(131072 / slot);
    if (k > 8) k = 8;
    if (k > T) k = T;
    return k < 2 ? 2 : k;
}
static size_t agg_smem_bytes(int N, int T, int ring)
{
    const int pad = ((T - 1) + 3) & ~3;
    const size_t ringb = 4 * (size_t)ring * (N + 2 * pad);
    const size_t scanb = 4 * (size_t)(3 * N + 2 * T);
    return ringb > scanb ? ringb : scanb;
}

template <int MODE, int NT, int G>
static cudaError_t launch_band2(cudaStream_t s, const BandGeom &g, const BandArgs &a, bool final_pass)
{
    if (!final_pass) {
        const int ring = agg_ring(g.N, g.T);
        return launch_kernel(agg_proj_kernel<MODE, NT, 4 * G>, dim3(g.nb), dim3(NT), agg_smem_bytes(g.N, g.T, ring),
                             s, a, g.log2N, g.T, ring);
    }
    const int ring = band2_ring(MODE, true, g.N, g.T);
    const size_t smem = band2_smem_bytes(MODE, g.N, g.T) + (size_t)ring * 4 * g.N;
    if constexpr (G < 4) {  // N <= 4096: rows through the bulk-copy ring
        if (ring)
            return launch_kernel(band2_kernel<MODE, NT, G, true, true>, dim3(g.nb), dim3(NT), smem, s, a, g.log2N,
                                 g.T, ring);
        return cudaErrorInvalidValue;
    } else {  // N = 8192: the carry windows fill shared memory
        return launch_kernel(band2_kernel<MODE, NT, G, true, false>, dim3(g.nb), dim3(NT), smem, s, a, g.log2N, g.T,
                             0);
    }
}

template <int MODE>
static cudaError_t launch_band2_n(cudaStream_t s, const BandGeom &g, const BandArgs &a, bool final_pass)
{
    switch (g.log2N) {  // NT = min(512, N / 4) threads, G = N / (4 NT) chunks a thread
    case 10:
        if constexpr (MODE == MODE_GRID64) return launch_band2<MODE, 256, 1>(s, g, a, final_pass);
        return cudaErrorInvalidValue;
    case 11: return launch_band2<MODE, 512, 1>(s, g, a, final_pass);
    case 12: return launch_band2<MODE, 512, 2>(s, g, a, final_pass);
    case 13: return launch_band2<MODE, 512, 4>(s, g, a, final_pass);
    default: return cudaErrorInvalidValue;
    }
}

template <int MODE, bool FINAL>
static cudaError_t launch_band_mode(cudaStream_t s, const BandGeom &g, const BandArgs &a)
{
    if (g.log2N >= interleaved_min_log2(MODE)) return launch_band2_n<MODE>(s, g, a, FINAL);
    switch (g.CPT) {
    case 1: return launch_kernel(band_kernel<MODE, 1, FINAL>, dim3(g.nb), dim3(g.NT), 0, s, a, g.log2N, g.T);
    case 4: return launch_kernel(band_kernel<MODE, 4, FINAL>, dim3(g.nb), dim3(g.NT), 0, s, a, g.log2N, g.T);
    case 8: return launch_kernel(band_kernel<MODE, 8, FINAL>, dim3(g.nb), dim3(g.NT), 0, s, a, g.log2N, g.T);
    case 16: return launch_kernel(band_kernel<MODE, 16, FINAL>, dim3(g.nb), dim3(g.NT), 0, s, a, g.log2N, g.T);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_band_agg(cudaStream_t s, const BandGeom &g, int mode, const BandArgs &a)
{
    switch (mode) {
    case MODE_COUNT: return launch_band_mode<MODE_COUNT, false>(s, g, a);
    case MODE_FLOAT: return launch_band_mode<MODE_FLOAT, false>(s, g, a);
    case MODE_GRID64: return launch_band_mode<MODE_GRID64, false>(s, g, a);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_band_final(cudaStream_t s, const BandGeom &g, int mode, const BandArgs &a)
{
    switch (mode) {
    case MODE_COUNT: return launch_band_mode<MODE_COUNT, true>(s, g, a);
    case MODE_FLOAT: return launch_band_mode<MODE_FLOAT, true>(s, g, a);
    case MODE_GRID64: return launch_band_mode<MODE_GRID64, true>(s, g, a);
    }
    return cudaErrorInvalidValue;
}

using FusedFn = void (*)(BandArgs, BandArgs, int, int, unsigned *, unsigned long long, unsigned);
template <int MODE, typename Sum>
static FusedFn fused_ptr(int CPT)
{
    if (CPT == 1) return band_fused_kernel<MODE, 1, Sum>;
    if (CPT == 4) return band_fused_kernel<MODE, 4, Sum>;
    return nullptr;
}
static FusedFn fused_kernel_for(const BandGeom &g, int mode, int carry_mode)
{
    if (g.log2N >= interleaved_min_log2(mode) || (mode != MODE_COUNT && mode != MODE_FLOAT)) return nullptr;
    if (5 * g.T > g.NT) return nullptr;  // carry lanes of a CTA: at most one per thread
    if (mode == MODE_COUNT) return fused_ptr<MODE_COUNT, ScanSum<uint32_t>>(g.CPT);
    if (carry_mode == DC_CARRY_F64) return fused_ptr<MODE_FLOAT, ScanF64>(g.CPT);
    return fused_ptr<MODE_FLOAT, ScanF2>(g.CPT);
}

bool band_fused_available(const BandGeom &g, int mode, int carry_mode, int device)
{
    auto k = fused_kernel_for(g, mode, carry_mode);
    if (!k) return false;
    int per_sm = 0, sms = 0, coop = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, g.NT, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return coop && per_sm * sms >= g.nb;
}

cudaError_t launch_band_fused(cudaStream_t s, const BandGeom &g, int mode, int carry_mode, const BandArgs &aagg,
                              const BandArgs &afin, unsigned *bar, unsigned long long limit_ns,
                              unsigned extra_arrivals)
{
    auto k = fused_kernel_for(g, mode, carry_mode);
    if (!k) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g.nb);
    cfg.blockDim = dim3(g.NT);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, aagg, afin, g.log2N, g.T, bar, limit_ns, extra_arrivals);
}

cudaError_t launch_carry(cudaStream_t s, const BandGeom &g, int mode, int carry_mode, const void *agg, void *carry)
{
    // groups of bands per block (one warp each): as many as keep all blocks
    // resident at once on the device's SMs of 2048 threads, at most 32 and nb
    const int nblk = (g.lanes + 31) / 32;
    int cap = g.sms * 64 / nblk;
    if (cap > 32) cap = 32;
    if (cap > g.nb) cap = g.nb;
    int ng = 1;
    while (2 * ng <= cap) ng *= 2;
    // but enough groups that each holds at most kCarryCache bands (registers)
    const int need = (g.nb + kCarryCache - 1) / kCarryCache;
    if (ng < need) ng = need > 32 ? 32 : need;
    const dim3 blocks((g.lanes + 31) / 32), threads(32 * ng);
    switch (mode) {
    case MODE_COUNT:
        return launch_kernel(carry_kernel<uint32_t, ScanSum<uint32_t>>, blocks, threads, 0, s,
                             static_cast<const uint32_t *>(agg), static_cast<uint32_t *>(carry), g.log2N, g.T, g.nb,
                             g.agg_stride);
    case MODE_GRID64:
        return launch_kernel(carry_kernel<unsigned long long, ScanSum<unsigned long long>>, blocks, threads, 0, s,
                             static_cast<const unsigned long long *>(agg), static_cast<unsigned long long *>(carry),
                             g.log2N, g.T, g.nb, g.agg_stride);
    case MODE_FLOAT:
        if (carry_mode == DC_CARRY_F64)
            return launch_kernel(carry_kernel<float, ScanF64>, blocks, threads, 0, s, static_cast<const float *>(agg),
                                 static_cast<float *>(carry), g.log2N, g.T, g.nb, g.agg_stride);
        return launch_kernel(carry_kernel<float, ScanF2>, blocks, threads, 0, s, static_cast<const float *>(agg),
                             static_cast<float *>(carry), g.log2N, g.T, g.nb, g.agg_stride);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_smooth_batched(cudaStream_t s, const PanelDesc *tab, int P, int log2N, const GaussW &w, int cur,
                                  bool zero_next)
{
    const int N = 1 << log2N;
    if (N < 32) return cudaErrorInvalidValue;
    const int TS = smooth_tile(log2N);
    const size_t bytes = (size_t)smooth_win_smem_bytes(TS, w.r);
    const dim3 grid(N / TS, N / TS, P);
    const int zn = zero_next ? 1 : 0;
#define DC_LAUNCH_BAT(RAD)                                                                                            \
    return TS == 64 ? launch_kernel(smooth_batched_kernel<64, 8, RAD>, grid, dim3(256), bytes, s, tab, log2N, w, cur, zn) \
                    : launch_kernel(smooth_batched_kernel<32, 8, RAD>, grid, dim3(256), bytes, s, tab, log2N, w, cur, zn)
    DC_RADIUS_DISPATCH(w.r, DC_LAUNCH_BAT)
#undef DC_LAUNCH_BAT
}

template <int MODE, int CPT>
static cudaError_t band_batched_mode(cudaStream_t s, const BandGeom &g, int carry_mode, const PanelDesc *tab, int P,
                                     int cur, bool zero_next)
{
    const dim3 grid(g.nb, P), block(g.NT);
    cudaError_t e =
        launch_kernel(band_batched_kernel<MODE, CPT, false>, grid, block, 0, s, tab, g.log2N, g.T, cur, zero_next ? 1 : 0);
    if (e != cudaSuccess) return e;
    int ng = 32;  // groups of bands per carry block: as launch_carry, so that
    {             // float carries are summed in the same order as for one panel
        const int nblk = (g.lanes + 31) / 32;
        int cap = g.sms * 64 / nblk;
        if (cap > 32) cap = 32;
        if (cap > g.nb) cap = g.nb;
        ng = 1;
        while (2 * ng <= cap) ng *= 2;
        const int need = (g.nb + kCarryCache - 1) / kCarryCache;
        if (ng < need) ng = need > 32 ? 32 : need;
    }
    const dim3 cgrid((g.lanes + 31) / 32, P), cblock(32 * ng);
    if constexpr (MODE == MODE_COUNT)
        e = launch_kernel(carry_batched_kernel<uint32_t, ScanSum<uint32_t>>, cgrid, cblock, 0, s, tab, g.log2N, g.T,
                          g.nb, g.agg_stride);
    else if (carry_mode == DC_CARRY_F64)
        e = launch_kernel(carry_batched_kernel<float, ScanF64>, cgrid, cblock, 0, s, tab, g.log2N, g.T, g.nb,
                          g.agg_stride);
    else
        e = launch_kernel(carry_batched_kernel<float, ScanF2>, cgrid, cblock, 0, s, tab, g.log2N, g.T, g.nb,
                          g.agg_stride);
    if (e != cudaSuccess) return e;
    return launch_kernel(band_batched_kernel<MODE, CPT, true>, grid, block, 0, s, tab, g.log2N, g.T, cur, 0);
}

cudaError_t launch_band_batched(cudaStream_t s, const BandGeom &g, int mode, int carry_mode, const PanelDesc *tab,
                                int P, int cur, bool zero_next)
{
    if (g.log2N >= interleaved_min_log2(mode)) return cudaErrorInvalidValue;  // per-thread-contiguous kernels only
    if (mode == MODE_COUNT) {
        if (g.CPT == 1) return band_batched_mode<MODE_COUNT, 1>(s, g, carry_mode, tab, P, cur, zero_next);
        if (g.CPT == 4) return band_batched_mode<MODE_COUNT, 4>(s, g, carry_mode, tab, P, cur, zero_next);
    } else if (mode == MODE_FLOAT) {
        if (g.CPT == 1) return band_batched_mode<MODE_FLOAT, 1>(s, g, carry_mode, tab, P, cur, zero_next);
        if (g.CPT == 4) return band_batched_mode<MODE_FLOAT, 4>(s, g, carry_mode, tab, P, cur, zero_next);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dc
