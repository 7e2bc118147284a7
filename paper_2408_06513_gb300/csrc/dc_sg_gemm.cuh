// BF16 tensor-core implicit GEMM for the 3x3 convolutions of the surrogate
// network (forward, backward-data, weight gradient).
//
// C[m][n] = sum_k A[m][k] B[k][n], FP32 accumulation, mma.sync m16n8k16 with
// bf16 operands.  CTA tile 64 x TN x 32, 4 warps: TN = 64 as 2 x 2 warps of
// 32 x 32, TN = 32 (narrow layers) as 4 x 1 warps of 16 x 32.
// Operands are staged into shared memory in 16-byte chunks of 8 bf16 by
// cp.async (zero-filled where the problem's loader returns null, e.g. the
// zero padding of the convolution), double-buffered along k.  Each operand is
// staged either with its k dimension contiguous ([rows][k]) or with its m / n
// dimension contiguous ([k][cols]); ldmatrix (.trans for the latter) turns
// either into mma fragments.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace dc {
namespace sg {

constexpr int BM = 64, BN = 64, BK = 32;
constexpr int GEMM_THREADS = 128;
constexpr int PAD = 8;  // bf16 elements of padding per smem row (bank spread)

enum Layout { K_CONTIG = 0, MN_CONTIG = 1 };

// gmem null: the 16 bytes are zero-filled (no byte is read from `valid`,
// which only has to be a mapped global address)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, const void *valid)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    const int bytes = gmem ? 16 : 0;
    const void *src = gmem ? gmem : valid;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(src), "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::); }

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void *p)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(p));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(s));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const void *p)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(p));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(s));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Problem P provides:
//   static constexpr int ALAYOUT, BLAYOUT;
//   int M, N, K;
//   const void *a_chunk(int m, int k) const;  // 8 bf16 along the contiguous dim
//   const void *b_chunk(int k, int n) const;
//   const void *base() const;   // any mapped global address (zero-fill source)
//   void epilogue(int m, int n, float v0, float v1) const;  // C[m][n], C[m][n+1]
//   k range of a CTA: [k_begin, k_end) from blockIdx.z (split-K)
template <class P, int TN = BN>
__global__ void __launch_bounds__(GEMM_THREADS) gemm_kernel(P p, int k_per_split)
{
    static_assert(TN == 64 || TN == 32, "tile width");
    constexpr int MI = TN == 64 ? 2 : 1;  // m16 blocks a warp
    // stage buffers: A and B, two stages each
    constexpr int A_ROWS = P::ALAYOUT == K_CONTIG ? BM : BK;
    constexpr int A_COLS = P::ALAYOUT == K_CONTIG ? BK : BM;
    constexpr int B_ROWS = P::BLAYOUT == K_CONTIG ? TN : BK;
    constexpr int B_COLS = P::BLAYOUT == K_CONTIG ? BK : TN;
    __shared__ __align__(16) __nv_bfloat16 sA[2][A_ROWS][A_COLS + PAD];
    __shared__ __align__(16) __nv_bfloat16 sB[2][B_ROWS][B_COLS + PAD];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = TN == 64 ? (warp >> 1) * 32 : warp * 16, wn = TN == 64 ? (warp & 1) * 32 : 0;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * TN;
    const int k_begin = blockIdx.z * k_per_split;
    const int k_end = min(p.K, k_begin + k_per_split);
    pdl_wait();
    if (k_begin >= k_end) return;

    auto stage = [&](int buf, int k0) {
        // A: BM * BK / 8 = 256 chunks, two per thread
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int c = tid + i * GEMM_THREADS;
            if constexpr (P::ALAYOUT == K_CONTIG) {
                const int r = c >> 2, kc = (c & 3) * 8;
                const int m = m0 + r, k = k0 + kc;
                cp_async16(&sA[buf][r][kc], (m < p.M && k < k_end) ? p.a_chunk(m, k) : nullptr, p.base());
            } else {
                const int r = c >> 3, mc = (c & 7) * 8;
                const int k = k0 + r, m = m0 + mc;
                cp_async16(&sA[buf][r][mc], (m < p.M && k < k_end) ? p.a_chunk(m, k) : nullptr, p.base());
            }
        }
#pragma unroll
        for (int i = 0; i < TN / 32; ++i) {
            const int c = tid + i * GEMM_THREADS;
            if constexpr (P::BLAYOUT == K_CONTIG) {
                const int r = c >> 2, kc = (c & 3) * 8;
                const int n = n0 + r, k = k0 + kc;
                cp_async16(&sB[buf][r][kc], (n < p.N && k < k_end) ? p.b_chunk(k, n) : nullptr, p.base());
            } else {
                constexpr int CPR = TN / 8;  // 16-byte chunks a row
                const int r = c / CPR, nc = (c % CPR) * 8;
                const int k = k0 + r, n = n0 + nc;
                cp_async16(&sB[buf][r][nc], (n < p.N && k < k_end) ? p.b_chunk(k, n) : nullptr, p.base());
            }
        }
        cp_async_commit();
    };

    float acc[MI][4][4];
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

    const int nk = (k_end - k_begin + BK - 1) / BK;
    stage(0, k_begin);
    for (int t = 0; t < nk; ++t) {
        const int buf = t & 1;
        if (t + 1 < nk) {
            stage(buf ^ 1, k_begin + (t + 1) * BK);
            cp_async_wait_one();
        } else {
            cp_async_wait_all();
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            unsigned af[MI][4];
#pragma unroll
            for (int i = 0; i < MI; ++i) {
                const int mb = wm + i * 16;
                const int mi = lane >> 3, rr = lane & 7;
                if constexpr (P::ALAYOUT == K_CONTIG) {
                    // matrices: (m 0-7, k 0-7), (m 8-15, k 0-7), (m 0-7, k 8-15), (m 8-15, k 8-15)
                    ldsm_x4(af[i], &sA[buf][mb + (mi & 1) * 8 + rr][ks + (mi >> 1) * 8]);
                } else {
                    ldsm_x4_t(af[i], &sA[buf][ks + (mi >> 1) * 8 + rr][mb + (mi & 1) * 8]);
                }
            }
            unsigned bf[4][2];
#pragma unroll
            for (int jj = 0; jj < 2; ++jj) {
                const int nb = wn + jj * 16;
                const int mi = lane >> 3, rr = lane & 7;
                unsigned r4[4];
                if constexpr (P::BLAYOUT == K_CONTIG) {
                    // matrices: (n 0-7, k 0-7), (n 0-7, k 8-15), (n 8-15, k 0-7), (n 8-15, k 8-15)
                    ldsm_x4(r4, &sB[buf][nb + (mi >> 1) * 8 + rr][ks + (mi & 1) * 8]);
                } else {
                    ldsm_x4_t(r4, &sB[buf][ks + (mi & 1) * 8 + rr][nb + (mi >> 1) * 8]);
                }
                bf[2 * jj][0] = r4[0];
                bf[2 * jj][1] = r4[1];
                bf[2 * jj + 1][0] = r4[2];
                bf[2 * jj + 1][1] = r4[3];
            }
#pragma unroll
            for (int i = 0; i < MI; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j][0], bf[j][1]);
        }
        __syncthreads();
    }

    const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + wm + i * 16 + gid;
            const int n = n0 + wn + j * 8 + tig * 2;
            if (n < p.N) {
                if (m < p.M) p.epilogue(m, n, acc[i][j][0], acc[i][j][1]);
                if (m + 8 < p.M) p.epilogue(m + 8, n, acc[i][j][2], acc[i][j][3]);
            }
        }
}

}  // namespace sg
}  // namespace dc
