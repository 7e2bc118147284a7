// Fifth-generation tensor-core (tcgen05) implicit GEMM for the forward
// convolutions of the surrogate network.
//
// C[m][n] = sum_k A[m][k] B[n][k] with bf16 A (im2col of the activations)
// and B (weights, K contiguous), FP32 accumulation in tensor memory.  One
// CTA of 256 threads computes a 128 x N tile (N = all output channels,
// 32..256, a power of two); K advances in stages of 64 through a ring of
// UM_STAGES shared-memory stages, UM_STAGES - 1 ahead of the tensor core.
// A (the im2col rows) is staged by every thread in 16-byte row segments with
// cp.async (zero fill where the convolution pads); B arrives by tensor memory
// access (cp.async.bulk.tensor, one 64 x N box a stage, issued by one thread
// and counted in bytes on the stage's mbarrier), or with cp.async where no
// tensor map could be made.  A landed stage is fenced into the async proxy
// and one thread issues four tcgen05.mma (K = 16 each) and commits them to
// the stage's mbarrier, which the refill of that stage waits for.  After the
// last stage the accumulator is read back with tcgen05.ld (warp w reads
// tensor-memory lanes 32 (w % 4) .. + 31, i.e. tile rows, of its half of
// each 32-column chunk) and handed to the problem's epilogue.
//
// Shared-memory operand layouts (K-major).  A, and B staged by cp.async: no
// swizzle, 8-row x 16-byte core matrices of 128 contiguous bytes; core matrix
// (row group g, k group q) at (g * 8 + q) * 128, so neighbours along K are
// 128 bytes apart (leading byte offset) and neighbours along M / N 1024
// bytes apart (stride byte offset).  B by tensor memory access: rows of 128
// bytes in the 128-byte swizzle (see um_desc_sw128).  Instruction
// descriptor: FP32 accumulator, BF16 A and B, both K-major, N >> 3 at bit 17,
// M >> 4 at bit 24.
#pragma once

#include <cuda.h>  // CUtensorMap (the encoder is fetched through the runtime)
#include <cuda_bf16.h>
#include <stdint.h>

#include "dc_sg_gemm.cuh"

namespace dc {
namespace sg {

constexpr int UM_TM = 128, UM_TK = 64, UM_THREADS = 256, UM_STAGES = 3;

__device__ __forceinline__ uint32_t um_smem(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ uint64_t um_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(128u >> 4) << 16;   // leading byte offset: next core matrix along K
    d |= (uint64_t)(1024u >> 4) << 32;  // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;             // descriptor version
    return d;                           // base offset 0, no swizzle
}

// The same for an operand that the tensor-memory-access unit stored with the
// 128-byte swizzle (rows of 64 bf16 = 128 B, 8-row groups 1024 B apart,
// 16-byte chunks of row r permuted by r mod 8): layout type 2 (128-byte
// swizzle) at bits 61..63; the leading byte offset is unused for a K-major
// swizzled operand (1 by convention).  A K step of 16 elements advances the
// start address by 32 bytes inside the swizzled rows.
__device__ __forceinline__ uint64_t um_desc_sw128(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;              // leading byte offset (unused)
    d |= (uint64_t)(1024u >> 4) << 32;   // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;              // descriptor version
    d |= (uint64_t)2 << 61;              // 128-byte swizzle
    return d;
}

// One 2-D tile (box) of a tensor map into shared memory, completion counted
// on an mbarrier in bytes (plain, single-GPU; no multicast).
__device__ __forceinline__ void um_tma_2d(void *smem_dst, const CUtensorMap *map, int c0, int c1,
                                          unsigned long long *mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(um_smem(smem_dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(um_smem(mbar))
        : "memory");
}
__device__ __forceinline__ void um_mbar_expect(unsigned long long *m, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(um_smem(m)), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint32_t um_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void um_mbar_init(unsigned long long *m)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(um_smem(m)) : "memory");
}
__device__ __forceinline__ bool um_mbar_try(unsigned long long *m, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(um_smem(m)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded: false after one second
__device__ __noinline__ bool um_mbar_wait_slow(unsigned long long *m, unsigned parity)
{
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (!um_mbar_try(m, parity)) {
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > 1000000000ull) return false;
    }
    return true;
}
__device__ __forceinline__ bool um_mbar_wait(unsigned long long *m, unsigned parity)
{
    return um_mbar_try(m, parity) || um_mbar_wait_slow(m, parity);
}

__device__ __forceinline__ void um_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void um_commit(unsigned long long *m)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(um_smem(m))
                 : "memory");
}
__device__ __forceinline__ void um_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// dynamic shared memory: UM_STAGES x (A 16 KB + B N * 128 B), 1 KB alignment slack
inline size_t umma_smem_bytes(int N)
{
    return UM_STAGES * ((size_t)UM_TM * UM_TK * 2 + (size_t)N * UM_TK * 2) + 1024;
}

// P: as for gemm_kernel (K_CONTIG A and B), with N a power of two in
// [32, 256] and M a multiple of 128.  status: device word, DC_ERR_TIMEOUT
// when a bounded wait expired.
// tmB / use_tma: with use_tma the B tiles (64 k x N rows of the K-contiguous
// weights) arrive by tensor memory access in the 128-byte swizzled layout,
// one copy a stage issued by thread 0 and counted on the stage's s_tb
// mbarrier; otherwise every thread stages them with cp.async.
template <class P>
__global__ void __launch_bounds__(UM_THREADS) umma_gemm_kernel(P p, int k_per_split, unsigned *status,
                                                               const __grid_constant__ CUtensorMap tmB, int use_tma)
{
    extern __shared__ unsigned char um_dyn[];
    __shared__ __align__(8) unsigned long long s_mbar[UM_STAGES + 1];
    __shared__ __align__(8) unsigned long long s_tb[UM_STAGES];
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = p.N;
    const uint32_t ncols = N < 32 ? 32u : (uint32_t)N;
    // 1024-byte aligned operand area
    unsigned char *base =
        um_dyn + ((1024u - (um_smem(um_dyn) & 1023u)) & 1023u);
    const size_t stage_bytes = (size_t)UM_TM * UM_TK * 2 + (size_t)N * UM_TK * 2;
    auto sA = [&](int st) { return base + st * stage_bytes; };
    auto sB = [&](int st) { return base + st * stage_bytes + UM_TM * UM_TK * 2; };

    const int m0 = blockIdx.x * UM_TM;
    const int k_begin = blockIdx.z * k_per_split;
    const int k_end = min(p.K, k_begin + k_per_split);

    pdl_wait();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(um_smem(&s_tmem)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i <= UM_STAGES; ++i) um_mbar_init(&s_mbar[i]);
        for (int i = 0; i < UM_STAGES; ++i) um_mbar_init(&s_tb[i]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = um_idesc(UM_TM, N);

    bool dead = false;
    const int nk = k_end > k_begin ? (k_end - k_begin + UM_TK - 1) / UM_TK : 0;
    auto load = [&](int kt, int st) {
        const int k0 = k_begin + kt * UM_TK;
        // A: 128 rows x 8 segments; consecutive threads take consecutive rows
#pragma unroll
        for (int i = 0; i < UM_TM * UM_TK / 8 / UM_THREADS; ++i) {
            const int c = tid + i * UM_THREADS;
            const int r = c & (UM_TM - 1), q = c >> 7;
            const int m = m0 + r, k = k0 + q * 8;
            cp_async16(sA(st) + ((r >> 3) * 8 + q) * 128 + (r & 7) * 16,
                       (m < p.M && k < k_end) ? p.a_chunk(m, k) : nullptr, p.base());
        }
        // B: N rows x 8 segments
        if (use_tma) {
            if (tid == 0) {
                um_mbar_expect(&s_tb[st], (uint32_t)N * UM_TK * 2);
                um_tma_2d(sB(st), &tmB, k0, 0, &s_tb[st]);
            }
            return;
        }
        for (int c = tid; c < N * 8; c += UM_THREADS) {
            const int r = c & (N - 1), q = c / N;
            const int k = k0 + q * 8;
            cp_async16(sB(st) + ((r >> 3) * 8 + q) * 128 + (r & 7) * 16, k < k_end ? p.b_chunk(k, r) : nullptr,
                       p.base());
        }
    };
    // prologue: UM_STAGES - 1 stages in flight (one commit group each, empty if past the end)
    for (int s = 0; s < UM_STAGES - 1; ++s) {
        if (s < nk) load(s, s);
        cp_async_commit();
    }
    for (int kt = 0; kt < nk; ++kt) {
        const int st = kt % UM_STAGES;
        const int kn = kt + UM_STAGES - 1;  // the stage refilled now
        if (kn < nk) {
            const int sn = kn % UM_STAGES;
            // its previous contents (k-step kn - UM_STAGES) must have been consumed
            if (kn >= UM_STAGES && !dead && !um_mbar_wait(&s_mbar[sn], ((kn - UM_STAGES) / UM_STAGES) & 1))
                dead = true;
            load(kn, sn);
        }
        cp_async_commit();
        asm volatile("cp.async.wait_group %0;\n" ::"n"(UM_STAGES - 1));  // k-step kt has landed
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        // the stage's B tile by tensor memory access (waited for by every
        // thread, so that a timeout is seen by all; a copy in flight is always
        // waited for, also after a timeout)
        if (use_tma && !um_mbar_wait(&s_tb[st], (kt / UM_STAGES) & 1)) dead = true;
        __syncthreads();
        if (tid == 0 && !dead) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = um_smem(sA(st)), b0 = um_smem(sB(st));
#pragma unroll
            for (int kk = 0; kk < UM_TK / 16; ++kk) {
                const uint64_t bd = use_tma ? um_desc_sw128(b0 + kk * 32) : um_desc(b0 + kk * 256);
                um_mma(tmem, um_desc(a0 + kk * 256), bd, idesc, (kt > 0 || kk > 0) ? 1u : 0u);
            }
            um_commit(&s_mbar[st]);
        }
    }
    cp_async_wait_all();
    if (tid == 0) um_commit(&s_mbar[UM_STAGES]);  // completes when every MMA above has
    if (!dead && !um_mbar_wait(&s_mbar[UM_STAGES], 0)) dead = true;
    if (dead && status) atomicOr(status, (unsigned)DC_ERR_TIMEOUT);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // epilogue, 32 columns at a time: warp w reads tensor-memory lanes
    // 32 (w % 4) .. + 31 (tile rows) of columns c0 + 16 (w / 4) .. + 15 with
    // tcgen05.ld; the rows go through shared memory (the operand stages are
    // free now) so that consecutive lanes hand the problem's epilogue
    // consecutive column pairs of one row.
    float *sT = reinterpret_cast<float *>(base);  // [2][128][17]
    const int wg = warp >> 2, wq = warp & 3;
    for (int c0 = 0; c0 < N; c0 += 32) {
        uint32_t v[16];
        um_ld16(tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)(c0 + 16 * wg), v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        __syncthreads();  // previous chunk's readers are done
        float *sTw = sT + wg * (UM_TM * 17);
#pragma unroll
        for (int j = 0; j < 16; ++j) sTw[(wq * 32 + lane) * 17 + j] = __uint_as_float(v[j]);
        __syncthreads();
        if (nk > 0) {
            // 128 rows x 16 pairs: thread t takes pair t & 15 of rows t >> 4, t >> 4 + 16, ...
            const int pr = tid & 15;
            const float *src = sT + (pr >> 3) * (UM_TM * 17);
            const int pc = pr & 7;
#pragma unroll
            for (int rr = tid >> 4; rr < UM_TM; rr += UM_THREADS / 16) {
                const int m = m0 + rr;
                if (m < p.M) p.epilogue(m, c0 + 2 * pr, src[rr * 17 + 2 * pc], src[rr * 17 + 2 * pc + 1]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

}  // namespace sg
}  // namespace dc
