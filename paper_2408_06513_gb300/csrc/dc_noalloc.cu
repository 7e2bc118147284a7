// integral_images_u32_noalloc(): the exact uint64 integral images of a
// uint32 grid without a context and without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need
// the integral images: applications that hand out all device memory from
// their own pool or budget and do not let a library allocate behind their
// back, and latency-bound loops that cannot afford the device-wide
// synchronisation that cudaMalloc and cudaFree may imply.  This entry point
// keeps its band aggregates and carries in one fixed array that the library
// declares at file scope; the caller passes only the grid and the outputs.
#include <cstdio>
#include <mutex>

#include "dc_internal.cuh"

using namespace dc;

namespace {

// 8.5 MiB: room for the aggregates and carries of the largest supported
// grid, 1024 x 1024 (7,299,360 bytes with one band per SM of a 152-SM GPU; on
// a GPU with more SMs the bands are made taller until they fit).  Every GPU
// that loads the library holds this array until the process exits.
constexpr size_t kNoallocScratchBytes = DC_NOALLOC_SCRATCH_BYTES;
constexpr uint32_t kNoallocMaxLog2Res = DC_NOALLOC_MAX_LOG2_RES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[256] = {};  // device address of the array, per device ordinal

thread_local char g_noalloc_msg[256];

dc_status noalloc_fail(dc_status st)
{
    set_last_error(g_noalloc_msg);
    return st;
}

}  // namespace

extern "C" dc_status integral_images_u32_noalloc(const uint32_t *grid, uint32_t log2_res, uint64_t *alpha_out,
                                                 uint64_t *alpha_t_out, void *cuda_stream)
{
    if (log2_res < 4) {
        snprintf(g_noalloc_msg, sizeof(g_noalloc_msg), "log2_res = %u is below 4", log2_res);
        return noalloc_fail(DC_ERR_NOT_POW2);
    }
    if (log2_res > kNoallocMaxLog2Res) {
        snprintf(g_noalloc_msg, sizeof(g_noalloc_msg),
                 "log2_res = %u exceeds the no-allocation limit of %u (fixed scratch of %zu bytes); "
                 "use integral_images_u32() with a context",
                 log2_res, kNoallocMaxLog2Res, kNoallocScratchBytes);
        return noalloc_fail(DC_ERR_INVALID_ARG);
    }
    if (!grid || (reinterpret_cast<uintptr_t>(grid) & 15) || (reinterpret_cast<uintptr_t>(alpha_out) & 15) ||
        (reinterpret_cast<uintptr_t>(alpha_t_out) & 15)) {
        snprintf(g_noalloc_msg, sizeof(g_noalloc_msg), "grid null, or a pointer not 16-byte aligned");
        return noalloc_fail(DC_ERR_INVALID_ARG);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        cudaGetLastError();
        snprintf(g_noalloc_msg, sizeof(g_noalloc_msg), "no current CUDA device");
        return noalloc_fail(DC_ERR_CUDA);
    }
    // the grid and the outputs must be device memory of the current device:
    // the kernels run there and the scratch array is that device's copy
    {
        const void *ptrs[3] = {grid, alpha_out, alpha_t_out};
        const char *names[3] = {"grid", "alpha_out", "alpha_t_out"};
        for (int k = 0; k < 3; ++k) {
            if (!ptrs[k]) continue;
            cudaPointerAttributes at{};
            if (cudaPointerGetAttributes(&at, ptrs[k]) != cudaSuccess) {
                cudaGetLastError();
                at.type = cudaMemoryTypeUnregistered;
            }
            if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev) {
                snprintf(g_noalloc_msg, sizeof(g_noalloc_msg),
                         "%s is not device memory of the current device %d (memory type %d, device %d)", names[k],
                         dev, (int)at.type, at.device);
                return noalloc_fail(DC_ERR_INVALID_ARG);
            }
        }
    }
    void *scratch = nullptr;
    {
        // once per device, with that device current: the array's device address
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                snprintf(g_noalloc_msg, sizeof(g_noalloc_msg), "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
                return noalloc_fail(DC_ERR_CUDA);
            }
            // kernel attributes (dynamic shared memory of the band kernels)
            const cudaError_t ek = prepare_kernels();
            if (ek != cudaSuccess) {
                snprintf(g_noalloc_msg, sizeof(g_noalloc_msg), "kernel attributes: %s", cudaGetErrorString(ek));
                return noalloc_fail(DC_ERR_CUDA);
            }
            g_noalloc_ptr[dev] = p;
        }
        scratch = g_noalloc_ptr[dev];
    }

    // the automatic band height, made taller while the bands' aggregates and
    // carries do not fit the array (the sums are exact for any height)
    const int sms = device_sms();
    BandGeom g = make_band_geom((int)log2_res, 0, sms);
    auto agg_size = [](const BandGeom &q) {
        return ((size_t)q.nb * q.agg_stride * sizeof(unsigned long long) + 255) & ~size_t(255);
    };
    // per band the lanes its final pass reads, then the 5N totals
    auto carry_size = [](const BandGeom &q) {
        return ((size_t)q.nb * ((3 * q.N + 2 * q.T - 2 + 3) & ~3) + (size_t)q.lanes) * sizeof(unsigned long long);
    };
    while (agg_size(g) + carry_size(g) > kNoallocScratchBytes && g.T < 64 && g.T < g.N)
        g = make_band_geom((int)log2_res, g.T + 1, sms);
    const size_t agg_bytes = agg_size(g);
    const size_t carry_bytes = carry_size(g);
    if (agg_bytes + carry_bytes > kNoallocScratchBytes) {
        snprintf(g_noalloc_msg, sizeof(g_noalloc_msg), "grid needs %zu scratch bytes, limit %zu",
                 agg_bytes + carry_bytes, kNoallocScratchBytes);
        return noalloc_fail(DC_ERR_INVALID_ARG);
    }
    // No element of the scratch has to start at zero: each one the kernels
    // read is written earlier in the same call.  There is no status word
    // here, so an expired bounded wait inside a kernel is not reported.
    BandArgs a{};
    a.src = grid;
    a.agg = scratch;
    a.agg_stride = g.agg_stride;
    void *carry = static_cast<unsigned char *>(scratch) + agg_bytes;
    a.carry = carry;
    a.alpha_out = alpha_out;
    a.alpha_t_out = alpha_t_out;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = launch_band_agg(s, g, MODE_GRID64, a);
    if (e == cudaSuccess) e = launch_carry(s, g, MODE_GRID64, DC_CARRY_COMPENSATED, a.agg, carry);
    if (e == cudaSuccess) e = launch_band_final(s, g, MODE_GRID64, a);
    if (e != cudaSuccess) {
        snprintf(g_noalloc_msg, sizeof(g_noalloc_msg), "launch: %s", cudaGetErrorString(e));
        return noalloc_fail(DC_ERR_CUDA);
    }
    return DC_OK;
}
