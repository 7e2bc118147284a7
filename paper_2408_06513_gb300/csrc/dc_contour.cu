// Contour lines of a density (Sec. 5: the original density's contours, drawn
// again after the transformation by moving their vertices with the samples).
//
// Marching squares on the pixel nodes: cell (i, j), 0 <= i, j < N - 1, has
// the corners v00 = f(i, j), v10 = f(i + 1, j), v11 = f(i + 1, j + 1),
// v01 = f(i, j + 1) at the node positions ((i + o) / N, (j + o) / N), o = 0 or
// 1/2 (pixel centres).  A corner is inside when f >= level.  Edges: e0 = v00-v10
// (row j), e1 = v10-v11 (column i + 1), e2 = v01-v11 (row j + 1), e3 = v00-v01
// (column i); a crossed edge A-B holds the vertex A + t (B - A) with
// t = (level - f(A)) / (f(B) - f(A)).  The two saddle cases take the side of
// the cell centre, the mean of the four corners summed as (v00 + v10) +
// (v11 + v01).  Every cell writes two segment slots (x0, y0, x1, y1) in
// domain units, NaN where it has fewer segments, so the output order is the
// cell order and needs no atomics.
#include <cmath>

#include "dc_internal.cuh"

namespace dc {

namespace {

// Segments of each case as edge pairs (first, second); 4 = none.  Cases 5
// and 10 (saddles) list the split for a centre outside; a centre inside uses
// the other split (kSaddleIn).
__constant__ signed char kSegs[16][4] = {
    {4, 4, 4, 4}, {3, 0, 4, 4}, {0, 1, 4, 4}, {3, 1, 4, 4},  //
    {1, 2, 4, 4}, {3, 0, 1, 2}, {0, 2, 4, 4}, {2, 3, 4, 4},  //
    {2, 3, 4, 4}, {0, 2, 4, 4}, {0, 1, 2, 3}, {1, 2, 4, 4},  //
    {3, 1, 4, 4}, {0, 1, 4, 4}, {3, 0, 4, 4}, {4, 4, 4, 4},
};
__constant__ signed char kSaddleIn[2][4] = {{0, 1, 2, 3}, {3, 0, 1, 2}};  // cases 5, 10

__device__ __forceinline__ float2 edge_vertex(int e, int i, int j, float off, float invN, float level, float v00,
                                              float v10, float v11, float v01)
{
    float a, b, x, y;
    switch (e) {
    case 0: a = v00; b = v10; break;
    case 1: a = v10; b = v11; break;
    case 2: a = v01; b = v11; break;
    default: a = v00; b = v01; break;
    }
    const float t = (level - a) / (b - a);
    switch (e) {
    case 0: x = ((float)i + off + t) * invN; y = ((float)j + off) * invN; break;
    case 1: x = ((float)(i + 1) + off) * invN; y = ((float)j + off + t) * invN; break;
    case 2: x = ((float)i + off + t) * invN; y = ((float)(j + 1) + off) * invN; break;
    default: x = ((float)i + off) * invN; y = ((float)j + off + t) * invN; break;
    }
    return make_float2(x, y);
}

__global__ void __launch_bounds__(256) contour_kernel(const float *__restrict__ f, int log2N, float level,
                                                      float off, float4 *__restrict__ segs)
{
    pdl_wait();
    const int N = 1 << log2N, M = N - 1;
    const int64_t cells = (int64_t)M * M;
    const float invN = 1.0f / (float)N;
    const float nan = __int_as_float(0x7fc00000);
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(c / M), i = (int)(c - (int64_t)j * M);
        const float *r0 = f + ((size_t)j << log2N), *r1 = r0 + N;
        const float v00 = r0[i], v10 = r0[i + 1], v11 = r1[i + 1], v01 = r1[i];
        const int k = (v00 >= level) | (v10 >= level) << 1 | (v11 >= level) << 2 | (v01 >= level) << 3;
        const signed char *sg = kSegs[k];
        if (k == 5 || k == 10) {
            const float centre = ((v00 + v10) + (v11 + v01)) * 0.25f;
            if (centre >= level) sg = kSaddleIn[k == 10];
        }
        float4 out[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (sg[2 * s] < 4) {
                const float2 p = edge_vertex(sg[2 * s], i, j, off, invN, level, v00, v10, v11, v01);
                const float2 q = edge_vertex(sg[2 * s + 1], i, j, off, invN, level, v00, v10, v11, v01);
                out[s] = make_float4(p.x, p.y, q.x, q.y);
            } else {
                out[s] = make_float4(nan, nan, nan, nan);
            }
        }
        segs[2 * c] = out[0];
        segs[2 * c + 1] = out[1];
    }
}

}  // namespace

cudaError_t launch_contour(cudaStream_t s, const float *field, int log2N, float level, int pixel_center,
                           float4 *segs)
{
    const int64_t M = ((int64_t)1 << log2N) - 1;
    const int64_t cells = M * M;
    int64_t blocks = (cells + 255) / 256;
    if (blocks > device_sms() * 16) blocks = device_sms() * 16;
    if (blocks < 1) blocks = 1;
    return launch_kernel(contour_kernel, dim3((unsigned)blocks), dim3(256), 0, s, field, log2N, level,
                         pixel_center ? 0.5f : 0.0f, segs);
}

}  // namespace dc
