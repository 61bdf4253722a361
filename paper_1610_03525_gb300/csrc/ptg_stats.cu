// ptg_stats.cu -- map statistics of the paper's quality measurements
// (Thorimbert & Chopard, arXiv:1610.03525, Sec. 5): coastline box counts for
// the fractal dimension (Sec. 5.3) and the frequency distributions of height
// and slope norm (Sec. 5.1), computed on the device from generated maps.
#include <cuda_runtime.h>

#include <cstdint>

#include "ptg_kernels.h"

namespace ptg {
namespace {

constexpr int kThreads = 256;

// Level 0 of the box pyramid: one byte per unit square (x, y) .. (x+1, y+1)
// of samples, bit 0 = a corner below `level`, bit 1 = a corner at or above.
__global__ void __launch_bounds__(kThreads) box_level0_kernel(const float* __restrict__ map, long long W,
                                                              long long H, float level, uint8_t* __restrict__ flags,
                                                              unsigned long long* __restrict__ count)
{
    const long long nx = W - 1, n = nx * (H - 1);
    unsigned int mine = 0;
    for (long long e = blockIdx.x * (long long)kThreads + threadIdx.x; e < n; e += (long long)gridDim.x * kThreads) {
        const long long y = e / nx, x = e - y * nx;
        const float* p = map + y * W + x;
        const float a = p[0], b = p[1], c = p[W], d = p[W + 1];
        const uint8_t f = (uint8_t)(((a < level) | (b < level) | (c < level) | (d < level)) |
                                    (((a >= level) | (b >= level) | (c >= level) | (d >= level)) << 1));
        flags[e] = f;
        mine += (f == 3);
    }
    __shared__ unsigned int s_sum;
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    if (mine) atomicAdd(&s_sum, mine);
    __syncthreads();
    if (threadIdx.x == 0 && s_sum) atomicAdd(count, (unsigned long long)s_sum);
}

// Level k from level k-1: a square of side 2^k is the union of (up to) four
// squares of side 2^(k-1); its flags are their OR.
__global__ void __launch_bounds__(kThreads) box_level_kernel(const uint8_t* __restrict__ child, long long cnx,
                                                             long long cny, uint8_t* __restrict__ parent,
                                                             long long pnx, long long pny,
                                                             unsigned long long* __restrict__ count)
{
    const long long n = pnx * pny;
    unsigned int mine = 0;
    for (long long e = blockIdx.x * (long long)kThreads + threadIdx.x; e < n; e += (long long)gridDim.x * kThreads) {
        const long long y = e / pnx, x = e - y * pnx;
        const long long x0 = 2 * x, y0 = 2 * y;
        uint8_t f = child[y0 * cnx + x0];
        if (x0 + 1 < cnx) f |= child[y0 * cnx + x0 + 1];
        if (y0 + 1 < cny) {
            f |= child[(y0 + 1) * cnx + x0];
            if (x0 + 1 < cnx) f |= child[(y0 + 1) * cnx + x0 + 1];
        }
        parent[e] = f;
        mine += (f == 3);
    }
    __shared__ unsigned int s_sum;
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    if (mine) atomicAdd(&s_sum, mine);
    __syncthreads();
    if (threadIdx.x == 0 && s_sum) atomicAdd(count, (unsigned long long)s_sum);
}

// Height or slope-norm histogram: bins + 2 counters per CTA in shared memory,
// then added to the global ones.  The arithmetic is rounded step by step (no
// contraction) so that every bin decision is the same as the FP32 definition.
__global__ void __launch_bounds__(kThreads) histogram_kernel(const float* __restrict__ maps, long long W, long long H,
                                                             long long count, float lo, float scale, int bins,
                                                             int what, unsigned long long* __restrict__ hist)
{
    extern __shared__ unsigned int s_hist[];
    for (int b = threadIdx.x; b < bins + 2; b += kThreads) s_hist[b] = 0;
    __syncthreads();
    const long long per = W * H, n = per * count;
    for (long long e = blockIdx.x * (long long)kThreads + threadIdx.x; e < n; e += (long long)gridDim.x * kThreads) {
        const long long f = e / per, r = e - f * per, y = r / W, x = r - y * W;
        const float* m = maps + f * per;
        float v;
        if (what == 0) {
            v = m[r];
        } else {
            if (x == 0 || y == 0 || x == W - 1 || y == H - 1) continue;
            const float dx = __fmul_rn(__fsub_rn(m[r + 1], m[r - 1]), 0.5f);
            const float dy = __fmul_rn(__fsub_rn(m[r + W], m[r - W]), 0.5f);
            v = __fsqrt_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)));
        }
        const float fb = floorf(__fmul_rn(__fsub_rn(v, lo), scale));
        const int b = !(fb >= 0.0f) ? 0 : (fb >= (float)bins ? bins + 1 : (int)fb + 1);
        atomicAdd(&s_hist[b], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < bins + 2; b += kThreads)
        if (s_hist[b]) atomicAdd(&hist[b], (unsigned long long)s_hist[b]);
}

int grid_for(long long n, int num_sms)
{
    const long long want = (n + kThreads - 1) / kThreads, cap = (long long)num_sms * 8;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace

cudaError_t launch_box_counts(const float* map, long long W, long long H, float level, int levels, uint8_t* buf0,
                              uint8_t* buf1, unsigned long long* counts, int num_sms, cudaStream_t stream)
{
    long long nx = W - 1, ny = H - 1;
    box_level0_kernel<<<grid_for(nx * ny, num_sms), kThreads, 0, stream>>>(map, W, H, level, buf0, counts);
    cudaError_t e = cudaGetLastError();
    uint8_t* child = buf0;
    uint8_t* parent = buf1;
    for (int k = 1; k < levels && e == cudaSuccess; ++k) {
        const long long px = (nx + 1) / 2, py = (ny + 1) / 2;
        box_level_kernel<<<grid_for(px * py, num_sms), kThreads, 0, stream>>>(child, nx, ny, parent, px, py,
                                                                              counts + k);
        e = cudaGetLastError();
        nx = px;
        ny = py;
        uint8_t* t = child;
        child = parent;
        parent = t;
    }
    return e;
}

cudaError_t launch_histogram(const float* maps, long long W, long long H, long long count, float lo, float scale,
                             int bins, int what, unsigned long long* hist, int num_sms, cudaStream_t stream)
{
    const size_t smem = sizeof(unsigned int) * (size_t)(bins + 2);
    histogram_kernel<<<grid_for(W * H * count, num_sms), kThreads, smem, stream>>>(maps, W, H, count, lo, scale, bins,
                                                                                   what, hist);
    return cudaGetLastError();
}

}  // namespace ptg
