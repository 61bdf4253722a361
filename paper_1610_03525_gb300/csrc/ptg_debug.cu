// ptg_debug.cu -- test hooks that run the generators' own device hash and
// fixed-point coordinate map on arbitrary inputs, so that lattice hashes and
// cell indices can be compared bit for bit with an independent implementation.
#include "ptg_device.cuh"
#include "ptg_kernels.h"

namespace ptg {
namespace {

__global__ void debug_hash_kernel(int dims, const uint32_t* __restrict__ keys, long long n, uint32_t* __restrict__ out)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += stride) {
        if (dims == 2) {
            uint32_t x = keys[3 * m], y = keys[3 * m + 1], z = keys[3 * m + 2];
            pcg3d(x, y, z);
            out[3 * m] = x;
            out[3 * m + 1] = y;
            out[3 * m + 2] = z;
        } else {
            uint32_t x = keys[4 * m], y = keys[4 * m + 1], z = keys[4 * m + 2], w = keys[4 * m + 3];
            pcg4d(x, y, z, w);
            out[4 * m] = x;
            out[4 * m + 1] = y;
            out[4 * m + 2] = z;
            out[4 * m + 3] = w;
        }
    }
}

__global__ void debug_axis_kernel(uint32_t origin_shifted, int s, int octave, const long long* __restrict__ j,
                                  long long n, uint32_t* __restrict__ cell, float* __restrict__ t)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += stride) {
        const uint32_t jj = (uint32_t)j[m];
        cell[m] = axis_cell(origin_shifted, jj, octave, s);
        t[m] = axis_t(jj, octave, s);
    }
}

// Evaluates one bounds check without any memory access at idx: in the debug
// build an out-of-range (idx, n) is recorded like a kernel's violation.
__global__ void bounds_selftest_kernel(int site, long long idx, long long n)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) (void)bounds_ok(site, idx, n);
}

int grid_for(long long n)
{
    long long b = (n + 255) / 256;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

cudaError_t launch_debug_hash(int dims, const uint32_t* keys, long long n, uint32_t* out, cudaStream_t stream)
{
    debug_hash_kernel<<<grid_for(n), 256, 0, stream>>>(dims, keys, n, out);
    return cudaGetLastError();
}

cudaError_t launch_debug_axis(long long origin, int s, int octave, const long long* j, long long n, uint32_t* cell,
                              float* t, cudaStream_t stream)
{
    const uint32_t o = (uint32_t)((unsigned long long)origin << octave);
    debug_axis_kernel<<<grid_for(n), 256, 0, stream>>>(o, s, octave, j, n, cell, t);
    return cudaGetLastError();
}

cudaError_t launch_bounds_selftest(int site, long long idx, long long n, cudaStream_t stream)
{
    bounds_selftest_kernel<<<1, 32, 0, stream>>>(site, idx, n);
    return cudaGetLastError();
}

}  // namespace ptg
