// ptg_fbm2d.cu -- fused all-octave 2D generator for the polynomial noise of
// Thorimbert & Chopard (arXiv:1610.03525) and for Perlin's polynomial.
//
// One CTA makes a 64 x 64 tile of samples with 128 threads; each thread owns
// 4 rows x 8 consecutive columns and keeps their fractal sums (Sec. 4) in
// registers across all octaves, then writes each sample once.
//
// Per octave i (cells of spc_i = spc / 2^i samples):
//   staged octave (spc_i >= 2): before the octave loop the CTA hashes the
//     corners of every cell its tile touches (Sec. 4.1's C_init, once per cell)
//     into shared memory, pre-scaled by the octave amplitude, and tabulates the
//     per-axis basis (S, B0, B1) of each of its 64 columns and 64 rows (the
//     space-only terms that the paper precomputes, Sec. 5.2).  The evaluation
//     (C_eval) is separable: for each row y of a cell it collapses the cell to
//     a 1D function of x,
//        h(x, y) = V0 + S(x) (V1 - V0) + B0(x) F0 + B1(x) F1,
//        V_a = v_a0 + S(y) (v_a1 - v_a0) + B0(y) g_a0 + B1(y) g_a1,
//        F_a = f_a0 + S(y) (f_a1 - f_a0),
//     which is the tensor-product Hermite cell (C1: cubic, C2: quintic) of
//     Eq. (polynomial) with the corner constraints of Eq. (mixedderiv) and
//     zero mixed derivatives, or Perlin's polynomial (Sec. 3.2) with v = 0 and
//     its own B0, B1.  Per sample that is 4 floating-point operations.
//   lattice octave (spc_i <= 1): every sample is a lattice point, where the
//     cell polynomial equals the corner value: one hash per sample (zero for
//     Perlin, whose value at lattice points is zero).
#include "ptg_device.cuh"
#include "ptg_kernels.h"

namespace ptg {
namespace {

constexpr int kTW = 64, kTH = 64, kThreads = 128;
constexpr int kCols = 8, kRows = 4;  // per thread

// Shared-memory layout (float4 units): x-basis [nst][8 cols][8 tx],
// y-basis [nst][4 rows][16 ty], then the staged corners.
__device__ __forceinline__ int xlut_index(int i, int col) { return i * 64 + (col & 7) * 8 + (col >> 3); }
__device__ __forceinline__ int ylut_index(int i, int row) { return i * 64 + (row & 3) * 16 + (row >> 2); }

template <int METHOD>
__device__ __forceinline__ void stage_tile(const FieldPlan& P, float4* sm, int j0x, int j0y, int s)
{
    const int tid = threadIdx.x;
    float4* xlut = sm;
    float4* ylut = sm + P.nst * 64;
    float4* corners = sm + P.nst * 128;
    for (int e = tid; e < P.nst * 64; e += kThreads) {
        const int i = e >> 6, c = e & 63;
        xlut[xlut_index(i, c)] = axis_basis<METHOD>(axis_t((uint32_t)(j0x + c), i, s));
        ylut[ylut_index(i, c)] = axis_basis<METHOD>(axis_t((uint32_t)(j0y + c), i, s));
    }
    for (int e = tid; e < P.ncorner; e += kThreads) {
        int i = 0;
        while (i + 1 < P.nst && e >= P.oct[i + 1].coff) ++i;
        const OctPlan& op = P.oct[i];
        const int local = e - op.coff;
        const int cy = local / op.ncx, cx = local - cy * op.ncx;
        uint32_t x = op.ox + ((uint32_t)j0x >> op.k) + (uint32_t)cx;
        uint32_t y = op.oy + ((uint32_t)j0y >> op.k) + (uint32_t)cy;
        uint32_t z = op.key;
        pcg3d(x, y, z);
        float4 c;
        if (METHOD == kC1 || METHOD == kC2) {
            c = make_float4(unit_value(x) * op.amp, unit_value(y) * op.ampw, unit_value(z) * op.ampw, 0.0f);
        } else {
            c = make_float4(0.0f, unit_value(y) * op.amp, unit_value(z) * op.amp, 0.0f);
        }
        corners[e] = c;
    }
}

// One staged octave for cells CW samples wide along x and RH rows tall.
template <int CW, int RH>
__device__ __forceinline__ void staged_octave(float (&acc)[kRows][kCols], const float4* __restrict__ sm,
                                              const FieldPlan& P, int i, int tx, int ty)
{
    const OctPlan& op = P.oct[i];
    const float4* ylut = sm + P.nst * 64;
    const float4* cg = sm + P.nst * 128 + op.coff;
    const int k = op.k, ncx = op.ncx;
    float4 xb[kCols];
#pragma unroll
    for (int c = 0; c < kCols; ++c) xb[c] = sm[xlut_index(i, tx * 8 + c)];
#pragma unroll
    for (int yq = 0; yq < kRows / RH; ++yq) {
        const int lcy = (ty * kRows + yq * RH) >> k;
        float4 yb[RH];
#pragma unroll
        for (int r = 0; r < RH; ++r) yb[r] = ylut[ylut_index(i, ty * kRows + yq * RH + r)];
#pragma unroll
        for (int xq = 0; xq < kCols / CW; ++xq) {
            const int lcx = (tx * kCols + xq * CW) >> k;
            const float4* c = cg + lcy * ncx + lcx;
            const float4 c00 = c[0], c10 = c[1], c01 = c[ncx], c11 = c[ncx + 1];
            const float dv0 = c01.x - c00.x, dv1 = c11.x - c10.x;
            const float df0 = c01.y - c00.y, df1 = c11.y - c10.y;
#pragma unroll
            for (int r = 0; r < RH; ++r) {
                const float Sy = yb[r].x, B0y = yb[r].y, B1y = yb[r].z;
                const float V0 = fmaf(B1y, c01.z, fmaf(B0y, c00.z, fmaf(Sy, dv0, c00.x)));
                const float V1 = fmaf(B1y, c11.z, fmaf(B0y, c10.z, fmaf(Sy, dv1, c10.x)));
                const float F0 = fmaf(Sy, df0, c00.y);
                const float F1 = fmaf(Sy, df1, c10.y);
                const float dV = V1 - V0;
#pragma unroll
                for (int q = 0; q < CW; ++q) {
                    const int col = xq * CW + q;
                    const float h = fmaf(xb[col].z, F1, fmaf(xb[col].y, F0, fmaf(xb[col].x, dV, V0)));
                    acc[yq * RH + r][col] += h;
                }
            }
        }
    }
}

// One lattice octave: every sample sits on a lattice point.
__device__ __forceinline__ void lattice_octave(float (&acc)[kRows][kCols], const OctPlan& op, uint32_t jx,
                                               uint32_t jy)
{
    const int sh = op.k;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const uint32_t iy = op.oy + ((jy + r) << sh);
#pragma unroll
        for (int c = 0; c < kCols; ++c) {
            const uint32_t ix = op.ox + ((jx + c) << sh);
            acc[r][c] = fmaf(op.amp, unit_value(pcg3d_value(ix, iy, op.key)), acc[r][c]);
        }
    }
}

template <typename OutT>
__device__ __forceinline__ void store_tile(const FieldPlan& P, const float (&acc)[kRows][kCols], int x0, int y0)
{
    OutT* out = reinterpret_cast<OutT*>(P.out);
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const int y = y0 + r;
        if (y >= P.H) break;
        OutT* row = out + (size_t)y * (size_t)P.W;
        if (P.vec_ok && x0 + kCols <= P.W) {
            if (sizeof(OutT) == 4) {
                float4* p = reinterpret_cast<float4*>(row + x0);
                p[0] = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
                p[1] = make_float4(acc[r][4], acc[r][5], acc[r][6], acc[r][7]);
            } else {
                __half2 h[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) h[q] = __floats2half2_rn(acc[r][2 * q], acc[r][2 * q + 1]);
                *reinterpret_cast<uint4*>(row + x0) = *reinterpret_cast<const uint4*>(h);
            }
        } else {
#pragma unroll
            for (int c = 0; c < kCols; ++c)
                if (x0 + c < P.W) store1(row + x0 + c, acc[r][c]);
        }
    }
}

// Whole tile: stage, evaluate all octaves, store.
template <int METHOD, typename OutT>
__device__ __forceinline__ void fbm2d_tile(const FieldPlan& P, float4* sm, int s, int bx, int by)
{
    const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
    const int x0 = bx * kTW, y0 = by * kTH;            // output tile origin
    const int j0x = x0 + P.jx0, j0y = y0 + P.jy0;      // sample indices
    stage_tile<METHOD>(P, sm, j0x, j0y, s);
    __syncthreads();
    float acc[kRows][kCols];
#pragma unroll
    for (int r = 0; r < kRows; ++r)
#pragma unroll
        for (int c = 0; c < kCols; ++c) acc[r][c] = 0.0f;
    for (int i = 0; i < P.N; ++i) {
        const int mode = P.oct[i].mode;
        if (mode == kModeRun8) staged_octave<8, 4>(acc, sm, P, i, tx, ty);
        else if (mode == kModeRun4) staged_octave<4, 4>(acc, sm, P, i, tx, ty);
        else if (mode == kModeRun2) staged_octave<2, 2>(acc, sm, P, i, tx, ty);
        else if (METHOD == kC1 || METHOD == kC2)
            lattice_octave(acc, P.oct[i], (uint32_t)(j0x + tx * kCols), (uint32_t)(j0y + ty * kRows));
    }
    store_tile<OutT>(P, acc, x0 + tx * kCols, y0 + ty * kRows);
}

template <int METHOD, typename OutT>
__global__ void __launch_bounds__(kThreads) fbm2d_kernel(const __grid_constant__ FieldPlan P, int s)
{
    extern __shared__ float4 sm[];
    fbm2d_tile<METHOD, OutT>(P, sm, s, blockIdx.x, blockIdx.y);
}

// Persistent batched generator: resident CTAs pull tiles of many fields from
// one work counter.  Field f owns tiles [tile_start[f], tile_start[f+1]); its
// plan is copied to shared memory when a CTA moves to it.  Every tile runs the
// same code as the single-field kernel, so results are identical.
__global__ void __launch_bounds__(kThreads) fbm2d_batch_kernel(const FieldPlan* __restrict__ plans,
                                                               const long long* __restrict__ tile_start, int n,
                                                               unsigned long long* __restrict__ counter)
{
    extern __shared__ float4 sm[];
    __shared__ FieldPlan plan;
    __shared__ long long s_tile;
    __shared__ int s_field;
    const long long total = tile_start[n];
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            const long long t = (long long)atomicAdd(counter, 1ULL);
            s_tile = t;
            if (t < total) {
                int lo = 0, hi = n - 1;  // last field whose first tile is <= t
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (tile_start[mid] <= t) lo = mid;
                    else hi = mid - 1;
                }
                s_field = lo;
            }
        }
        __syncthreads();
        const long long t = s_tile;
        if (t >= total) break;
        const int f = s_field;
        if (f != cur) {
            const int4* src = reinterpret_cast<const int4*>(plans + f);
            int4* dst = reinterpret_cast<int4*>(&plan);
            for (int q = threadIdx.x; q < (int)(sizeof(FieldPlan) / 16); q += kThreads) dst[q] = src[q];
            cur = f;
            __syncthreads();
        }
        const long long local = t - tile_start[f];
        const int bx = (int)(local % plan.tiles_x), by = (int)(local / plan.tiles_x);
        const int s = plan.s;
        const bool f16 = plan.dtype == 1;
        switch (plan.method) {
        case kC1:
            if (f16) fbm2d_tile<kC1, __half>(plan, sm, s, bx, by);
            else fbm2d_tile<kC1, float>(plan, sm, s, bx, by);
            break;
        case kC2:
            if (f16) fbm2d_tile<kC2, __half>(plan, sm, s, bx, by);
            else fbm2d_tile<kC2, float>(plan, sm, s, bx, by);
            break;
        case kPerlinS5:
            if (f16) fbm2d_tile<kPerlinS5, __half>(plan, sm, s, bx, by);
            else fbm2d_tile<kPerlinS5, float>(plan, sm, s, bx, by);
            break;
        default:
            if (f16) fbm2d_tile<kPerlinS3, __half>(plan, sm, s, bx, by);
            else fbm2d_tile<kPerlinS3, float>(plan, sm, s, bx, by);
            break;
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_fbm2d_batch(const FieldPlan* plans, const long long* tile_start, int n,
                               unsigned long long* counter, size_t smem, int blocks, cudaStream_t stream)
{
    cudaError_t e = cudaFuncSetAttribute(fbm2d_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fbm2d_batch_kernel<<<blocks, kThreads, smem, stream>>>(plans, tile_start, n, counter);
    return cudaGetLastError();
}

int fbm2d_batch_blocks_per_sm(size_t smem)
{
    int nb = 0;
    cudaFuncSetAttribute(fbm2d_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fbm2d_batch_kernel, kThreads, smem) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

size_t fbm2d_smem_bytes(const FieldPlan& P) { return sizeof(float4) * (size_t)(P.nst * 128 + P.ncorner); }

cudaError_t launch_fbm2d(const FieldPlan& P, int method, int s, cudaStream_t stream)
{
    const dim3 grid(P.tiles_x, P.tiles_y, 1);
    const size_t smem = fbm2d_smem_bytes(P);
    const bool f16 = P.dtype == 1;
#define PTG_LAUNCH2D(M, T)                                                                           \
    do {                                                                                             \
        auto kfn = fbm2d_kernel<M, T>;                                                               \
        cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                             (int)smem);                                             \
        if (e != cudaSuccess) return e;                                                              \
        kfn<<<grid, kThreads, smem, stream>>>(P, s);                                                 \
        return cudaGetLastError();                                                                   \
    } while (0)
    switch (method) {
    case kC1: if (f16) PTG_LAUNCH2D(kC1, __half); else PTG_LAUNCH2D(kC1, float);
    case kC2: if (f16) PTG_LAUNCH2D(kC2, __half); else PTG_LAUNCH2D(kC2, float);
    case kPerlinS5: if (f16) PTG_LAUNCH2D(kPerlinS5, __half); else PTG_LAUNCH2D(kPerlinS5, float);
    case kPerlinS3: if (f16) PTG_LAUNCH2D(kPerlinS3, __half); else PTG_LAUNCH2D(kPerlinS3, float);
    default: return cudaErrorInvalidValue;
    }
#undef PTG_LAUNCH2D
}

}  // namespace ptg
