// ptg_fbm3d.cu -- fused all-octave 3D generator (D3M1N3 / D3M2N5 cells of
// Thorimbert & Chopard, arXiv:1610.03525, Sec. 3.4; fractal sum of Sec. 4).
//
// One CTA makes a 32 x 16 x 8 tile (x, y, z) with 128 threads; each thread
// owns 8 consecutive x samples in 4 rows of one z plane (32 sums in
// registers).  Staged octaves keep the tile's corners (value and gradient,
// pre-scaled by the amplitude) and the per-axis bases in shared memory.  The
// cell is separable: for the thread's plane z it is first reduced along z,
//    W_ab = v_ab0 + S(z) (v_ab1 - v_ab0) + B0(z) e_ab0 + B1(z) e_ab1,
//    F_ab = f_ab0 + S(z) (f_ab1 - f_ab0),   G_ab = g_ab0 + S(z) (g_ab1 - g_ab0),
// which leaves exactly the 2D cell with (v, f, g) -> (W, F, G); that one is
// reduced per row to a 1D function of x and evaluated with 4 operations per
// sample.  Lattice octaves take one pcg4d corner value per sample.
#include "ptg_device.cuh"
#include "ptg_kernels.h"

namespace ptg {
namespace {

constexpr int kTW = kTile3dX, kTH = kTile3dY, kTD = kTile3dZ, kThreads = 128;
constexpr int kCols = 8, kRows = 4;

// float4 units: x-basis [nst][8 c][4 tx], y-basis [nst][4 r][4 ty],
// z-basis [nst][8 tz], corners.
__device__ __forceinline__ int xl(int i, int col) { return i * 32 + (col & 7) * 4 + (col >> 3); }
__device__ __forceinline__ int yl(int nst, int i, int row) { return nst * 32 + i * 16 + (row & 3) * 4 + (row >> 2); }
__device__ __forceinline__ int zl(int nst, int i, int pl) { return nst * 48 + i * 8 + pl; }

template <int METHOD>
__device__ __forceinline__ void stage_tile3(const FieldPlan& P, float4* sm, int j0x, int j0y, int j0z, int s)
{
    const int tid = threadIdx.x, nst = P.nst;
    for (int e = tid; e < nst * 56; e += kThreads) {
        const int i = e / 56, r = e - i * 56;
        if (r < 32) sm[xl(i, r)] = axis_basis<METHOD>(axis_t((uint32_t)(j0x + r), i, s));
        else if (r < 48) sm[yl(nst, i, r - 32)] = axis_basis<METHOD>(axis_t((uint32_t)(j0y + r - 32), i, s));
        else sm[zl(nst, i, r - 48)] = axis_basis<METHOD>(axis_t((uint32_t)(j0z + r - 48), i, s));
    }
    float4* corners = sm + nst * 56;
    for (int e = tid; e < P.ncorner; e += kThreads) {
        int i = 0;
        while (i + 1 < nst && e >= P.oct[i + 1].coff) ++i;
        const OctPlan& op = P.oct[i];
        const int local = e - op.coff;
        const int nxy = op.ncx * op.ncy;
        const int cz = local / nxy, rem = local - cz * nxy;
        const int cy = rem / op.ncx, cx = rem - cy * op.ncx;
        uint32_t x = op.ox + ((uint32_t)j0x >> op.k) + (uint32_t)cx;
        uint32_t y = op.oy + ((uint32_t)j0y >> op.k) + (uint32_t)cy;
        uint32_t z = op.oz + ((uint32_t)j0z >> op.k) + (uint32_t)cz;
        uint32_t w = op.key;
        pcg4d(x, y, z, w);
        corners[e] = make_float4(unit_value(x) * op.amp, unit_value(y) * op.ampw, unit_value(z) * op.ampw,
                                 unit_value(w) * op.ampw);
    }
}

template <int CW, int RH>
__device__ __forceinline__ void staged_octave3(float (&acc)[kRows][kCols], const float4* __restrict__ sm,
                                               const FieldPlan& P, int i, int tx, int ty, int tz)
{
    const OctPlan& op = P.oct[i];
    const int nst = P.nst, k = op.k, ncx = op.ncx, nxy = op.ncx * op.ncy;
    const float4* cg = sm + nst * 56 + op.coff;
    float4 xb[kCols];
#pragma unroll
    for (int c = 0; c < kCols; ++c) xb[c] = sm[xl(i, tx * 8 + c)];
    const float4 zb = sm[zl(nst, i, tz)];
    const int lcz = tz >> k;
#pragma unroll
    for (int yq = 0; yq < kRows / RH; ++yq) {
        const int lcy = (ty * kRows + yq * RH) >> k;
        float4 yb[RH];
#pragma unroll
        for (int r = 0; r < RH; ++r) yb[r] = sm[yl(nst, i, ty * kRows + yq * RH + r)];
#pragma unroll
        for (int xq = 0; xq < kCols / CW; ++xq) {
            const int lcx = (tx * kCols + xq * CW) >> k;
            const float4* c = cg + (lcz * op.ncy + lcy) * ncx + lcx;
            // z reduction of the four (a, b) corner columns
            float Wv[2][2], Fv[2][2], Gv[2][2];
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const float4 lo = c[b * ncx + a], hi = c[nxy + b * ncx + a];
                    Wv[a][b] = fmaf(zb.z, hi.w, fmaf(zb.y, lo.w, fmaf(zb.x, hi.x - lo.x, lo.x)));
                    Fv[a][b] = fmaf(zb.x, hi.y - lo.y, lo.y);
                    Gv[a][b] = fmaf(zb.x, hi.z - lo.z, lo.z);
                }
            const float dv0 = Wv[0][1] - Wv[0][0], dv1 = Wv[1][1] - Wv[1][0];
            const float df0 = Fv[0][1] - Fv[0][0], df1 = Fv[1][1] - Fv[1][0];
#pragma unroll
            for (int r = 0; r < RH; ++r) {
                const float Sy = yb[r].x, B0y = yb[r].y, B1y = yb[r].z;
                const float V0 = fmaf(B1y, Gv[0][1], fmaf(B0y, Gv[0][0], fmaf(Sy, dv0, Wv[0][0])));
                const float V1 = fmaf(B1y, Gv[1][1], fmaf(B0y, Gv[1][0], fmaf(Sy, dv1, Wv[1][0])));
                const float F0 = fmaf(Sy, df0, Fv[0][0]);
                const float F1 = fmaf(Sy, df1, Fv[1][0]);
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

__device__ __forceinline__ void lattice_octave3(float (&acc)[kRows][kCols], const OctPlan& op, uint32_t jx,
                                                uint32_t jy, uint32_t jz)
{
    const int sh = op.k;
    const uint32_t iz = op.oz + (jz << sh);
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const uint32_t iy = op.oy + ((jy + r) << sh);
#pragma unroll
        for (int c = 0; c < kCols; ++c) {
            const uint32_t ix = op.ox + ((jx + c) << sh);
            acc[r][c] = fmaf(op.amp, unit_value(pcg4d_value(ix, iy, iz, op.key)), acc[r][c]);
        }
    }
}

template <typename OutT>
__device__ __forceinline__ void store_tile3(const FieldPlan& P, const float (&acc)[kRows][kCols], int x0, int y0,
                                            int z)
{
    if (z >= P.D) return;
    OutT* out = reinterpret_cast<OutT*>(P.out) + (size_t)z * (size_t)P.H * (size_t)P.W;
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

template <int METHOD, typename OutT>
__global__ void __launch_bounds__(kThreads) fbm3d_kernel(const __grid_constant__ FieldPlan P, int s)
{
    extern __shared__ float4 sm[];
    const int tid = threadIdx.x, tx = tid & 3, ty = (tid >> 2) & 3, tz = tid >> 4;
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH, z0 = blockIdx.z * kTD;  // output tile
    const int j0x = x0 + P.jx0, j0y = y0 + P.jy0, j0z = z0 + P.jz0;                  // sample indices
    stage_tile3<METHOD>(P, sm, j0x, j0y, j0z, s);
    __syncthreads();
    float acc[kRows][kCols];
#pragma unroll
    for (int r = 0; r < kRows; ++r)
#pragma unroll
        for (int c = 0; c < kCols; ++c) acc[r][c] = 0.0f;
    for (int i = 0; i < P.N; ++i) {
        const int mode = P.oct[i].mode;
        if (mode == kModeRun8) staged_octave3<8, 4>(acc, sm, P, i, tx, ty, tz);
        else if (mode == kModeRun4) staged_octave3<4, 4>(acc, sm, P, i, tx, ty, tz);
        else if (mode == kModeRun2) staged_octave3<2, 2>(acc, sm, P, i, tx, ty, tz);
        else
            lattice_octave3(acc, P.oct[i], (uint32_t)(j0x + tx * kCols), (uint32_t)(j0y + ty * kRows),
                            (uint32_t)(j0z + tz));
    }
    store_tile3<OutT>(P, acc, x0 + tx * kCols, y0 + ty * kRows, z0 + tz);
}

}  // namespace

size_t fbm3d_smem_bytes(const FieldPlan& P) { return sizeof(float4) * (size_t)(P.nst * 56 + P.ncorner); }

cudaError_t launch_fbm3d(const FieldPlan& P, int method, int s, cudaStream_t stream)
{
    const dim3 grid(P.tiles_x, P.tiles_y, P.tiles_z);
    const size_t smem = fbm3d_smem_bytes(P);
    const bool f16 = P.dtype == 1;
#define PTG_LAUNCH3D(M, T)                                                                           \
    do {                                                                                             \
        auto kfn = fbm3d_kernel<M, T>;                                                               \
        cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                             (int)smem);                                             \
        if (e != cudaSuccess) return e;                                                              \
        kfn<<<grid, kThreads, smem, stream>>>(P, s);                                                 \
        return cudaGetLastError();                                                                   \
    } while (0)
    switch (method) {
    case kC1: if (f16) PTG_LAUNCH3D(kC1, __half); else PTG_LAUNCH3D(kC1, float);
    case kC2: if (f16) PTG_LAUNCH3D(kC2, __half); else PTG_LAUNCH3D(kC2, float);
    default: return cudaErrorInvalidValue;
    }
#undef PTG_LAUNCH3D
}

}  // namespace ptg
