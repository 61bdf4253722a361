// ptg_general3d.cu -- 3D polynomial-noise (C1, C2) and Perlin fields with any
// spc or frequency ratio f between octaves (Thorimbert & Chopard,
// arXiv:1610.03525, Sec. 3.4 and Sec. 4: frequency f^i).
//
// The 2D per-sample generator (ptg_general2d.cu) with a third axis: every
// sample finds its cell and in-cell position at each octave (FP64 tile base,
// two-float offsets), reduces the cell along z at its plane (the fused 3D
// generator's reduction), collapses the row and evaluates it.
#include "ptg_device.cuh"
#include "ptg_eval.cuh"
#include "ptg_kernels.h"

namespace ptg {
namespace {

constexpr int kTW = kTile3dX, kTH = kTile3dY, kTD = kTile3dZ, kThreads = 128;
constexpr int kCols = 8, kRows = 4;  // per thread: 8 consecutive columns in 4 rows of one plane

template <int METHOD>
__device__ __forceinline__ float4 corner3(uint32_t cx, uint32_t cy, uint32_t cz, uint32_t key, float amp, float ampw)
{
    uint32_t x = cx, y = cy, z = cz, w = key;
    pcg4d(x, y, z, w);
    const float m3a = -3.0f * amp, m3w = -3.0f * ampw;
    if (METHOD == kPerlinS5 || METHOD == kPerlinS3)  // Perlin: no value, gradient unweighted
        return make_float4(0.0f, unit_scaled(y, amp, m3a), unit_scaled(z, amp, m3a), unit_scaled(w, amp, m3a));
    return make_float4(unit_scaled(x, amp, m3a), unit_scaled(y, ampw, m3w), unit_scaled(z, ampw, m3w),
                       unit_scaled(w, ampw, m3w));
}

// Adds one octave's value h to a sample's sum: plain, or (kRidged) the ridge
// (1 - |h|)^2 w weighted by wgt, w then the clamped doubled ridge.
template <bool kRidged>
__device__ __forceinline__ void add_octave3(float& acc, float& wt, float h, float wgt)
{
    if (kRidged) {
        const float a = 1.0f - fabsf(h);
        const float ridge = a * a * wt;
        acc = fmaf(wgt, ridge, acc);
        wt = __saturatef(2.0f * ridge);
    } else {
        acc += h;
    }
}

// kRidged: ridged noise, as in the 2D per-sample generator.
template <int METHOD, bool kRidged>
__global__ void __launch_bounds__(kThreads) general3d_kernel(const __grid_constant__ General3Plan P)
{
    extern __shared__ float4 sm[];
    __shared__ uint32_t s_c[3][kMaxOctaves];
    __shared__ float s_f[3][kMaxOctaves];
    const int tid = threadIdx.x, tx = tid & 3, ty = (tid >> 2) & 3, tz = tid >> 4;
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH, z0 = blockIdx.z * kTD;
    const int N = P.N;

    // the tile's base cell and fraction at every octave (FP64, one thread per octave and axis)
    if (tid < 3 * N) {
        const int a = tid / N, i = tid - a * N;
        const int o = a == 0 ? x0 : (a == 1 ? y0 : z0);
        const double b = fma((double)o, P.scale[i], P.base[a][i]);
        const double fl = floor(b);
        s_c[a][i] = (uint32_t)(unsigned long long)(long long)fl;
        s_f[a][i] = (float)(b - fl);
    }
    __syncthreads();

    // staged corner boxes from one cell before the tile's base cell on each axis
    for (int i = 0; i < N; ++i) {
        const int wx = P.box_w[0][i];
        if (wx == 0) continue;
        const int wy = P.box_w[1][i], wz = P.box_w[2][i], wxy = wx * wy;
        const uint32_t bx = s_c[0][i] - 1u, by = s_c[1][i] - 1u, bz = s_c[2][i] - 1u, key = P.key[i];
        const uint32_t mx = P.box_magic[0][i], mxy = P.box_magic[1][i];
        const float amp = P.amp[i], ampw = P.ampw[i];
        float4* box = sm + P.box_off[i];
        for (int e = tid; e < wxy * wz; e += kThreads) {
            const int cz = (int)__umulhi((uint32_t)e, mxy);
            const int rem = e - cz * wxy;
            const int cy = (int)__umulhi((uint32_t)rem, mx);
            const int cx = rem - cy * wx;
            box[e] = corner3<METHOD>(bx + (uint32_t)cx, by + (uint32_t)cy, bz + (uint32_t)cz, key, amp, ampw);
        }
    }
    __syncthreads();

    float acc[kRows][kCols], wt[kRows][kCols];
#pragma unroll
    for (int r = 0; r < kRows; ++r)
#pragma unroll
        for (int c = 0; c < kCols; ++c) {
            acc[r][c] = 0.0f;
            wt[r][c] = 1.0f;
        }
    const float kx0 = (float)(tx * kCols), ky0 = (float)(ty * kRows), kz = (float)tz;
    for (int i = 0; i < N; ++i) {
        const float shi = P.scale_hi[i], slo = P.scale_lo[i];
        const int wx = P.box_w[0][i], wy = P.box_w[1][i], wz = P.box_w[2][i];
        if ((P.lattice_mask >> i) & 1u) {
            // every sample sits on a lattice point: the corner value (Perlin: zero)
            int nx[kCols], nz;
            float t;
            lattice_split(kz, shi, slo, s_f[2][i], nz, t);
#pragma unroll
            for (int c = 0; c < kCols; ++c) lattice_split(kx0 + (float)c, shi, slo, s_f[0][i], nx[c], t);
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                int ny;
                lattice_split(ky0 + (float)r, shi, slo, s_f[1][i], ny, t);
#pragma unroll
                for (int c = 0; c < kCols; ++c) {
                    float h = 0.0f;
                    if (METHOD != kPerlinS5 && METHOD != kPerlinS3)
                        h = corner3<METHOD>(s_c[0][i] + (uint32_t)nx[c], s_c[1][i] + (uint32_t)ny,
                                            s_c[2][i] + (uint32_t)nz, P.key[i], P.amp[i], P.ampw[i]).x;
                    add_octave3<kRidged>(acc[r][c], wt[r][c], h, P.wgt[i]);
                }
            }
            continue;
        }
        const float4* box = sm + P.box_off[i];
        int nx[kCols], nz;
        float4 xb[kCols], zb;
        {
            float t;
            lattice_split(kz, shi, slo, s_f[2][i], nz, t);
            zb = axis_basis<METHOD>(t);
        }
#pragma unroll
        for (int c = 0; c < kCols; ++c) {
            float t;
            lattice_split(kx0 + (float)c, shi, slo, s_f[0][i], nx[c], t);
            xb[c] = axis_basis<METHOD>(t);
        }
        if (wx > 0 && nx[0] == nx[kCols - 1]) {
            // the thread's run lies in one cell: reduce it along z and collapse
            // each row once (per thread: warps diverge only at cell edges)
            const int lx = min(max(nx[0] + 1, 0), wx - 2), lz = min(max(nz + 1, 0), wz - 2);
            const int plane = wx * wy;
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                int ny;
                float t;
                lattice_split(ky0 + (float)r, shi, slo, s_f[1][i], ny, t);
                const float4 yb = axis_basis<METHOD>(t);
                const int ly = min(max(ny + 1, 0), wy - 2);
                const float4* p = box + (lz * wy + ly) * wx + lx;
                Cell cell;
                cell.c00 = zreduce(p[0], p[plane], zb);
                cell.c10 = zreduce(p[1], p[plane + 1], zb);
                cell.c01 = zreduce(p[wx], p[plane + wx], zb);
                cell.c11 = zreduce(p[wx + 1], p[plane + wx + 1], zb);
                const Row R = row_of(cell, yb.x, yb.y, yb.z);
#pragma unroll
                for (int c = 0; c < kCols; ++c)
                    add_octave3<kRidged>(acc[r][c], wt[r][c], eval_row(R, xb[c].x, xb[c].y, xb[c].z), P.wgt[i]);
            }
            continue;
        }
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            int ny;
            float t;
            lattice_split(ky0 + (float)r, shi, slo, s_f[1][i], ny, t);
            const float4 yb = axis_basis<METHOD>(t);
#pragma unroll
            for (int c = 0; c < kCols; ++c) {
                float4 lo[4], hi[4];  // corners (a, b) = (0,0), (1,0), (0,1), (1,1) at z = 0 and 1
                if (wx > 0) {         // clamped into the box: a guard, the box covers every cell of the tile
                    const int lx = min(max(nx[c] + 1, 0), wx - 2), ly = min(max(ny + 1, 0), wy - 2);
                    const int lz = min(max(nz + 1, 0), wz - 2);
                    const float4* p = box + (lz * wy + ly) * wx + lx;
                    const int plane = wx * wy;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4* pq = p + (q >> 1) * wx + (q & 1);
                        lo[q] = pq[0];
                        hi[q] = pq[plane];
                    }
                } else {
                    const uint32_t cx = s_c[0][i] + (uint32_t)nx[c], cy = s_c[1][i] + (uint32_t)ny;
                    const uint32_t cz = s_c[2][i] + (uint32_t)nz;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        lo[q] = corner3<METHOD>(cx + (q & 1), cy + (q >> 1), cz, P.key[i], P.amp[i], P.ampw[i]);
                        hi[q] = corner3<METHOD>(cx + (q & 1), cy + (q >> 1), cz + 1u, P.key[i], P.amp[i], P.ampw[i]);
                    }
                }
                Cell cell;
                cell.c00 = zreduce(lo[0], hi[0], zb);
                cell.c10 = zreduce(lo[1], hi[1], zb);
                cell.c01 = zreduce(lo[2], hi[2], zb);
                cell.c11 = zreduce(lo[3], hi[3], zb);
                const Row R = row_of(cell, yb.x, yb.y, yb.z);
                add_octave3<kRidged>(acc[r][c], wt[r][c], eval_row(R, xb[c].x, xb[c].y, xb[c].z), P.wgt[i]);
            }
        }
    }

    // store
    const int z = z0 + tz;
    if (z >= P.D) return;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const int y = y0 + ty * kRows + r, x = x0 + tx * kCols;
        if (y >= P.H) break;
        const size_t rowoff = ((size_t)z * (size_t)P.H + (size_t)y) * (size_t)P.W;
        if (P.dtype == 1) {
            __half* row = reinterpret_cast<__half*>(P.out) + rowoff;
            if (P.vec_ok && x + kCols <= P.W) {
                __half2 h[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) h[q] = __floats2half2_rn(acc[r][2 * q], acc[r][2 * q + 1]);
                *reinterpret_cast<uint4*>(row + x) = *reinterpret_cast<const uint4*>(h);
            } else {
#pragma unroll
                for (int c = 0; c < kCols; ++c)
                    if (x + c < P.W) store1(row + x + c, acc[r][c]);
            }
        } else {
            float* row = reinterpret_cast<float*>(P.out) + rowoff;
            if (P.vec_ok && x + kCols <= P.W) {
                float4* p = reinterpret_cast<float4*>(row + x);
                p[0] = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
                p[1] = make_float4(acc[r][4], acc[r][5], acc[r][6], acc[r][7]);
            } else {
#pragma unroll
                for (int c = 0; c < kCols; ++c)
                    if (x + c < P.W) store1(row + x + c, acc[r][c]);
            }
        }
    }
}

}  // namespace

cudaError_t launch_general3d(const General3Plan& P, cudaStream_t stream)
{
    const dim3 grid(P.tiles_x, P.tiles_y, P.tiles_z);
    const size_t smem = sizeof(float4) * (size_t)P.box_words;
#define PTG_LAUNCHG3(M)                                                                              \
    do {                                                                                             \
        auto kfn = P.ridged ? general3d_kernel<M, true> : general3d_kernel<M, false>;                \
        cudaError_t e = set_kernel_smem((const void*)kfn, smem);                                     \
        if (e != cudaSuccess) return e;                                                              \
        kfn<<<grid, kThreads, smem, stream>>>(P);                                                    \
        return cudaGetLastError();                                                                   \
    } while (0)
    switch (P.method) {
    case kC1: PTG_LAUNCHG3(kC1);
    case kC2: PTG_LAUNCHG3(kC2);
    case kPerlinS5: PTG_LAUNCHG3(kPerlinS5);
    case kPerlinS3: PTG_LAUNCHG3(kPerlinS3);
    default: return cudaErrorInvalidValue;
    }
#undef PTG_LAUNCHG3
}

}  // namespace ptg
