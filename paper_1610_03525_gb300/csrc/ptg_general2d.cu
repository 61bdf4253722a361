// ptg_general2d.cu -- 2D polynomial-noise and Perlin fields with any
// frequency ratio f between octaves (Thorimbert & Chopard, arXiv:1610.03525,
// Sec. 4: amplitude p^i, frequency f^i).
//
// With f = 2 every octave's cells line up with the tiles and the fused
// generator (ptg_fbm2d.cu) evaluates rows of samples as polynomials of the
// column.  Any other f puts cell edges anywhere inside a tile, so here each
// sample finds its own cell and in-cell position at each octave and
// evaluates the cell polynomial there (Eq. polynomial with the corner data of
// Eq. mixedderiv; Perlin's polynomial of Sec. 3.2).
//
// Precision: the lattice coordinate of a tile's first sample is formed in
// FP64 (one thread per octave, into shared memory) and split into an integer
// cell (mod 2^32) and a fraction; a sample k samples further adds k * scale
// with scale = hi + lo in two floats and the exact product error of k * hi,
// so its position in the cell is good to about 2^-23 whatever the world
// offset.  A sample that lands within rounding of a cell edge may be placed
// in the neighbouring cell at t ~ 1 instead of t ~ 0; the fields are
// continuous across cell faces, so the value is the same to rounding.
#include "ptg_device.cuh"
#include "ptg_eval.cuh"
#include "ptg_kernels.h"

namespace ptg {
namespace {

constexpr int kTW = kTile2dX, kTH = kTile2dY, kThreads = 128;
constexpr int kCols = 8, kRows = 4;  // per thread: 8 consecutive columns in 4 rows

// The four corners of cell (cx, cy) hashed in place (octaves whose cells are
// too small to stage per tile).
template <int METHOD>
__device__ __forceinline__ Cell hashed_cell(uint32_t cx, uint32_t cy, uint32_t key, float amp, float ampw)
{
    Cell c;
    uint32_t x = cx, y = cy, z = key;
    pcg3d(x, y, z);
    c.c00 = corner_data<METHOD>(x, y, z, amp, ampw);
    x = cx + 1u, y = cy, z = key;
    pcg3d(x, y, z);
    c.c10 = corner_data<METHOD>(x, y, z, amp, ampw);
    x = cx, y = cy + 1u, z = key;
    pcg3d(x, y, z);
    c.c01 = corner_data<METHOD>(x, y, z, amp, ampw);
    x = cx + 1u, y = cy + 1u, z = key;
    pcg3d(x, y, z);
    c.c11 = corner_data<METHOD>(x, y, z, amp, ampw);
    return c;
}

// kRidged: each octave adds wgt_i r with r = (1 - |h|)^2 w, w the clamped
// doubled ridge of the octave before (1 at octave 0); otherwise the octave
// value (its amplitude already in the corner data).
template <bool kRidged>
__device__ __forceinline__ void add_octave(float& acc, float& wt, float h, float wgt)
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

template <int METHOD, bool kRidged>
__global__ void __launch_bounds__(kThreads) general2d_kernel(const __grid_constant__ GeneralPlan P)
{
    extern __shared__ float4 sm[];
    __shared__ uint32_t s_cx[kMaxOctaves], s_cy[kMaxOctaves];
    __shared__ float s_fx[kMaxOctaves], s_fy[kMaxOctaves];
    const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH;
    const int N = P.N;

    // the tile's base cell and fraction at every octave (FP64, one thread each)
    if (tid < N) {
        const double bx = fma((double)x0, P.scale[tid], P.base_x[tid]);
        const double by = fma((double)y0, P.scale[tid], P.base_y[tid]);
        const double fx = floor(bx), fy = floor(by);
        s_cx[tid] = (uint32_t)(unsigned long long)(long long)fx;
        s_cy[tid] = (uint32_t)(unsigned long long)(long long)fy;
        s_fx[tid] = (float)(bx - fx);
        s_fy[tid] = (float)(by - fy);
    }
    __syncthreads();

    // staged corner boxes: box_w x box_w corners from one cell before the
    // tile's base cell (a sample within rounding of the base cell's left edge
    // can land in the cell before it)
    for (int i = 0; i < N; ++i) {
        const int w = P.box_w[i];
        if (w == 0) continue;
        const uint32_t bx = s_cx[i] - 1u, by = s_cy[i] - 1u, key = P.key[i], magic = P.box_magic[i];
        const float amp = P.amp[i], ampw = P.ampw[i];
        float4* box = sm + P.box_off[i];
        for (int e = tid; e < w * w; e += kThreads) {
            const int cy = (int)__umulhi((uint32_t)e, magic);
            const int cx = e - cy * w;
            uint32_t x = bx + (uint32_t)cx, y = by + (uint32_t)cy, z = key;
            pcg3d(x, y, z);
            box[e] = corner_data<METHOD>(x, y, z, amp, ampw);
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
    const float kx0 = (float)(tx * kCols), ky0 = (float)(ty * kRows);
    for (int i = 0; i < N; ++i) {
        const float shi = P.scale_hi[i], slo = P.scale_lo[i];
        const int w = P.box_w[i];
        if ((P.lattice_mask >> i) & 1u) {
            // every sample sits on a lattice point (ridged fields with spc a power
            // of two): the octave is the corner value, one hash word a sample
            // (Perlin: zero)
            int nx[kCols];
#pragma unroll
            for (int c = 0; c < kCols; ++c) {
                float t;
                lattice_split(kx0 + (float)c, shi, slo, s_fx[i], nx[c], t);
            }
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                int ny;
                float t;
                lattice_split(ky0 + (float)r, shi, slo, s_fy[i], ny, t);
#pragma unroll
                for (int c = 0; c < kCols; ++c) {
                    float h = 0.0f;
                    if (METHOD != kPerlinS5 && METHOD != kPerlinS3) {
                        uint32_t x = s_cx[i] + (uint32_t)nx[c], y = s_cy[i] + (uint32_t)ny, z = P.key[i];
                        pcg3d(x, y, z);
                        h = corner_data<METHOD>(x, y, z, P.amp[i], P.ampw[i]).x;
                    }
                    add_octave<kRidged>(acc[r][c], wt[r][c], h, P.wgt[i]);
                }
            }
            continue;
        }
        const float4* box = sm + P.box_off[i];
        int nx[kCols];
        float4 xb[kCols];
#pragma unroll
        for (int c = 0; c < kCols; ++c) {
            float t;
            lattice_split(kx0 + (float)c, shi, slo, s_fx[i], nx[c], t);
            xb[c] = axis_basis<METHOD>(t);
        }
        if (w > 0 && nx[0] == nx[kCols - 1]) {
            // the thread's run lies in one cell: collapse each row once (per
            // thread, so warps diverge only where a run crosses a cell edge)
            const int lx = min(max(nx[0] + 1, 0), w - 2);
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                int ny;
                float t;
                lattice_split(ky0 + (float)r, shi, slo, s_fy[i], ny, t);
                const int ly = min(max(ny + 1, 0), w - 2);
                const float4* p = box + ly * w + lx;
                Cell cell;
                cell.c00 = p[0];
                cell.c10 = p[1];
                cell.c01 = p[w];
                cell.c11 = p[w + 1];
                const Row R = Model<METHOD>::row(cell, axis_basis<METHOD>(t));
#pragma unroll
                for (int c = 0; c < kCols; ++c)
                    add_octave<kRidged>(acc[r][c], wt[r][c], Model<METHOD>::eval(R, xb[c]), P.wgt[i]);
            }
            continue;
        }
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            int ny;
            float t;
            lattice_split(ky0 + (float)r, shi, slo, s_fy[i], ny, t);
            const float4 yb = axis_basis<METHOD>(t);
#pragma unroll
            for (int c = 0; c < kCols; ++c) {
                Cell cell;
                if (w > 0) {  // clamped into the box: a guard, the box covers every cell of the tile
                    const int lx = min(max(nx[c] + 1, 0), w - 2), ly = min(max(ny + 1, 0), w - 2);
                    const float4* p = box + ly * w + lx;
                    cell.c00 = p[0];
                    cell.c10 = p[1];
                    cell.c01 = p[w];
                    cell.c11 = p[w + 1];
                } else {
                    cell = hashed_cell<METHOD>(s_cx[i] + (uint32_t)nx[c], s_cy[i] + (uint32_t)ny, P.key[i], P.amp[i],
                                               P.ampw[i]);
                }
                add_octave<kRidged>(acc[r][c], wt[r][c], Model<METHOD>::eval(Model<METHOD>::row(cell, yb), xb[c]),
                                    P.wgt[i]);
            }
        }
    }

    // store
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const int y = y0 + ty * kRows + r, x = x0 + tx * kCols;
        if (y >= P.H) break;
        if (P.dtype == 1) {
            __half* row = reinterpret_cast<__half*>(P.out) + (size_t)y * (size_t)P.W;
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
            float* row = reinterpret_cast<float*>(P.out) + (size_t)y * (size_t)P.W;
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

cudaError_t launch_general2d(const GeneralPlan& P, cudaStream_t stream)
{
    const dim3 grid(P.tiles_x, P.tiles_y, 1);
    const size_t smem = sizeof(float4) * (size_t)P.box_words;
#define PTG_LAUNCHG(M)                                                                               \
    do {                                                                                             \
        auto kfn = P.ridged ? general2d_kernel<M, true> : general2d_kernel<M, false>;                \
        cudaError_t e = set_kernel_smem((const void*)kfn, smem);                                     \
        if (e != cudaSuccess) return e;                                                              \
        kfn<<<grid, kThreads, smem, stream>>>(P);                                                    \
        return cudaGetLastError();                                                                   \
    } while (0)
    switch (P.method) {
    case kC1: PTG_LAUNCHG(kC1);
    case kC2: PTG_LAUNCHG(kC2);
    case kPaperGauge: PTG_LAUNCHG(kPaperGauge);
    case kZeroGrad: PTG_LAUNCHG(kZeroGrad);
    case kPerlinS5: PTG_LAUNCHG(kPerlinS5);
    case kPerlinS3: PTG_LAUNCHG(kPerlinS3);
    default: return cudaErrorInvalidValue;
    }
#undef PTG_LAUNCHG
}

}  // namespace ptg
