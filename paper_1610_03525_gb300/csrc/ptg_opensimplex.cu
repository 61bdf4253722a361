// ptg_opensimplex.cu -- OpenSimplex-style 2D gradient noise, the simplex-lattice
// comparison point of Thorimbert & Chopard (arXiv:1610.03525, Sec. 1, 5.1,
// 5.2), with the same fractal sum (Sec. 4) as the polynomial generators.
//
// Lattice: integer points (a, b) of a "stretched" plane, mapped to real space
// by the squish (a + (a+b) q, b + (a+b) q), q = (sqrt(3) - 1)/2, which makes
// equilateral triangles of edge sqrt(2).  A point's stretched coordinates are
// x + (x+y) r, y + (x+y) r with r = (1/sqrt(3) - 1)/2.  Each vertex within
// distance sqrt(2) adds (2 - |d|^2)^4 (g . d); g = hash words 1, 2.
//
// Vertex choice: the point lies in one triangle of its stretched unit square
// (lower if xi + yi < 1).  Besides the triangle's three vertices, at most one
// more vertex is in range: the one across the triangle edge nearest to the
// point, i.e. opposite the vertex with the smallest barycentric weight.  Four
// vertices per sample and octave; the exclusion of out-of-range ones is
// branch-free (max(0, 2 - r^2)).
//
// Precision: the octave-i position of the CTA tile's first sample is formed in
// FP64 once per octave and split into an integer vertex and a fraction.  A
// sample's offset (cs, rs) from it is exact in FP32 (multiples of 2^i / spc);
// its stretched coordinates add K r with K = cs + rs, where the product with the
// irrational r is taken in two pieces, r = r_hi + r_lo, with the rounding error
// of K r_hi recovered by an FMA, and integer parts are removed before any
// fractions are summed, so the in-cell position keeps full FP32 accuracy at
// every octave.
#include <cstdint>

#include "ptg_device.cuh"
#include "ptg_kernels.h"

namespace ptg {
namespace {

constexpr int kTW = 64, kTH = 64, kThreads = 128, kCols = 8, kRows = 4;
constexpr float kSquish = 0.36602540378443865f;   // (sqrt(3) - 1) / 2
constexpr double kStretchD = -0.21132486540518713; // (1/sqrt(3) - 1) / 2
constexpr float kStretchHi = (float)kStretchD;
constexpr float kStretchLo = (float)(kStretchD - (double)kStretchHi);
constexpr float kScale = 0.125f;

struct TileOctave {
    int32_t a0, b0;  // integer stretched vertex of the tile's first sample
    float fx, fy;    // its fractional stretched coordinates
};

__device__ __forceinline__ float vertex_term(int32_t a, int32_t b, uint32_t key, float dx, float dy)
{
    uint32_t x = (uint32_t)a, y = (uint32_t)b, z = key;
    pcg3d(x, y, z);
    const float gx = unit_value(y), gy = unit_value(z);
    const float k = fmaxf(0.0f, 2.0f - fmaf(dx, dx, dy * dy));
    const float k2 = k * k;
    return (k2 * k2) * fmaf(gx, dx, gy * dy);
}

// Contribution of vertex (a + da, b + db) at stretched fraction (xi, yi).
__device__ __forceinline__ float vertex_at(int32_t a, int32_t b, int da, int db, uint32_t key, float xi, float yi)
{
    const float u = xi - (float)da, v = yi - (float)db;
    const float s = (u + v) * kSquish;
    return vertex_term(a + da, b + db, key, u + s, v + s);
}

template <typename OutT>
__global__ void __launch_bounds__(kThreads) opensimplex2d_kernel(const __grid_constant__ SimplexPlan P)
{
    __shared__ TileOctave tile[kMaxOctaves];
    const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
    const int j0x = blockIdx.x * kTW, j0y = blockIdx.y * kTH;
    if (tid < P.N) {
        const int i = tid;
        const double X = P.base_x[i] + (double)j0x * (double)P.step[i];
        const double Y = P.base_y[i] + (double)j0y * (double)P.step[i];
        const double sh = (X + Y) * kStretchD;
        const double xs = X + sh, ys = Y + sh;
        const double fa = floor(xs), fb = floor(ys);
        tile[i].a0 = (int32_t)(long long)fa;
        tile[i].b0 = (int32_t)(long long)fb;
        tile[i].fx = (float)(xs - fa);
        tile[i].fy = (float)(ys - fb);
    }
    __syncthreads();
    float acc[kRows][kCols];
#pragma unroll
    for (int r = 0; r < kRows; ++r)
#pragma unroll
        for (int c = 0; c < kCols; ++c) acc[r][c] = 0.0f;

    for (int i = 0; i < P.N; ++i) {
        const TileOctave T = tile[i];
        const float step = P.step[i], amp = P.amp[i] * kScale;
        const uint32_t key = P.key[i];
        float cs[kCols], fxc[kCols];
        int32_t icx[kCols];
#pragma unroll
        for (int c = 0; c < kCols; ++c) {
            cs[c] = (float)(tx * kCols + c) * step;  // exact
            const float fl = floorf(cs[c]);
            icx[c] = (int32_t)fl;
            fxc[c] = T.fx + (cs[c] - fl);
        }
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const float rs = (float)(ty * kRows + r) * step;  // exact
            const float fl = floorf(rs);
            const int32_t iry = (int32_t)fl;
            const float fyr = T.fy + (rs - fl);
#pragma unroll
            for (int c = 0; c < kCols; ++c) {
                const float K = cs[c] + rs;                      // exact
                const float p = K * kStretchHi;
                const float e = fmaf(K, kStretchHi, -p);         // exact rounding error of p
                const float ip = floorf(p);
                const float t = (p - ip) + (e + K * kStretchLo);
                const float sx = fxc[c] + t, sy = fyr + t;
                const float flx = floorf(sx), fly = floorf(sy);
                const float xi = sx - flx, yi = sy - fly;
                const int32_t iip = (int32_t)ip;
                const int32_t a = T.a0 + icx[c] + iip + (int32_t)flx;
                const int32_t b = T.b0 + iry + iip + (int32_t)fly;
                float h;
                if (xi + yi < 1.0f) {
                    h = vertex_at(a, b, 0, 0, key, xi, yi) + vertex_at(a, b, 1, 0, key, xi, yi) +
                        vertex_at(a, b, 0, 1, key, xi, yi);
                    const float w00 = 1.0f - xi - yi;
                    int da, db;
                    if (w00 <= xi && w00 <= yi) { da = 1; db = 1; }
                    else if (xi <= yi) { da = -1; db = 1; }
                    else { da = 1; db = -1; }
                    h += vertex_at(a, b, da, db, key, xi, yi);
                } else {
                    h = vertex_at(a, b, 1, 1, key, xi, yi) + vertex_at(a, b, 1, 0, key, xi, yi) +
                        vertex_at(a, b, 0, 1, key, xi, yi);
                    const float w11 = xi + yi - 1.0f, w10 = 1.0f - yi, w01 = 1.0f - xi;
                    int da, db;
                    if (w11 <= w10 && w11 <= w01) { da = 0; db = 0; }
                    else if (w10 <= w01) { da = 0; db = 2; }
                    else { da = 2; db = 0; }
                    h += vertex_at(a, b, da, db, key, xi, yi);
                }
                acc[r][c] = fmaf(amp, h, acc[r][c]);
            }
        }
    }
    OutT* out = reinterpret_cast<OutT*>(P.out);
    const int x0 = j0x + tx * kCols, y0 = j0y + ty * kRows;
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
                __half2 hh[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) hh[q] = __floats2half2_rn(acc[r][2 * q], acc[r][2 * q + 1]);
                *reinterpret_cast<uint4*>(row + x0) = *reinterpret_cast<const uint4*>(hh);
            }
        } else {
#pragma unroll
            for (int c = 0; c < kCols; ++c)
                if (x0 + c < P.W) store1(row + x0 + c, acc[r][c]);
        }
    }
}

}  // namespace

cudaError_t launch_opensimplex2d(const SimplexPlan& P, cudaStream_t stream)
{
    const dim3 grid(P.tiles_x, P.tiles_y, 1);
    if (P.dtype == 1) opensimplex2d_kernel<__half><<<grid, kThreads, 0, stream>>>(P);
    else opensimplex2d_kernel<float><<<grid, kThreads, 0, stream>>>(P);
    return cudaGetLastError();
}

}  // namespace ptg
