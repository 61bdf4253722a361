// ptg_eval.cuh -- cell evaluation shared by the 2D and 3D generators.
//
// Inside a cell every method is separable.  For one row y (and, in 3D, after
// the reduction along z) the cell collapses to a 1D function of x,
//     h(x) = V0 + S(x) (V1 - V0) + B0(x) F0 + B1(x) F1,
//     V_a = v_a0 + S(y) (v_a1 - v_a0) + B0(y) g_a0 + B1(y) g_a1,
//     F_a = f_a0 + S(y) (f_a1 - f_a0),
// the tensor-product Hermite cell of Eq. (polynomial) with the corner
// constraints of Eq. (mixedderiv) (Thorimbert & Chopard, arXiv:1610.03525,
// Sec. 2-3) or Perlin's polynomial of Sec. 3.2 (v = 0, its own B0, B1).
// Along a run of columns inside one cell, h is a polynomial of degree d in the
// column index, evaluated at d + 1 node columns and interpolated elsewhere.
#pragma once

#include "ptg_device.cuh"

namespace ptg {

// Degree along x of one cell row, per method.
template <int METHOD>
struct Deg {
    static constexpr int value = (METHOD == kC1 || METHOD == kPaperGauge || METHOD == kZeroGrad) ? 3
                               : METHOD == kC2 ? 5 : METHOD == kPerlinS3 ? 4 : 6;
};

// Node columns of a run of RW columns (8 or 16) for degree D: d + 1 of the
// run's columns, chosen so that the interpolation weights of the other columns
// are small (max sum |w| over a column: RW = 8: 1.4, 2.1, 2.3, 2.7 for
// D = 3, 4, 5, 6; RW = 16: 1.55, 1.66, 1.95, 2.22).
template <int D, int RW = 8>
__host__ __device__ constexpr int node_col(int q)
{
    return RW == 8
        ? (D == 3 ? (q == 0 ? 0 : q == 1 ? 2 : q == 2 ? 5 : 7)
         : D == 4 ? (q == 0 ? 0 : q == 1 ? 1 : q == 2 ? 3 : q == 3 ? 6 : 7)
         : D == 5 ? (q == 0 ? 0 : q == 1 ? 1 : q == 2 ? 2 : q == 3 ? 4 : q == 4 ? 6 : 7)
                  : (q < 4 ? q : q + 1))
        : (D == 3 ? (q == 0 ? 0 : q == 1 ? 4 : q == 2 ? 11 : 15)
         : D == 4 ? (q == 0 ? 0 : q == 1 ? 3 : q == 2 ? 7 : q == 3 ? 12 : 15)
         : D == 5 ? (q == 0 ? 0 : q == 1 ? 2 : q == 2 ? 6 : q == 3 ? 9 : q == 4 ? 13 : 15)
                  : (q == 0 ? 0 : q == 1 ? 1 : q == 2 ? 4 : q == 3 ? 7 : q == 4 ? 11 : q == 5 ? 14 : 15));
}

template <int D, int RW = 8>
__host__ __device__ constexpr int node_of_col(int c)  // node index of column c, or -1
{
    int r = -1;
    for (int q = 0; q <= D; ++q)
        if (node_col<D, RW>(q) == c) r = q;
    return r;
}

// Lagrange weight of node q at column c: prod_{m != q} (c - x_m) / (x_q - x_m),
// a ratio of small integers (folded to a constant once loops are unrolled).
template <int D, int RW = 8>
__host__ __device__ constexpr float lagrange(int c, int q)
{
    long long num = 1, den = 1;
    for (int m = 0; m <= D; ++m) {
        if (m == q) continue;
        num *= (long long)(c - node_col<D, RW>(m));
        den *= (long long)(node_col<D, RW>(q) - node_col<D, RW>(m));
    }
    return (float)num / (float)den;
}

// Tile nodes: d + 1 positions along a 64-sample tile side at which the sum of
// the octaves whose cells cover the whole tile is sampled; that sum is one
// polynomial of degree d per axis over the tile, so its values there fix it.
// Chosen by search for a small Lebesgue constant over the 64 positions: 1.45,
// 1.59, 1.71, 1.89 for d = 3, 4, 5, 6.
template <int D>
__host__ __device__ constexpr int tile_node(int q)
{
    return D == 3 ? (q == 0 ? 0 : q == 1 ? 18 : q == 2 ? 45 : 63)
         : D == 4 ? (q == 0 ? 0 : q == 1 ? 11 : q == 2 ? 31 : q == 3 ? 51 : 63)
         : D == 5 ? (q == 0 ? 0 : q == 1 ? 8 : q == 2 ? 23 : q == 3 ? 40 : q == 4 ? 55 : 63)
                  : (q == 0 ? 0 : q == 1 ? 6 : q == 2 ? 17 : q == 3 ? 32 : q == 4 ? 45 : q == 5 ? 57 : 63);
}

template <int D>
__host__ __device__ constexpr float tile_lagrange(int c, int q)
{
    long long num = 1, den = 1;
    for (int m = 0; m <= D; ++m) {
        if (m == q) continue;
        num *= (long long)(c - tile_node<D>(m));
        den *= (long long)(tile_node<D>(q) - tile_node<D>(m));
    }
    return (float)num / (float)den;
}

// Weights that carry the tile nodes' values to a thread: ly[y] = weights of
// the d + 1 tile rows at tile row y; lx[q'][tx] = weights of the d + 1 tile
// columns at the q'-th node column of the run of thread column tx.  Rows are
// padded to a multiple of 4 floats for vector loads; lx is node-column major,
// so the 8 thread columns of a load phase read consecutive 16-byte words
// (distinct banks).
template <int D, int RW>
struct alignas(16) TileWeights {
    static constexpr int NN = D + 1, LW = (NN + 3) & ~3, TXN = 64 / RW;
    float ly[64][LW];
    float lx[NN][TXN][LW];
};

template <int D, int RW>
constexpr TileWeights<D, RW> make_tile_weights()
{
    TileWeights<D, RW> w{};
    for (int y = 0; y < 64; ++y)
        for (int q = 0; q <= D; ++q) w.ly[y][q] = tile_lagrange<D>(y, q);
    for (int tx = 0; tx < 64 / RW; ++tx)
        for (int n = 0; n <= D; ++n)
            for (int q = 0; q <= D; ++q) w.lx[n][tx][q] = tile_lagrange<D>(tx * RW + node_col<D, RW>(n), q);
    return w;
}

// Corner data of one staged corner from its hash words, pre-scaled by the
// octave amplitude (and the gradient weight w of Sec. 4): (v, f, g, 0) for
// the Hermite cells and the paper's D2M1N3, (v, 0, 0, 0) for the
// zero-gradient model, (0, f, g, 0) for Perlin.
template <int METHOD>
__device__ __forceinline__ float4 corner_data(uint32_t hx, uint32_t hy, uint32_t hz, float amp, float ampw)
{
    const float m3a = -3.0f * amp, m3w = -3.0f * ampw;  // per octave: hoisted out of the staging loops
    if (METHOD == kZeroGrad) return make_float4(unit_scaled(hx, amp, m3a), 0.0f, 0.0f, 0.0f);
    if (METHOD == kC1 || METHOD == kC2 || METHOD == kPaperGauge)
        return make_float4(unit_scaled(hx, amp, m3a), unit_scaled(hy, ampw, m3w), unit_scaled(hz, ampw, m3w), 0.0f);
    return make_float4(0.0f, unit_scaled(hy, amp, m3a), unit_scaled(hz, amp, m3a), 0.0f);
}

// Per-axis basis of an in-cell position t as compile-time values, computed in
// double and rounded once: the functions of axis_basis.
struct alignas(16) Basis4 {
    float x, y, z, w;
};

template <int METHOD>
constexpr Basis4 basis_const(double t)
{
    const double t2 = t * t, u = t - 1.0;
    const double S3 = t2 * (3.0 - 2.0 * t), S5 = t2 * t * (10.0 + t * (-15.0 + 6.0 * t));
    if (METHOD == kZeroGrad) return Basis4{(float)S3, (float)t, 0.0f, 0.0f};
    if (METHOD == kPaperGauge) return Basis4{(float)t, 0.0f, 0.0f, 0.0f};
    if (METHOD == kC1) return Basis4{(float)S3, (float)(t * u * u), (float)(t2 * u), 0.0f};
    if (METHOD == kC2)
        return Basis4{(float)S5, (float)(t * u * u * (-u) * (1.0 + 3.0 * t)), (float)(t2 * t * u * (4.0 - 3.0 * t)),
                      0.0f};
    const double S = METHOD == kPerlinS5 ? S5 : S3;
    return Basis4{(float)S, (float)((1.0 - S) * t), (float)(S * u), 0.0f};
}

// Run octaves with cells of 2^K samples, RW <= 2^K <= 64.  Tiles start at
// multiples of min(64, spc) samples, so tile column c lies at (c mod 2^K) / 2^K
// of its cell in every tile: the basis at a thread's node columns and rows
// is one table for all tiles, with 2^K / RW distinct thread columns and 2^K
// distinct rows per K.  Flat: x at xoff(K) + q (2^K / RW) + (tx mod 2^K / RW),
// y at yoff(K) + (row mod 2^K).
template <int METHOD, int RW>
struct RunBasis {
    static constexpr int NN = Deg<METHOD>::value + 1, LOG = RW == 8 ? 3 : 4;
    static constexpr int NX = NN * ((64 / RW) * 2 - 1), NY = 64 * 2 - (1 << LOG);  // sums over K = LOG .. 6
    __host__ __device__ static constexpr int xoff(int K) { return NN * ((1 << (K - LOG)) - 1); }
    __host__ __device__ static constexpr int yoff(int K) { return (1 << K) - (1 << LOG); }
    Basis4 x[NX];
    Basis4 y[NY];
};

template <int METHOD, int RW>
constexpr RunBasis<METHOD, RW> make_run_basis()
{
    using B = RunBasis<METHOD, RW>;
    B b{};
    for (int K = B::LOG; K <= 6; ++K) {
        const int m = (1 << K) - 1, nx = (1 << K) / RW;
        for (int q = 0; q < B::NN; ++q)
            for (int tx = 0; tx < nx; ++tx)
                b.x[B::xoff(K) + q * nx + tx] = basis_const<METHOD>((double)(tx * RW + node_col<B::NN - 1, RW>(q)) / (m + 1));
        for (int row = 0; row <= m; ++row) b.y[B::yoff(K) + row] = basis_const<METHOD>((double)row / (m + 1));
    }
    return b;
}

// Corner data of one cell: (v, f, g) at (0,0), (1,0), (0,1), (1,1).
struct Cell {
    float4 c00, c10, c01, c11;
};

// Row collapse of a cell at y-basis (Sy, B0y, B1y): V0, V1 - V0, F0, F1.
struct Row {
    float V0, dV, F0, F1;
};

__device__ __forceinline__ Row row_of(const Cell& c, float Sy, float B0y, float B1y)
{
    const float dv0 = c.c01.x - c.c00.x, dv1 = c.c11.x - c.c10.x;
    const float df0 = c.c01.y - c.c00.y, df1 = c.c11.y - c.c10.y;
    Row r;
    r.V0 = fmaf(B1y, c.c01.z, fmaf(B0y, c.c00.z, fmaf(Sy, dv0, c.c00.x)));
    const float V1 = fmaf(B1y, c.c11.z, fmaf(B0y, c.c10.z, fmaf(Sy, dv1, c.c10.x)));
    r.F0 = fmaf(Sy, df0, c.c00.y);
    r.F1 = fmaf(Sy, df1, c.c10.y);
    r.dV = V1 - r.V0;
    return r;
}

// Row collapse at t_y = 0 (the cell's own corner row).
__device__ __forceinline__ Row row_at_zero(const Cell& c)
{
    Row r;
    r.V0 = c.c00.x;
    r.dV = c.c10.x - c.c00.x;
    r.F0 = c.c00.y;
    r.F1 = c.c10.y;
    return r;
}

__device__ __forceinline__ float eval_row(const Row& r, float Sx, float B0x, float B1x)
{
    return fmaf(B1x, r.F1, fmaf(B0x, r.F0, fmaf(Sx, r.dV, r.V0)));
}


// 3D cells: reduction along z of a corner pair (lo at z = 0, hi at z = 1;
// each (v, f, g, e) with e the z gradient) at z-basis zb: the 2D corner
// (W, F, G) of the thread's plane,
//   W = v0 + S(z) (v1 - v0) + B0(z) e0 + B1(z) e1,  F = f0 + S(z) (f1 - f0),
//   G = g0 + S(z) (g1 - g0).
__device__ __forceinline__ float4 zreduce(float4 lo, float4 hi, float4 zb)
{
    return make_float4(fmaf(zb.z, hi.w, fmaf(zb.y, lo.w, fmaf(zb.x, hi.x - lo.x, lo.x))),
                       fmaf(zb.x, hi.y - lo.y, lo.y), fmaf(zb.x, hi.z - lo.z, lo.z), 0.0f);
}

// Per-method cell model: the row collapse at a y-basis entry, the row at
// t_y = 0, and the evaluation of a collapsed row at an x-basis entry.
// eval_add(r, xb, a): the same evaluation with the row's V0 term replaced by
// a, i.e. eval(r, xb) - V0 + a (a caller that sums V0 separately, once per
// row, adds each node's other terms to its own accumulator).
template <int METHOD>
struct Model {  // tensor-product Hermite cells (C1, C2) and Perlin
    __device__ static __forceinline__ Row row(const Cell& c, float4 yb) { return row_of(c, yb.x, yb.y, yb.z); }
    __device__ static __forceinline__ Row row0(const Cell& c) { return row_at_zero(c); }
    __device__ static __forceinline__ float eval(const Row& r, float4 xb) { return eval_row(r, xb.x, xb.y, xb.z); }
    __device__ static __forceinline__ float eval_add(const Row& r, float4 xb, float a)
    {
        return fmaf(xb.z, r.F1, fmaf(xb.y, r.F0, fmaf(xb.x, r.dV, a)));
    }
};

// Zero-gradient D2M1N3 (Eq. zg with -xy): for a row at height y,
//   h(x) = [h00 + S3(y) dy] + S3(x) [dx + A y] + x [A (S3(y) - y)],
// dx = h10 - h00, dy = h01 - h00, A = h11 + h00 - h10 - h01.
// Row fields: V0, dV, F0 = the x coefficient; basis entries (S3, t).
template <>
struct Model<kZeroGrad> {
    __device__ static __forceinline__ Row row(const Cell& c, float4 yb)
    {
        const float dx = c.c10.x - c.c00.x, dy = c.c01.x - c.c00.x;
        const float A = (c.c11.x - c.c01.x) - dx;
        Row r;
        r.V0 = fmaf(yb.x, dy, c.c00.x);
        r.dV = fmaf(A, yb.y, dx);
        r.F0 = A * (yb.x - yb.y);
        r.F1 = 0.0f;
        return r;
    }
    __device__ static __forceinline__ Row row0(const Cell& c)
    {
        Row r;
        r.V0 = c.c00.x;
        r.dV = c.c10.x - c.c00.x;
        r.F0 = 0.0f;
        r.F1 = 0.0f;
        return r;
    }
    __device__ static __forceinline__ float eval(const Row& r, float4 xb) { return fmaf(xb.y, r.F0, fmaf(xb.x, r.dV, r.V0)); }
    __device__ static __forceinline__ float eval_add(const Row& r, float4 xb, float a)
    {
        return fmaf(xb.y, r.F0, fmaf(xb.x, r.dV, a));
    }
};

// The D2M1N3 polynomial with the coefficients printed in Sec. 3.1
// (c22 = c33 = c32 = c23 = 0; c_ji from c_ij by swapping indices and f <-> g).
// For a row at height y it is the cubic a0 + a1 x + a2 x^2 + a3 x^3 with
// a_i = sum_j c_ij y^j.  Row fields: V0..F1 = a0..a3; basis entries (t).
template <>
struct Model<kPaperGauge> {
    struct Coef {
        float c00, c10, c01, c20, c30, c02, c03, c21, c31, c12, c13, c11;
    };
    __device__ static __forceinline__ Coef coef(const Cell& c)
    {
        const float h00 = c.c00.x, h10 = c.c10.x, h01 = c.c01.x, h11 = c.c11.x;
        const float f00 = c.c00.y, f10 = c.c10.y, f01 = c.c01.y, f11 = c.c11.y;
        const float g00 = c.c00.z, g10 = c.c10.z, g01 = c.c01.z, g11 = c.c11.z;
        Coef k;
        k.c00 = h00;
        k.c10 = f00;
        k.c01 = g00;
        const float dx0 = h10 - h00, dy0 = h01 - h00, dx1 = h11 - h01, dy1 = h11 - h10;
        k.c20 = fmaf(3.0f, dx0, -fmaf(2.0f, f00, f10));
        k.c30 = fmaf(-2.0f, dx0, f10 + f00);
        k.c02 = fmaf(3.0f, dy0, -fmaf(2.0f, g00, g01));
        k.c03 = fmaf(-2.0f, dy0, g01 + g00);
        k.c21 = fmaf(3.0f, dx1, -fmaf(2.0f, f01, f11)) - k.c20;
        k.c31 = fmaf(-2.0f, dx1, f11 + f01) - k.c30;
        k.c12 = fmaf(3.0f, dy1, -fmaf(2.0f, g10, g11)) - k.c02;
        k.c13 = fmaf(-2.0f, dy1, g11 + g10) - k.c03;
        k.c11 = ((h01 + h10) - (h00 + h11)) + ((f01 - f00) + (g10 - g00));
        return k;
    }
    __device__ static __forceinline__ Row row(const Cell& c, float4 yb)
    {
        const Coef k = coef(c);
        const float y = yb.x;
        Row r;
        r.V0 = fmaf(y, fmaf(y, fmaf(y, k.c03, k.c02), k.c01), k.c00);
        r.dV = fmaf(y, fmaf(y, fmaf(y, k.c13, k.c12), k.c11), k.c10);
        r.F0 = fmaf(y, k.c21, k.c20);
        r.F1 = fmaf(y, k.c31, k.c30);
        return r;
    }
    __device__ static __forceinline__ Row row0(const Cell& c)
    {
        const Coef k = coef(c);
        Row r;
        r.V0 = k.c00;
        r.dV = k.c10;
        r.F0 = k.c20;
        r.F1 = k.c30;
        return r;
    }
    __device__ static __forceinline__ float eval(const Row& r, float4 xb)
    {
        const float t = xb.x;
        return fmaf(t, fmaf(t, fmaf(t, r.F1, r.F0), r.dV), r.V0);
    }
    __device__ static __forceinline__ float eval_add(const Row& r, float4 xb, float a)
    {
        const float t = xb.x;
        return fmaf(t, fmaf(t, fmaf(t, r.F1, r.F0), r.dV), a);
    }
};

}  // namespace ptg
