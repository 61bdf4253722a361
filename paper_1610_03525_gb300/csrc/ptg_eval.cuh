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
    static constexpr int value = METHOD == kC1 ? 3 : METHOD == kC2 ? 5 : METHOD == kPerlinS3 ? 4 : 6;
};

// Node columns of the run8 evaluation for degree D (d + 1 of the 8 columns,
// chosen so that the interpolation weights of the other columns are small:
// sum |w| <= 1.4, 2.1, 2.3, 2.7 for D = 3, 4, 5, 6).
template <int D>
__host__ __device__ constexpr int node_col(int q)
{
    return D == 3 ? (q == 0 ? 0 : q == 1 ? 2 : q == 2 ? 5 : 7)
         : D == 4 ? (q == 0 ? 0 : q == 1 ? 1 : q == 2 ? 3 : q == 3 ? 6 : 7)
         : D == 5 ? (q == 0 ? 0 : q == 1 ? 1 : q == 2 ? 2 : q == 3 ? 4 : q == 4 ? 6 : 7)
                  : (q < 4 ? q : q + 1);
}

template <int D>
__host__ __device__ constexpr int node_of_col(int c)  // node index of column c, or -1
{
    int r = -1;
    for (int q = 0; q <= D; ++q)
        if (node_col<D>(q) == c) r = q;
    return r;
}

// Lagrange weight of node q at column c: prod_{m != q} (c - x_m) / (x_q - x_m),
// a ratio of small integers (folded to a constant once loops are unrolled).
template <int D>
__host__ __device__ constexpr float lagrange(int c, int q)
{
    long long num = 1, den = 1;
    for (int m = 0; m <= D; ++m) {
        if (m == q) continue;
        num *= (long long)(c - node_col<D>(m));
        den *= (long long)(node_col<D>(q) - node_col<D>(m));
    }
    return (float)num / (float)den;
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


}  // namespace ptg
