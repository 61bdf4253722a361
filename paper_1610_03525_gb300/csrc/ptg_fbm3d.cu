// ptg_fbm3d.cu -- fused all-octave 3D generator (D3M1N3 / D3M2N5 cells of
// Thorimbert & Chopard, arXiv:1610.03525, Sec. 3.4; fractal sum of Sec. 4),
// and Perlin's polynomial (Sec. 3.2) in 3D as a baseline.
//
// One CTA makes a 32 x 16 x 8 tile (x, y, z) with 128 threads; each thread
// owns 8 consecutive x samples in 4 rows of one z plane (32 sums in
// registers).  The cell is separable: for the thread's plane it is first
// reduced along z,
//    W_ab = v_ab0 + S(z) (v_ab1 - v_ab0) + B0(z) e_ab0 + B1(z) e_ab1,
//    F_ab = f_ab0 + S(z) (f_ab1 - f_ab0),   G_ab = g_ab0 + S(z) (g_ab1 - g_ab0),
// which leaves the 2D cell with (v, f, g) -> (W, F, G), handled as in 2D.
// Perlin has v = 0 and its own B0 = (1 - S) t, B1 = S (t - 1), so the same
// reduction gives W_ab = B0(z) e_ab0 + B1(z) e_ab1 (the z part of the corner
// dot products) and the 2D Perlin cell with those values:
// octaves whose cells are >= 8 samples wide evaluate node columns only and
// interpolate once; cells of 4 and 2 samples use constant in-cell positions
// along x and y; lattice octaves take one pcg4d corner value per sample.
//
// Tile octaves (C1): an octave whose cells are 32 samples or more covers the
// whole tile with one cell (tiles start at multiples of min(spc, tile)), so
// over the tile it is one polynomial of degree 3 per axis, and so is the sum
// of all such octaves.  With two or more of them the CTA evaluates that sum
// at 4 x 4 x 4 tile nodes ({0, 9, 22, 31} x {0, 4, 11, 15} x {0, 2, 5, 7},
// Lebesgue constants 1.42, 1.55, 1.4) and every thread interpolates it to its
// rows and node columns (exact for the tricubic up to rounding).
#include "ptg_device.cuh"
#include "ptg_eval.cuh"
#include "ptg_kernels.h"

namespace ptg {
namespace {

constexpr int kTW = kTile3dX, kTH = kTile3dY, kTD = kTile3dZ, kThreads = 128;
constexpr int kCols = 8, kRows = 4;

// Shared memory (float4 units): x-basis at node columns [n8][D+1][4 tx],
// y-basis [n8][4 r][4 ty], z-basis [n8][8 tz], staged corners (planes of
// ncy swizzled rows).
template <int METHOD>
__host__ __device__ constexpr int xnode_words3(int n8) { return n8 * (Deg<METHOD>::value + 1) * 4; }

template <int METHOD>
__host__ __device__ constexpr int corner_base3(int n8) { return xnode_words3<METHOD>(n8) + n8 * 24; }

__device__ __forceinline__ int n_run8(const FieldPlan& P)
{
    const int n = P.s - 2;
    return n < 0 ? 0 : (n < P.N ? n : P.N);
}

// Tile octaves (cells >= 32 samples, octaves 0 .. s - 5), used for C1 when
// there are at least two of them; else 0.
template <int METHOD>
__host__ __device__ __forceinline__ int n_tile3(const FieldPlan& P)
{
    if (METHOD != kC1) return 0;
    int n = P.s - 4;
    n = n < 0 ? 0 : (n < P.N ? n : P.N);
    return n >= 2 ? n : 0;
}

// Tile node position q along axis a (x, y, z), packed one byte each.
__host__ __device__ constexpr int node3(int a, int q)
{
    return (int)(((a == 0 ? 0x1F160900u : (a == 1 ? 0x0F0B0400u : 0x07050200u)) >> (8 * q)) & 0xffu);
}

// Lagrange weight of node q at integer position p along axis a.
__host__ __device__ constexpr float lagrange3(int a, int p, int q)
{
    long long num = 1, den = 1;
    for (int m = 0; m < 4; ++m) {
        if (m == q) continue;
        num *= (long long)(p - node3(a, m));
        den *= (long long)(node3(a, q) - node3(a, m));
    }
    return (float)((double)num / (double)den);
}

// Interpolation weights of the tile nodes: along z for each plane, along y
// for each row, along x for each thread's node columns (x = 8 tx + node_col).
struct alignas(16) Tile3Weights {
    float wz[kTD][4];
    float wy[kTH][4];
    float wx[4][4][4];  // [tx][node column q][tile node a]
};

constexpr Tile3Weights make_tile3_weights()
{
    Tile3Weights W{};
    for (int p = 0; p < kTD; ++p)
        for (int q = 0; q < 4; ++q) W.wz[p][q] = lagrange3(2, p, q);
    for (int p = 0; p < kTH; ++p)
        for (int q = 0; q < 4; ++q) W.wy[p][q] = lagrange3(1, p, q);
    for (int t = 0; t < 4; ++t)
        for (int c = 0; c < 4; ++c)
            for (int q = 0; q < 4; ++q) W.wx[t][c][q] = lagrange3(0, 8 * t + node_col<3>(c), q);
    return W;
}

__device__ const Tile3Weights kTile3Weights = make_tile3_weights();

template <int METHOD>
__device__ __forceinline__ void stage_tile3(const FieldPlan& P, float4* sm, int j0x, int j0y, int j0z)
{
    constexpr int NN = Deg<METHOD>::value + 1;
    const int tid = threadIdx.x, s = P.s, n8 = n_run8(P), nt = n_tile3<METHOD>(P);
    float4* xnode = sm;
    float4* ylut = sm + xnode_words3<METHOD>(n8);
    float4* zlut = ylut + n8 * 16;
    float4* corners = sm + corner_base3<METHOD>(n8);
    for (int e = tid + nt * NN * 4; e < n8 * NN * 4; e += kThreads) {  // no tables for the tile octaves
        const int i = e / (NN * 4), rem = e - i * (NN * 4);
        const int q = rem >> 2, tx = rem & 3;
        sst(kSiteStage, &xnode[e], axis_basis<METHOD>(axis_t((uint32_t)(j0x + tx * 8 + node_col<Deg<METHOD>::value>(q)), i, s)));
    }
    for (int e = tid + nt * 24; e < n8 * 24; e += kThreads) {
        const int i = e / 24, slot = e - i * 24;
        if (slot < 16) {  // y: slot = r * 4 + ty, row 4 ty + r
            const int row = (slot & 3) * 4 + (slot >> 2);
            sst(kSiteStage, &ylut[i * 16 + slot], axis_basis<METHOD>(axis_t((uint32_t)(j0y + row), i, s)));
        } else {
            sst(kSiteStage, &zlut[i * 8 + slot - 16], axis_basis<METHOD>(axis_t((uint32_t)(j0z + slot - 16), i, s)));
        }
    }
    // Corners, octave by octave (uniform loops); octaves with at most 32
    // corners go to one warp each, in turn (see the 2D generator).
    const int warp = tid >> 5, lane = tid & 31;
    int small = 0;
    for (int i = 0; i < P.nst; ++i) {
        const OctPlan& op = P.oct[i];
        const int nxy = op.ncx * op.ncy, n = nxy * op.ncz;
        int e0 = tid, step = kThreads;
        if (n <= 32) {
            if ((small++ & 3) != warp) continue;
            e0 = lane;
            step = 32;
        }
        const uint32_t bx = op.ox + ((uint32_t)j0x >> op.k), by = op.oy + ((uint32_t)j0y >> op.k);
        const uint32_t bz = op.oz + ((uint32_t)j0z >> op.k);
        float4* cg = corners + op.coff;
        const float m3a = -3.0f * op.amp, m3w = -3.0f * op.ampw;
        for (int e = e0; e < n; e += step) {
            const int cz = (int)__umulhi((uint32_t)e, op.magic2);
            const int rem = e - cz * nxy;
            const int cy = (int)__umulhi((uint32_t)rem, op.magic);
            const int cx = rem - cy * op.ncx;
            uint32_t x = bx + (uint32_t)cx, y = by + (uint32_t)cy, z = bz + (uint32_t)cz, w = op.key;
            pcg4d(x, y, z, w);
            const int slot = (cz * op.ncy + cy) * op.rowlen + corner_slot(cx);
            if (bounds_ok(kSiteStage, slot, op.rowlen * op.ncy * op.ncz))
                sst(kSiteStage, &cg[slot],
                    (METHOD == kPerlinS5 || METHOD == kPerlinS3)  // Perlin: no value, gradient unweighted
                        ? make_float4(0.0f, unit_scaled(y, op.amp, m3a), unit_scaled(z, op.amp, m3a),
                                      unit_scaled(w, op.amp, m3a))
                        : make_float4(unit_scaled(x, op.amp, m3a), unit_scaled(y, op.ampw, m3w),
                                      unit_scaled(z, op.ampw, m3w), unit_scaled(w, op.ampw, m3w)));
        }
    }
}

// The 2D cell (W, F, G per corner) of the thread's plane: reduction along z
// of the 8 corners of cell (lcx, lcy, lcz) with z-basis zb.
__device__ __forceinline__ Cell zcell(const float4* __restrict__ cg, const OctPlan& op, int lcx, int lcy, int lcz,
                                      float4 zb)
{
    const int plane = op.ncy * op.rowlen;
    const float4* p0 = cg + (lcz * op.ncy + lcy) * op.rowlen;
    const int s0 = corner_slot(lcx), s1 = corner_slot(lcx + 1);
    float4 r[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {  // q = a + 2 b
        const float4* p = p0 + (q >> 1) * op.rowlen + ((q & 1) ? s1 : s0);
        const int at = (int)(p - cg), n = plane * op.ncz;  // slots of the octave's block (debug build)
        const float4 lo = bounds_ok(kSiteCorner, at, n) ? sld(kSiteCorner, &p[0]) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 hi = bounds_ok(kSiteCorner, at + plane, n) ? sld(kSiteCorner, &p[plane]) : make_float4(0.f, 0.f, 0.f, 0.f);
        r[q] = zreduce(lo, hi, zb);
    }
    Cell c;
    c.c00 = r[0];
    c.c10 = r[1];
    c.c01 = r[2];
    c.c11 = r[3];
    return c;
}

// The tile octaves' sum at the 64 tile nodes, into G[(z * 4 + y) * 4 + x]:
// two lanes a node, each taking every other octave, added by one shuffle.
template <int METHOD>
__device__ __forceinline__ void tile_grid3(const FieldPlan& P, const float4* __restrict__ corners, float* G, int j0x,
                                           int j0y, int j0z, int nt)
{
    const int tid = threadIdx.x, node = tid >> 1, part = tid & 1;
    const uint32_t jx = (uint32_t)(j0x + node3(0, node & 3)), jy = (uint32_t)(j0y + node3(1, (node >> 2) & 3));
    const uint32_t jz = (uint32_t)(j0z + node3(2, node >> 4));
    float v = 0.0f;
    for (int i = part; i < nt; i += 2) {
        const OctPlan& op = P.oct[i];
        const float4 xb = axis_basis<METHOD>(axis_t(jx, i, P.s)), yb = axis_basis<METHOD>(axis_t(jy, i, P.s));
        const float4 zb = axis_basis<METHOD>(axis_t(jz, i, P.s));
        const Cell c = zcell(corners + op.coff, op, 0, 0, 0, zb);  // the tile's one cell of this octave
        const Row R = row_of(c, yb.x, yb.y, yb.z);
        v += eval_row(R, xb.x, xb.y, xb.z);
    }
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    if (part == 0) sst(kSiteTable, &G[node], v);
}

// Interpolate the tile nodes to the thread's plane, rows and node columns.
__device__ __forceinline__ void add_tile_grid3(float (&nacc)[kRows][4], const float* __restrict__ G, int tx, int ty,
                                               int tz)
{
    const Tile3Weights& W = kTile3Weights;
    const float4 wz = bounds_ok(kSiteConst, tz, 8) ? __ldg(reinterpret_cast<const float4*>(W.wz[tz]))
                                                   : make_float4(0.f, 0.f, 0.f, 0.f);
    float hz[4][4];  // [y node][x node] in the thread's plane
    const float4* G4 = reinterpret_cast<const float4*>(G);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const float4 g0 = sld(kSiteTable, &G4[b]), g1 = sld(kSiteTable, &G4[4 + b]);
        const float4 g2 = sld(kSiteTable, &G4[8 + b]), g3 = sld(kSiteTable, &G4[12 + b]);
        hz[b][0] = fmaf(wz.w, g3.x, fmaf(wz.z, g2.x, fmaf(wz.y, g1.x, wz.x * g0.x)));
        hz[b][1] = fmaf(wz.w, g3.y, fmaf(wz.z, g2.y, fmaf(wz.y, g1.y, wz.x * g0.y)));
        hz[b][2] = fmaf(wz.w, g3.z, fmaf(wz.z, g2.z, fmaf(wz.y, g1.z, wz.x * g0.z)));
        hz[b][3] = fmaf(wz.w, g3.w, fmaf(wz.z, g2.w, fmaf(wz.y, g1.w, wz.x * g0.w)));
    }
    float4 wx[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
        wx[q] = bounds_ok(kSiteConst, tx, 4) ? __ldg(reinterpret_cast<const float4*>(W.wx[tx][q]))
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const float4 wy = bounds_ok(kSiteConst, ty * kRows + r, 16)
                              ? __ldg(reinterpret_cast<const float4*>(W.wy[ty * kRows + r]))
                              : make_float4(0.f, 0.f, 0.f, 0.f);
        float hy[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) hy[a] = fmaf(wy.w, hz[3][a], fmaf(wy.z, hz[2][a], fmaf(wy.y, hz[1][a], wy.x * hz[0][a])));
#pragma unroll
        for (int q = 0; q < 4; ++q)
            nacc[r][q] = fmaf(wx[q].w, hy[3], fmaf(wx[q].z, hy[2], fmaf(wx[q].y, hy[1], fmaf(wx[q].x, hy[0], nacc[r][q]))));
    }
}

template <int METHOD>
__device__ __forceinline__ void run8_octave3(float (&nacc)[kRows][Deg<METHOD>::value + 1],
                                             const float4* __restrict__ sm, const FieldPlan& P, int i, int tx,
                                             int ty, int tz, int n8)
{
    constexpr int NN = Deg<METHOD>::value + 1;
    const OctPlan& op = P.oct[i];
    const float4* ylut = sm + xnode_words3<METHOD>(n8);
    const float4* zlut = ylut + n8 * 16;
    const float4* cg = sm + corner_base3<METHOD>(n8) + op.coff;
    const Cell c = zcell(cg, op, (tx * kCols) >> op.k, (ty * kRows) >> op.k, tz >> op.k,
                         sld(kSiteTable, &zlut[i * 8 + tz]));
    float4 xb[NN];
#pragma unroll
    for (int q = 0; q < NN; ++q) xb[q] = sld(kSiteTable, &sm[(i * NN + q) * 4 + tx]);
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const float4 yb = sld(kSiteTable, &ylut[i * 16 + r * 4 + ty]);
        const Row R = row_of(c, yb.x, yb.y, yb.z);
#pragma unroll
        for (int q = 0; q < NN; ++q) nacc[r][q] += eval_row(R, xb[q].x, xb[q].y, xb[q].z);
    }
}

// Cells of CW = 4 or 2 samples: in-cell positions along x and y are constants;
// along z the thread's plane has position (tz mod CW) / CW.
template <int METHOD, int CW>
__device__ __forceinline__ void small_octave3(float (&acc)[kRows][kCols], const float4* __restrict__ sm,
                                              const FieldPlan& P, int i, int tx, int ty, int tz, int n8)
{
    const OctPlan& op = P.oct[i];
    const float4* cg = sm + corner_base3<METHOD>(n8) + op.coff;
    constexpr float inv = 1.0f / CW;
    const float4 zb = axis_basis<METHOD>((float)(tz & (CW - 1)) * inv);
    const int lcz = tz / CW;
#pragma unroll
    for (int yq = 0; yq < kRows / CW; ++yq) {
        const int lcy = (ty * kRows + yq * CW) / CW;
#pragma unroll
        for (int xq = 0; xq < kCols / CW; ++xq) {
            const Cell c = zcell(cg, op, (tx * kCols + xq * CW) / CW, lcy, lcz, zb);
#pragma unroll
            for (int rr = 0; rr < CW; ++rr) {
                Row R;
                if (rr == 0) {
                    R = row_at_zero(c);
                } else {
                    const float4 yb = axis_basis<METHOD>(rr * inv);
                    R = row_of(c, yb.x, yb.y, yb.z);
                }
#pragma unroll
                for (int q = 0; q < CW; ++q) {
                    float h;
                    if (q == 0) {
                        h = R.V0;
                    } else {
                        const float4 xb = axis_basis<METHOD>(q * inv);
                        h = eval_row(R, xb.x, xb.y, xb.z);
                    }
                    acc[yq * CW + rr][xq * CW + q] += h;
                }
            }
        }
    }
}

// Adds amp unit_mant(h); the -3 amp terms of all lattice octaves are added
// once, at the store (FieldPlan::lat_bias).
__device__ __forceinline__ void lattice_octave3(float (&acc)[kRows][kCols], const OctPlan& op, uint32_t jx,
                                                uint32_t jy, uint32_t jz)
{
    const int sh = op.k;
    const uint32_t z1 = pcg_lcg(op.oz + (jz << sh)), w1 = pcg_lcg(op.key);
    const uint32_t dx = 1664525u << sh, x0 = op.ox + (jx << sh);  // x's LCG step advances by dx a column
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const uint32_t y1 = pcg_lcg(op.oy + ((jy + r) << sh));
        const uint32_t base = pcg4d_run_base(x0, y1, w1);
#pragma unroll
        for (int c = 0; c < kCols; ++c) {
            const uint32_t h = pcg4d_run_value(base + (uint32_t)c * dx, y1, z1, w1);
            acc[r][c] = fmaf(op.amp, unit_mant(h), acc[r][c]);
        }
    }
}

// Elements [x, x + n) of row y of plane z lie inside the output (checked in
// the debug build only).
__device__ __forceinline__ bool out_ok3(const FieldPlan& P, int x, int y, int z, int n)
{
    return bounds_ok(kSiteStore, x + n - 1, P.W) && bounds_ok(kSiteStore, y, P.H) && bounds_ok(kSiteStore, z, P.D);
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
            if (!out_ok3(P, x0, y, z, kCols)) continue;
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
                if (x0 + c < P.W && out_ok3(P, x0 + c, y, z, 1)) store1(row + x0 + c, acc[r][c]);
        }
    }
}

template <int METHOD, typename OutT>
__global__ void __launch_bounds__(kThreads) fbm3d_kernel(const __grid_constant__ FieldPlan P)
{
    constexpr int D = Deg<METHOD>::value, NN = D + 1;
    extern __shared__ float4 sm[];
    const int tid = threadIdx.x, tx = tid & 3, ty = (tid >> 2) & 3, tz = tid >> 4;
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH, z0 = blockIdx.z * kTD;  // output tile
    const int j0x = x0 + P.jx0, j0y = y0 + P.jy0, j0z = z0 + P.jz0;                  // sample indices
    const int s = P.s, N = P.N, n8 = n_run8(P), nt = n_tile3<METHOD>(P);
    stage_tile3<METHOD>(P, sm, j0x, j0y, j0z);
    __syncthreads();

    // tile octaves: their sum at the tile nodes (read back after the barrier below)
    float* G = reinterpret_cast<float*>(sm + corner_base3<METHOD>(n8) + P.ncorner);
    if (nt > 0) tile_grid3<METHOD>(P, sm + corner_base3<METHOD>(n8), G, j0x, j0y, j0z, nt);

    float nacc[kRows][NN];
#pragma unroll
    for (int r = 0; r < kRows; ++r)
#pragma unroll
        for (int q = 0; q < NN; ++q) nacc[r][q] = 0.0f;
    for (int i = nt; i < n8; ++i) run8_octave3<METHOD>(nacc, sm, P, i, tx, ty, tz, n8);
    if constexpr (NN == 4) {
        if (nt > 0) {  // uniform over the CTA
            __syncthreads();
            add_tile_grid3(nacc, G, tx, ty, tz);
        }
    }
    float acc[kRows][kCols];
#pragma unroll
    for (int r = 0; r < kRows; ++r)
#pragma unroll
        for (int c = 0; c < kCols; ++c) {
            const int q = node_of_col<D>(c);
            if (q >= 0) {
                acc[r][c] = nacc[r][q];
            } else {
                float v = 0.0f;
#pragma unroll
                for (int m = 0; m < NN; ++m) v = fmaf(lagrange<D>(c, m), nacc[r][m], v);
                acc[r][c] = v;
            }
        }
    if (s >= 2 && s - 2 < N) small_octave3<METHOD, 4>(acc, sm, P, s - 2, tx, ty, tz, n8);
    if (s >= 1 && s - 1 < N) small_octave3<METHOD, 2>(acc, sm, P, s - 1, tx, ty, tz, n8);
    if (METHOD != kPerlinS5 && METHOD != kPerlinS3 && s < N) {  // Perlin is zero at lattice points
        const uint32_t jx = (uint32_t)(j0x + tx * kCols), jy = (uint32_t)(j0y + ty * kRows), jz = (uint32_t)(j0z + tz);
        for (int i = s; i < N; ++i) lattice_octave3(acc, P.oct[i], jx, jy, jz);
#pragma unroll
        for (int r = 0; r < kRows; ++r)
#pragma unroll
            for (int c = 0; c < kCols; ++c) acc[r][c] += P.lat_bias;
    }
    store_tile3<OutT>(P, acc, x0 + tx * kCols, y0 + ty * kRows, z0 + tz);
}

template <int METHOD>
size_t smem_words3(const FieldPlan& P)
{
    int n8 = P.s - 2;
    n8 = n8 < 0 ? 0 : (n8 < P.N ? n8 : P.N);
    return (size_t)corner_base3<METHOD>(n8) + (size_t)P.ncorner + (n_tile3<METHOD>(P) > 0 ? 16 : 0);
}

}  // namespace

size_t fbm3d_smem_bytes(const FieldPlan& P)
{
    size_t w = 0;
    switch (P.method) {
    case kC2: w = smem_words3<kC2>(P); break;
    case kPerlinS5: w = smem_words3<kPerlinS5>(P); break;
    case kPerlinS3: w = smem_words3<kPerlinS3>(P); break;
    default: w = smem_words3<kC1>(P); break;
    }
    return sizeof(float4) * w;
}

cudaError_t launch_fbm3d(const FieldPlan& P, int method, int /*s*/, cudaStream_t stream)
{
    const dim3 grid(P.tiles_x, P.tiles_y, P.tiles_z);
    const size_t smem = fbm3d_smem_bytes(P);
    const bool f16 = P.dtype == 1;
#define PTG_LAUNCH3D(M, T)                                                                           \
    do {                                                                                             \
        auto kfn = fbm3d_kernel<M, T>;                                                               \
        cudaError_t e = set_kernel_smem((const void*)kfn, smem);                                     \
        if (e != cudaSuccess) return e;                                                              \
        kfn<<<grid, kThreads, smem, stream>>>(P);                                                    \
        return cudaGetLastError();                                                                   \
    } while (0)
    switch (method) {
    case kC1: if (f16) PTG_LAUNCH3D(kC1, __half); else PTG_LAUNCH3D(kC1, float);
    case kC2: if (f16) PTG_LAUNCH3D(kC2, __half); else PTG_LAUNCH3D(kC2, float);
    case kPerlinS5: if (f16) PTG_LAUNCH3D(kPerlinS5, __half); else PTG_LAUNCH3D(kPerlinS5, float);
    case kPerlinS3: if (f16) PTG_LAUNCH3D(kPerlinS3, __half); else PTG_LAUNCH3D(kPerlinS3, float);
    default: return cudaErrorInvalidValue;
    }
#undef PTG_LAUNCH3D
}

}  // namespace ptg
