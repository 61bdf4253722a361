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
// Node rows (C1): the run and tile octaves' sum over the 8 rows of a thread
// pair (ty = 2b, 2b + 1; lanes l and l ^ 4) lies in one cell of the finest
// run octave, so, as in 2D, the pair evaluates rows 0, 2 and 7, 5 of its
// block only (the odd thread mirrored) and interpolates the other four.
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

// Rows a thread evaluates (node rows for degree 3) and the thread's row of
// its k-th evaluated row (par = ty & 1).
template <int METHOD>
__host__ __device__ constexpr bool node_rows3() { return Deg<METHOD>::value == 3; }
template <int METHOD>
__host__ __device__ constexpr int n_rows3() { return node_rows3<METHOD>() ? 2 : kRows; }
template <int METHOD>
__device__ __forceinline__ int eval_row3(int k, int par)
{
    return node_rows3<METHOD>() ? (k == 0 ? 3 * par : 2 - par) : k;
}

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
// there are at least four of them; else 0.  With node rows a run octave
// costs a thread about what its share of the tile-node sum does, and the
// sum's code (a kernel of its own, so that fields without it carry none of
// it) adds a barrier.  By measurement on GB300 (512^3, FP16, back-to-back
// launches), against the kernel without that code: 12% faster with six such
// octaves and 4% with four, 1.8% slower with three and 3% with two.
template <int METHOD>
__host__ __device__ __forceinline__ int n_tile3(const FieldPlan& P)
{
    if (METHOD != kC1) return 0;
    int n = P.s - 4;
    n = n < 0 ? 0 : (n < P.N ? n : P.N);
    return n >= 4 ? n : 0;
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

// Corner grid of a 32 x 16 x 8 tile at cells of 2^K samples: corners along
// x, y, z and float4 slots per swizzled corner row.
__host__ __device__ constexpr int ncx3(int K) { return (kTW - 1 >> K) + 2; }
__host__ __device__ constexpr int ncy3(int K) { return (kTH - 1 >> K) + 2; }
__host__ __device__ constexpr int ncz3(int K) { return (kTD - 1 >> K) + 2; }
__host__ __device__ constexpr int rowlen3(int K) { return corner_rowlen3(ncx3(K)); }
static_assert(rowlen3(1) == 19 && rowlen3(2) == 11 && rowlen3(3) == 5 && rowlen3(4) == 3 && rowlen3(5) == 2, "");

// Corner data from the four pcg4d words, pre-scaled by the octave amplitude
// (and the gradient weight): (v, f, g, e); Perlin: (0, f, g, e), unweighted.
template <int METHOD>
__device__ __forceinline__ float4 corner_data4(uint32_t x, uint32_t y, uint32_t z, uint32_t w, float amp, float ampw)
{
    const float m3a = -3.0f * amp, m3w = -3.0f * ampw;
    if (METHOD == kPerlinS5 || METHOD == kPerlinS3)
        return make_float4(0.0f, unit_scaled(y, amp, m3a), unit_scaled(z, amp, m3a), unit_scaled(w, amp, m3a));
    return make_float4(unit_scaled(x, amp, m3a), unit_scaled(y, ampw, m3w), unit_scaled(z, ampw, m3w),
                       unit_scaled(w, ampw, m3w));
}

// Corners of every staged octave of the tile, hashed once each, in four passes
// with each fine octave's corner grid known at compile time:
//   1. octaves with cells of 32 samples or more (2 x 2 x 2 corners each): all
//      of them at once, a lane a corner, from the last thread down;
//   2. cells of 16 and 8 samples (3 x 2 x 2 and 5 x 3 x 2 corners): one flat
//      pass of 42 corners;
//   3. cells of 4 samples (9 x 5 x 3 corners): a flat loop of constant shape;
//   4. cells of 2 samples (17 x 9 x 5 corners): a warp two corner rows at a
//      time (16 lanes a row), with x's LCG step taken once per lane and the
//      others once per row; column 16 by the last threads down.
template <int METHOD, bool kUnit = false>
__device__ __forceinline__ void stage_corners3(const FieldPlan& P, float4* __restrict__ corners, int j0x, int j0y,
                                               int j0z)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int s = P.s, N = P.N;
    {  // 1. octaves i <= s - 5, eight slots each from the first (rowlen 2)
        int n5 = s - 4;
        n5 = n5 < 0 ? 0 : (n5 < P.nst ? n5 : P.nst);
        for (int e = kThreads - 1 - tid; e < 8 * n5; e += kThreads) {
            const int i = e >> 3, c = e & 7;
            const OctPlan& op = P.oct[i];
            uint32_t x = op.ox + ((uint32_t)j0x >> op.k) + (uint32_t)(c & 1);
            uint32_t y = op.oy + ((uint32_t)j0y >> op.k) + (uint32_t)((c >> 1) & 1);
            uint32_t z = op.oz + ((uint32_t)j0z >> op.k) + (uint32_t)(c >> 2);
            uint32_t w = op.key;
            pcg4d(x, y, z, w);
            if (bounds_ok(kSiteStage, c, op.rowlen * op.ncy * op.ncz))
                sst(kSiteStage, &corners[op.coff + c], corner_data4<METHOD>(x, y, z, w, kUnit ? 1.0f : op.amp, kUnit ? P.grad_w : op.ampw));
        }
    }
    {  // 2. cells of 16 and 8 samples
        const int n4 = (s >= 4 && s - 4 < N) ? ncx3(4) * ncy3(4) * ncz3(4) : 0;
        const int n3 = (s >= 3 && s - 3 < N) ? ncx3(3) * ncy3(3) * ncz3(3) : 0;
        static_assert(ncx3(4) * ncy3(4) * ncz3(4) + ncx3(3) * ncy3(3) * ncz3(3) <= kThreads, "one corner a thread");
        int e = tid, K = 4;
        if (e >= n4) {
            e -= n4;
            K = 3;
        }
        if (K == 4 || e < n3) {
            const OctPlan& op = P.oct[s - K];
            const int nxy = op.ncx * op.ncy;
            const int cz = (int)__umulhi((uint32_t)e, op.magic2);
            const int rem = e - cz * nxy;
            const int cy = (int)__umulhi((uint32_t)rem, op.magic);
            const int cx = rem - cy * op.ncx;
            uint32_t x = op.ox + ((uint32_t)j0x >> K) + (uint32_t)cx, y = op.oy + ((uint32_t)j0y >> K) + (uint32_t)cy;
            uint32_t z = op.oz + ((uint32_t)j0z >> K) + (uint32_t)cz, w = op.key;
            pcg4d(x, y, z, w);
            const int slot = (cz * op.ncy + cy) * op.rowlen + corner_slot(cx);
            if (bounds_ok(kSiteStage, slot, op.rowlen * op.ncy * op.ncz))
                sst(kSiteStage, &corners[op.coff + slot], corner_data4<METHOD>(x, y, z, w, kUnit ? 1.0f : op.amp, kUnit ? P.grad_w : op.ampw));
        }
    }
    if (s >= 2 && s - 2 < N) {  // 3. cells of 4 samples
        const OctPlan& op = P.oct[s - 2];
        constexpr int NX = ncx3(2), NY = ncy3(2), NZ = ncz3(2), RL = rowlen3(2);
        const uint32_t bx = op.ox + ((uint32_t)j0x >> 2), by = op.oy + ((uint32_t)j0y >> 2);
        const uint32_t bz = op.oz + ((uint32_t)j0z >> 2);
        float4* cg = corners + op.coff;
        const float amp = kUnit ? 1.0f : op.amp, ampw = kUnit ? P.grad_w : op.ampw;
        const uint32_t key = op.key;
        for (int e = tid; e < NX * NY * NZ; e += kThreads) {
            const int cz = e / (NX * NY), rem = e - cz * (NX * NY);
            const int cy = rem / NX, cx = rem - cy * NX;
            uint32_t x = bx + (uint32_t)cx, y = by + (uint32_t)cy, z = bz + (uint32_t)cz, w = key;
            pcg4d(x, y, z, w);
            sst(kSiteStage, &cg[(cz * NY + cy) * RL + corner_slot(cx)], corner_data4<METHOD>(x, y, z, w, amp, ampw));
        }
    }
    if (s >= 1 && s - 1 < N) {  // 4. cells of 2 samples
        const OctPlan& op = P.oct[s - 1];
        constexpr int NX = ncx3(1), NY = ncy3(1), NZ = ncz3(1), RL = rowlen3(1);
        static_assert(NX == 17, "17 corners a row: 16 lanes and one extra column");
        const uint32_t bx = op.ox + ((uint32_t)j0x >> 1), by = op.oy + ((uint32_t)j0y >> 1);
        const uint32_t bz = op.oz + ((uint32_t)j0z >> 1);
        float4* cg = corners + op.coff;
        const float amp = kUnit ? 1.0f : op.amp, ampw = kUnit ? P.grad_w : op.ampw;
        const int half = lane >> 4, col = lane & 15;
        const uint32_t w1 = pcg_lcg(op.key), x1 = pcg_lcg(bx + (uint32_t)col);
        float4* dst = cg + corner_slot(col);
        for (int pr = warp; pr < (NY * NZ + 1) / 2; pr += kThreads / 32) {
            const int r = 2 * pr + half;  // corner row r = cz * NY + cy
            if (r < NY * NZ) {
                const int cz = r / NY, cy = r - cz * NY;
                uint32_t x = x1, y = pcg_lcg(by + (uint32_t)cy), z = pcg_lcg(bz + (uint32_t)cz), w = w1;
                pcg4d_post(x, y, z, w);
                sst(kSiteStage, &dst[r * RL], corner_data4<METHOD>(x, y, z, w, amp, ampw));
            }
        }
        for (int r = kThreads - 1 - tid; r < NY * NZ; r += kThreads) {  // column 16
            const int cz = r / NY, cy = r - cz * NY;
            uint32_t x = bx + 16u, y = by + (uint32_t)cy, z = bz + (uint32_t)cz, w = op.key;
            pcg4d(x, y, z, w);
            sst(kSiteStage, &cg[r * RL + corner_slot(NX - 1)], corner_data4<METHOD>(x, y, z, w, amp, ampw));
        }
    }
}

template <int METHOD, bool kTile>
__device__ __forceinline__ void stage_tile3(const FieldPlan& P, float4* sm, int j0x, int j0y, int j0z)
{
    constexpr int NN = Deg<METHOD>::value + 1;
    const int tid = threadIdx.x, s = P.s, n8 = n_run8(P), nt = kTile ? n_tile3<METHOD>(P) : 0;
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
    stage_corners3<METHOD>(P, corners, j0x, j0y, j0z);
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

// The tile octaves' sum at the 64 tile nodes, two lanes a node, each taking
// every other octave, added by one shuffle.  Warp w holds the 16 nodes of
// tile-node row y = w (lane 8 x + 2 z + part), so it can reduce them along z
// for every plane: Hz[(plane * 4 + y) * 4 + x] = sum_c wz[plane][c] G(x, y, c),
// the tile polynomial at the plane and the (y, x) nodes.
template <int METHOD>
__device__ __forceinline__ void tile_grid3(const FieldPlan& P, const float4* __restrict__ corners, float* Hz, int j0x,
                                           int j0y, int j0z, int nt)
{
    const int tid = threadIdx.x, lane = tid & 31, part = lane & 1;
    const int nx = lane >> 3, ny = tid >> 5, nz = (lane >> 1) & 3;
    const uint32_t jx = (uint32_t)(j0x + node3(0, nx)), jy = (uint32_t)(j0y + node3(1, ny));
    const uint32_t jz = (uint32_t)(j0z + node3(2, nz));
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
    const int plane = lane >> 2, a = lane & 3;  // this lane's table entry (plane, y = w, x = a)
    float g[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) g[c] = __shfl_sync(0xffffffffu, v, (a << 3) | (c << 1));
    const float4 wz = __ldg(reinterpret_cast<const float4*>(kTile3Weights.wz[plane]));
    sst(kSiteTable, &Hz[(plane * 4 + ny) * 4 + a], fmaf(wz.w, g[3], fmaf(wz.z, g[2], fmaf(wz.y, g[1], wz.x * g[0]))));
}

// Interpolate the tile nodes to the thread's plane (from the z-reduced table),
// evaluated rows and node columns.
__device__ __forceinline__ void add_tile_grid3(float (&nacc)[2][4], const float* __restrict__ Hz, int tx, int ty,
                                               int tz, int par)
{
    const Tile3Weights& W = kTile3Weights;
    float hz[4][4];  // [y node][x node] in the thread's plane
    const float4* H4 = reinterpret_cast<const float4*>(Hz) + tz * 4;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const float4 h = sld(kSiteTable, &H4[b]);
        hz[b][0] = h.x;
        hz[b][1] = h.y;
        hz[b][2] = h.z;
        hz[b][3] = h.w;
    }
    float4 wx[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
        wx[q] = bounds_ok(kSiteConst, tx, 4) ? __ldg(reinterpret_cast<const float4*>(W.wx[tx][q]))
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int row = ty * kRows + eval_row3<kC1>(r, par);
        const float4 wy = bounds_ok(kSiteConst, row, 16) ? __ldg(reinterpret_cast<const float4*>(W.wy[row]))
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
__device__ __forceinline__ void run8_octave3(float (&nacc)[n_rows3<METHOD>()][Deg<METHOD>::value + 1],
                                             float (&vacc)[n_rows3<METHOD>()], const float4* __restrict__ sm,
                                             const FieldPlan& P, int i, int tx, int ty, int tz, int n8, int par)
{
    constexpr int NN = Deg<METHOD>::value + 1, NRW = n_rows3<METHOD>();
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
    for (int r = 0; r < NRW; ++r) {
        const float4 yb = sld(kSiteTable, &ylut[i * 16 + eval_row3<METHOD>(r, par) * 4 + ty]);
        const Row R = row_of(c, yb.x, yb.y, yb.z);
        vacc[r] += R.V0;  // the same at every node: summed once per row
#pragma unroll
        for (int q = 0; q < NN; ++q) nacc[r][q] = Model<METHOD>::eval_add(R, xb[q], nacc[r][q]);
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
                for (int q = 0; q < CW; q += 2) {  // neighbouring columns: one paired add
                    float h0;
                    if (q == 0) {
                        h0 = R.V0;
                    } else {
                        const float4 xb = axis_basis<METHOD>(q * inv);
                        h0 = eval_row(R, xb.x, xb.y, xb.z);
                    }
                    const float4 xb1 = axis_basis<METHOD>((q + 1) * inv);
                    const float h1 = eval_row(R, xb1.x, xb1.y, xb1.z);
                    float& a0 = acc[yq * CW + rr][xq * CW + q];
                    float& a1 = acc[yq * CW + rr][xq * CW + q + 1];
                    const float2 a = __fadd2_rn(make_float2(a0, a1), make_float2(h0, h1));
                    a0 = a.x;
                    a1 = a.y;
                }
            }
        }
    }
}

// Adds amp unit_mant(h), neighbouring columns by one paired FMA; the -3 amp
// terms of all lattice octaves (FieldPlan::lat_bias) start every sample's sum
// instead.
__device__ __forceinline__ void lattice_octave3(float (&acc)[kRows][kCols], const OctPlan& op, uint32_t jx,
                                                uint32_t jy, uint32_t jz)
{
    const int sh = op.k;
    const uint32_t z1 = pcg_lcg(op.oz + (jz << sh)), w1 = pcg_lcg(op.key);
    const uint32_t dx = 1664525u << sh, x0 = op.ox + (jx << sh);  // x's LCG step advances by dx a column
    const float2 amp2 = make_float2(op.amp, op.amp);
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const uint32_t y1 = pcg_lcg(op.oy + ((jy + r) << sh));
        const uint32_t base = pcg4d_run_base(x0, y1, w1);
#pragma unroll
        for (int c = 0; c < kCols; c += 2) {
            const uint32_t h0 = pcg4d_run_value(base + (uint32_t)c * dx, y1, z1, w1);
            const uint32_t h1 = pcg4d_run_value(base + (uint32_t)(c + 1) * dx, y1, z1, w1);
            const float2 a = __ffma2_rn(make_float2(unit_mant(h0), unit_mant(h1)), amp2,
                                        make_float2(acc[r][c], acc[r][c + 1]));
            acc[r][c] = a.x;
            acc[r][c + 1] = a.y;
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

// Six CTAs a SM for C1 (at most 80 registers; the compiler's own choice is
// 86, which leaves five); the other models keep the compiler's choice.
template <int METHOD>
constexpr int min_ctas3() { return METHOD == kC1 ? 6 : 0; }

// kTile: the field sums its tile octaves at the tile nodes (n_tile3 > 0).
template <int METHOD, typename OutT, bool kTile>
__global__ void __launch_bounds__(kThreads, min_ctas3<METHOD>()) fbm3d_kernel(const __grid_constant__ FieldPlan P)
{
    constexpr int D = Deg<METHOD>::value, NN = D + 1;
    extern __shared__ float4 sm[];
    const int tid = threadIdx.x, tx = tid & 3, ty = (tid >> 2) & 3, tz = tid >> 4;
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH, z0 = blockIdx.z * kTD;  // output tile
    const int j0x = x0 + P.jx0, j0y = y0 + P.jy0, j0z = z0 + P.jz0;                  // sample indices
    const int s = P.s, N = P.N, n8 = n_run8(P), nt = kTile ? n_tile3<METHOD>(P) : 0;
    stage_tile3<METHOD, kTile>(P, sm, j0x, j0y, j0z);
    __syncthreads();

    // tile octaves: their sum at the tile nodes, reduced along z for every
    // plane (read back after the barrier below)
    float* Hz = reinterpret_cast<float*>(sm + corner_base3<METHOD>(n8) + P.ncorner);
    if (nt > 0) tile_grid3<METHOD>(P, sm + corner_base3<METHOD>(n8), Hz, j0x, j0y, j0z, nt);

    constexpr int NRW = n_rows3<METHOD>();
    const int par = node_rows3<METHOD>() ? (ty & 1) : 0;
    float nacc[NRW][NN], vacc[NRW];
#pragma unroll
    for (int r = 0; r < NRW; ++r) {
        vacc[r] = 0.0f;
#pragma unroll
        for (int q = 0; q < NN; ++q) nacc[r][q] = 0.0f;
    }
    for (int i = nt; i < n8; ++i) run8_octave3<METHOD>(nacc, vacc, sm, P, i, tx, ty, tz, n8, par);
#pragma unroll
    for (int r = 0; r < NRW; ++r)
#pragma unroll
        for (int q = 0; q < NN; ++q) nacc[r][q] += vacc[r];
    // the run and tile octaves' sum at the node columns of all rows
    float rowv[kRows][NN];
    if constexpr (!node_rows3<METHOD>()) {
#pragma unroll
        for (int r = 0; r < kRows; ++r)
#pragma unroll
            for (int q = 0; q < NN; ++q) rowv[r][q] = nacc[r][q];
    } else {
        if (nt > 0) {  // uniform over the CTA
            __syncthreads();
            add_tile_grid3(nacc, Hz, tx, ty, tz, par);
        }
        // mirrored block rows: own nodes at 0, 2, the partner's at 5, 7
#pragma unroll
        for (int q = 0; q < NN; ++q) {
            const float p5 = __shfl_xor_sync(0xffffffffu, nacc[1][q], 4);
            const float p7 = __shfl_xor_sync(0xffffffffu, nacc[0][q], 4);
            float v[4];
            v[0] = nacc[0][q];
            v[2] = nacc[1][q];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int y = 2 * j + 1;
                v[y] = fmaf(lagrange<3>(y, 3), p7, fmaf(lagrange<3>(y, 2), p5,
                           fmaf(lagrange<3>(y, 1), v[2], lagrange<3>(y, 0) * v[0])));
            }
#pragma unroll
            for (int r = 0; r < kRows; ++r) rowv[r][q] = par ? v[kRows - 1 - r] : v[r];
        }
    }
    // the -3 amp offsets of all lattice octaves start every sample's sum
    constexpr bool kPerlin = METHOD == kPerlinS5 || METHOD == kPerlinS3;
    const float lat = (!kPerlin && s < N) ? P.lat_bias : 0.0f;
    float acc[kRows][kCols];
#pragma unroll
    for (int r = 0; r < kRows; ++r)
#pragma unroll
        for (int c = 0; c < kCols; ++c) {
            const int q = node_of_col<D>(c);
            if (q >= 0) {
                acc[r][c] = rowv[r][q] + lat;
            } else {
                float v = lat;
#pragma unroll
                for (int m = 0; m < NN; ++m) v = fmaf(lagrange<D>(c, m), rowv[r][m], v);
                acc[r][c] = v;
            }
        }
    if (s >= 2 && s - 2 < N) small_octave3<METHOD, 4>(acc, sm, P, s - 2, tx, ty, tz, n8);
    if (s >= 1 && s - 1 < N) small_octave3<METHOD, 2>(acc, sm, P, s - 1, tx, ty, tz, n8);
    if (!kPerlin && s < N) {  // Perlin is zero at lattice points
        const uint32_t jx = (uint32_t)(j0x + tx * kCols), jy = (uint32_t)(j0y + ty * kRows), jz = (uint32_t)(j0z + tz);
        for (int i = s; i < N; ++i) lattice_octave3(acc, P.oct[i], jx, jy, jz);
    }
    store_tile3<OutT>(P, acc, x0 + tx * kCols, y0 + ty * kRows, z0 + tz);
}

// ---------------------------------------------------------------------------
// Ridged multifractal (PTG_RIDGED), fused 3D form: as the 2D ridged kernel
// (every octave at every sample, in octave order, r = (1 - |h|)^2 w added
// with weight p^i and w = clamp(2 r, 0, 1)), on this kernel's tiles and
// staging.  Per-CTA tables hold the x-, y- and z-bases of the octaves with
// cells of 8 samples or more (32 + 16 + 8 an octave; x rotated so that a
// quarter warp's four runs read four bank groups).
// ---------------------------------------------------------------------------
constexpr int kRidgeTab3 = kTW + kTH + kTD;  // basis-table entries an octave

__device__ __forceinline__ int ridge_xslot3(int j) { return j ^ ((j >> 3) & 3); }

__device__ __forceinline__ void ridge2_3(float& acc0, float& acc1, float& w0, float& w1, float h0, float h1, float wgt)
{
    const float2 a = make_float2(1.0f - fabsf(h0), 1.0f - fabsf(h1));
    const float2 r = __fmul2_rn(__fmul2_rn(a, a), make_float2(w0, w1));
    const float2 ac = __ffma2_rn(make_float2(wgt, wgt), r, make_float2(acc0, acc1));
    acc0 = ac.x;
    acc1 = ac.y;
    w0 = __saturatef(2.0f * r.x);
    w1 = __saturatef(2.0f * r.y);
}

// Cells of CW = 4 or 2 samples: constant in-cell positions along x and y,
// the thread's plane at (tz mod CW) / CW along z (as small_octave3).
template <int METHOD, int CW>
__device__ __forceinline__ void small_ridged3(float (&acc)[kRows][kCols], float (&w)[kRows][kCols],
                                              const float4* __restrict__ corners, const OctPlan& op, int tx, int ty,
                                              int tz)
{
    const float4* cg = corners + op.coff;
    constexpr float inv = 1.0f / CW;
    const float4 zb = axis_basis<METHOD>((float)(tz & (CW - 1)) * inv);
    const int lcz = tz / CW;
    const float wgt = op.amp;
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
                for (int q = 0; q < CW; q += 2) {
                    const float4 xb1 = axis_basis<METHOD>((q + 1) * inv);
                    float h0 = R.V0;
                    if (q > 0) {
                        const float4 xb = axis_basis<METHOD>(q * inv);
                        h0 = eval_row(R, xb.x, xb.y, xb.z);
                    }
                    const float h1 = eval_row(R, xb1.x, xb1.y, xb1.z);
                    const int y = yq * CW + rr, x = xq * CW + q;
                    ridge2_3(acc[y][x], acc[y][x + 1], w[y][x], w[y][x + 1], h0, h1, wgt);
                }
            }
        }
    }
}

template <int METHOD, typename OutT>
__global__ void __launch_bounds__(kThreads) fbm3d_ridged_kernel(const __grid_constant__ FieldPlan P)
{
    extern __shared__ float4 sm[];
    const int tid = threadIdx.x, tx = tid & 3, ty = (tid >> 2) & 3, tz = tid >> 4;
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH, z0 = blockIdx.z * kTD;
    const int j0x = x0 + P.jx0, j0y = y0 + P.jy0, j0z = z0 + P.jz0;
    const int s = P.s, N = P.N, nb = n_run8(P);
    for (int e = tid; e < nb * kRidgeTab3; e += kThreads) {  // bases of the octaves with cells >= 8
        const int i = e / kRidgeTab3, j = e - i * kRidgeTab3;
        const uint32_t pos = (uint32_t)(j < kTW ? j0x + j : (j < kTW + kTH ? j0y + j - kTW : j0z + j - kTW - kTH));
        sst(kSiteStage, &sm[i * kRidgeTab3 + (j < kTW ? ridge_xslot3(j) : j)], axis_basis<METHOD>(axis_t(pos, i, s)));
    }
    float4* corners = sm + nb * kRidgeTab3;
    stage_corners3<METHOD, true>(P, corners, j0x, j0y, j0z);
    __syncthreads();

    float acc[kRows][kCols], w[kRows][kCols];
#pragma unroll
    for (int r = 0; r < kRows; ++r)
#pragma unroll
        for (int c = 0; c < kCols; ++c) {
            acc[r][c] = 0.0f;
            w[r][c] = 1.0f;
        }
    for (int i = 0; i < nb; ++i) {  // one cell a thread; octaves in order (the weights chain)
        const OctPlan& op = P.oct[i];
        const float4* tb = sm + i * kRidgeTab3;
        const Cell c = zcell(corners + op.coff, op, (tx * kCols) >> op.k, (ty * kRows) >> op.k, tz >> op.k,
                             sld(kSiteTable, &tb[kTW + kTH + tz]));
        const float wgt = op.amp;
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const float4 yb = sld(kSiteTable, &tb[kTW + ty * kRows + r]);
            const Row R = row_of(c, yb.x, yb.y, yb.z);
#pragma unroll
            for (int q = 0; q < kCols; q += 2) {
                const float4 xa = sld(kSiteTable, &tb[ridge_xslot3(tx * kCols + q)]);
                const float4 xc = sld(kSiteTable, &tb[ridge_xslot3(tx * kCols + q + 1)]);
                ridge2_3(acc[r][q], acc[r][q + 1], w[r][q], w[r][q + 1], eval_row(R, xa.x, xa.y, xa.z),
                         eval_row(R, xc.x, xc.y, xc.z), wgt);
            }
        }
    }
    if (s >= 2 && s - 2 < N) small_ridged3<METHOD, 4>(acc, w, corners, P.oct[s - 2], tx, ty, tz);
    if (s >= 1 && s - 1 < N) small_ridged3<METHOD, 2>(acc, w, corners, P.oct[s - 1], tx, ty, tz);
    const uint32_t jx = (uint32_t)(j0x + tx * kCols), jy = (uint32_t)(j0y + ty * kRows), jz = (uint32_t)(j0z + tz);
    for (int i = s; i < N; ++i) {  // lattice octaves: the corner value (zero for Perlin)
        const OctPlan& op = P.oct[i];
        const float wgt = op.amp;
        if constexpr (METHOD == kPerlinS5 || METHOD == kPerlinS3) {
#pragma unroll
            for (int r = 0; r < kRows; ++r)
#pragma unroll
                for (int c = 0; c < kCols; c += 2) ridge2_3(acc[r][c], acc[r][c + 1], w[r][c], w[r][c + 1], 0.f, 0.f, wgt);
        } else {
            const int sh = op.k;
            const uint32_t z1 = pcg_lcg(op.oz + (jz << sh)), w1 = pcg_lcg(op.key);
            const uint32_t dx = 1664525u << sh, xs = op.ox + (jx << sh);
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                const uint32_t y1 = pcg_lcg(op.oy + ((jy + r) << sh));
                const uint32_t base = pcg4d_run_base(xs, y1, w1);
#pragma unroll
                for (int c = 0; c < kCols; c += 2)
                    ridge2_3(acc[r][c], acc[r][c + 1], w[r][c], w[r][c + 1],
                             unit_value(pcg4d_run_value(base + (uint32_t)c * dx, y1, z1, w1)),
                             unit_value(pcg4d_run_value(base + (uint32_t)(c + 1) * dx, y1, z1, w1)), wgt);
            }
        }
    }
    store_tile3<OutT>(P, acc, x0 + tx * kCols, y0 + ty * kRows, z0 + tz);
}

template <int METHOD>
size_t smem_words3(const FieldPlan& P)
{
    int n8 = P.s - 2;
    n8 = n8 < 0 ? 0 : (n8 < P.N ? n8 : P.N);
    if (P.ridged) return (size_t)n8 * kRidgeTab3 + (size_t)P.ncorner;
    return (size_t)corner_base3<METHOD>(n8) + (size_t)P.ncorner + (n_tile3<METHOD>(P) > 0 ? kTD * 16 / 4 : 0);
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
        auto kfn = P.ridged ? fbm3d_ridged_kernel<M, T>                                              \
                   : (M == kC1 && n_tile3<M>(P) > 0 ? fbm3d_kernel<M, T, M == kC1> : fbm3d_kernel<M, T, false>); \
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
