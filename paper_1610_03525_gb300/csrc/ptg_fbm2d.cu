// ptg_fbm2d.cu -- fused all-octave 2D generator for the polynomial noise of
// Thorimbert & Chopard (arXiv:1610.03525) and for Perlin's polynomial.
//
// One CTA makes a 64 x 64 tile of samples with 128 threads; each thread owns a
// run of RW consecutive columns in RR rows (RW x RR = 8 x 4 or 16 x 2, the
// "thread shape") and keeps their fractal sums (Sec. 4) in registers across
// all octaves, then writes each sample once.
//
// Inside a cell every method is separable.  For one row y the cell collapses
// to a 1D function of x,
//     h(x, y) = V0 + S(x) (V1 - V0) + B0(x) F0 + B1(x) F1,
//     V_a = v_a0 + S(y) (v_a1 - v_a0) + B0(y) g_a0 + B1(y) g_a1,
//     F_a = f_a0 + S(y) (f_a1 - f_a0),
// the tensor-product Hermite cell (C1: cubic, C2: quintic) of Eq. (polynomial)
// with the corner constraints of Eq. (mixedderiv) and zero mixed derivatives,
// or Perlin's polynomial (Sec. 3.2) with v = 0 and its own B0, B1.
//
// Octave i has cells of spc_i = spc / 2^i samples.  Four regimes:
//   spc_i >= 64 ("tile" octaves): the cell covers the whole tile, so each
//     octave -- and their sum -- is one polynomial of degree d per axis over
//     the tile.  The CTA evaluates that sum at (d + 1)^2 tile nodes once and
//     every thread interpolates it to its own node columns.
//   RW <= spc_i < 64 ("run" octaves): a thread's run lies in one cell, so each of
//     its rows is one polynomial of degree d in the column (d = 3 for C1, 5 for
//     C2, 4 / 6 for Perlin S3 / S5), and so is the sum over all such octaves.
//     The kernel evaluates d + 1 node columns per octave and fills the other
//     columns once, at the end, by exact Lagrange interpolation.  The wider
//     run halves the per-sample cost of these octaves and adds interpolated
//     columns; which shape is faster depends on the octave mix.
//     With degree 3 and runs of 8 the same holds along y: the two threads
//     that share an 8 x 8 block (one cell of the finest run octave) evaluate
//     rows 0, 2 and 5, 7 of it only, swap them, and interpolate rows 1, 3, 4
//     and 6 (the "node rows"; together with the tile octaves' sum, which is a
//     cubic over the whole tile).
//   2 <= spc_i < RW: in-cell column positions are the constants q / spc_i and
//     positions t = 0 take the corner data directly.
//   spc_i <= 1 ("lattice"): every sample is a lattice point, where the cell
//     polynomial equals the corner value: one hash per sample (zero for
//     Perlin, whose value at lattice points is zero).
// Corners of every staged octave (cells >= 2 samples) are hashed once per CTA
// into shared memory, pre-scaled by the octave amplitude (Sec. 4.1's C_init),
// and the per-axis basis of the run octaves is tabulated per CTA (the paper's
// precomputed space-only terms, Sec. 5.2).
#include "ptg_device.cuh"
#include "ptg_eval.cuh"
#include "ptg_kernels.h"

namespace ptg {
namespace {

constexpr int kTW = kTile2dX, kTH = kTile2dY, kThreads = 128;

// Thread shape: RW consecutive columns x RR rows per thread.
template <int RW>
struct Shape {
    static_assert(RW == 8 || RW == 16, "run width 8 or 16");
    static constexpr int RR = 32 / RW;        // rows per thread
    static constexpr int TXN = kTW / RW;      // threads along x
    static constexpr int TYN = kTH / RR;      // threads along y
    static constexpr int LOG = RW == 8 ? 3 : 4;
};
static_assert(Shape<8>::TXN * Shape<8>::TYN == kThreads && Shape<16>::TXN * Shape<16>::TYN == kThreads, "");

// Node rows (degree 3, runs of 8 x 4): the sum of the run and tile octaves
// over an 8 x 8 block (the thread pair ty = 2b, 2b + 1, lanes l and l ^ 8 of
// one warp) is one bicubic, so it is evaluated at the block's rows 0, 2, 5, 7
// (the node columns' positions, Lebesgue constant 1.4) and interpolated at
// the other four.  The even thread evaluates its rows 0 and 2, the odd one
// its rows 3 and 1 (block rows 7 and 5): mirrored, so that both take the
// same interpolation weights.  NRW = rows a thread evaluates.
template <int METHOD, int RW>
__host__ __device__ constexpr bool node_rows() { return Deg<METHOD>::value == 3 && RW == 8; }

template <int METHOD, int RW>
__host__ __device__ constexpr int n_rows() { return node_rows<METHOD, RW>() ? 2 : Shape<RW>::RR; }

// Row (within the thread's RR rows) of its k-th evaluated row; par = ty & 1.
template <int METHOD, int RW>
__device__ __forceinline__ int eval_row(int k, int par)
{
    return node_rows<METHOD, RW>() ? (k == 0 ? 3 * par : 2 - par) : k;
}

// Shared-memory layout (float4 units), with ng = run octaves with cells of
// 128 samples or more that are not tile octaves (their basis depends on the
// tile's place in the cell; finer run octaves read constant tables):
//   x-basis of those octaves at node columns [ng][D+1][TXN],
//   y-basis of those octaves [ng][RR rows][TYN] (64 per octave),
//   a copy of the constant basis tables of the finer run octaves (Perlin, if any),
//   staged corners of every staged octave (rows swizzled by corner_slot),
//   with tile octaves: the tile nodes' values [D+1][LW], then a copy of the
//   interpolation weights (TileWeights) made while the corners are hashed,
//   then (degree 3) the tile polynomial at every tile row and node column.
template <int METHOD, int RW>
__host__ __device__ constexpr int xnode_words(int ng) { return ng * (Deg<METHOD>::value + 1) * Shape<RW>::TXN; }

// The tile polynomial at every tile row and each of the d + 1 tile-node
// columns, Tt[q][64] (degree 3: built by the warps that hold the node values).
template <int METHOD>
__host__ __device__ constexpr int row_table_words() { return Deg<METHOD>::value == 3 ? 4 * 64 / 4 : 0; }

template <int METHOD, int RW>
__host__ __device__ constexpr int grid_words()  // float4 words: tile nodes' values, their weights, the row table
{
    return ((Deg<METHOD>::value + 1) * TileWeights<Deg<METHOD>::value, RW>::LW +
            (int)sizeof(TileWeights<Deg<METHOD>::value, RW>) / 4) / 4 + row_table_words<METHOD>();
}

// Tile octaves: octaves with cells >= 64 samples that the host chose to sum
// at the tile nodes (P.nt; never for degree > 4, where the (d+1)^2 nodes cost
// about what they save).
template <int METHOD>
__host__ __device__ __forceinline__ int n_tile(const FieldPlan& P)
{
    return Deg<METHOD>::value <= 4 ? P.nt : 0;
}

// Octaves with cells of 128 samples or more (the first ones in the corner
// layout), and those of them that are run octaves (not tile octaves).
__host__ __device__ __forceinline__ int n_coarse(const FieldPlan& P)
{
    const int n = P.s - 6;
    return n < 0 ? 0 : (n < P.N ? n : P.N);
}

template <int METHOD>
__host__ __device__ __forceinline__ int n_generic(const FieldPlan& P)
{
    const int n = n_coarse(P) - n_tile<METHOD>(P);
    return n > 0 ? n : 0;
}

// Whether the field has run octaves with cells of 2^LOG .. 64 samples (the
// octaves that read the constant basis tables).
template <int METHOD, int RW>
__host__ __device__ __forceinline__ bool has_fine_runs(const FieldPlan& P)
{
    int kmax = P.s - n_tile<METHOD>(P), kmin = P.s - P.N + 1;
    kmax = kmax < 6 ? kmax : 6;
    kmin = kmin > Shape<RW>::LOG ? kmin : Shape<RW>::LOG;
    return kmax >= kmin;
}

// Where run_octave_k reads the constant basis tables: a shared-memory copy
// made while the corners are hashed (Perlin) or the global tables through the
// read-only cache (the polynomial models).  Each is the faster of the two for
// its kernels, by measurement on GB300 (2-9%).
template <int METHOD>
__host__ __device__ constexpr bool shared_run_basis() { return METHOD == kPerlinS5 || METHOD == kPerlinS3; }

template <int METHOD, int RW>
__host__ __device__ __forceinline__ int run_basis_words(const FieldPlan& P)  // shared-memory copy, float4 words
{
    return shared_run_basis<METHOD>() && has_fine_runs<METHOD, RW>(P) ? (int)sizeof(RunBasis<METHOD, RW>) / 16 : 0;
}

// Basis tables of the run octaves with cells of 8 .. 64 samples.
template <int METHOD, int RW>
__device__ const RunBasis<METHOD, RW> kRunBasis = make_run_basis<METHOD, RW>();

// Interpolation weights of the tile nodes (compile-time tables).
template <int D, int RW>
__device__ const TileWeights<D, RW> kTileWeights = make_tile_weights<D, RW>();

// Corners of every staged octave of a 64 x 64 tile, hashed once each (Sec. 4.1's
// C_init), pre-scaled by the octave amplitude (kUnit: at unit amplitude, with
// the gradient weight alone, for the ridged sum).  The layout fixes each fine
// octave's corner grid, so the work is split into four passes with that
// geometry known at compile time:
//   1. octaves with cells of 64 samples or more: 2 x 2 corners each, at 4 i,
//      all of them at once, a lane a corner (from the last thread down);
//   2. cells of 32, 16 and 8 samples (3 x 3, 5 x 5 and 9 x 9 corners): their
//      115 corners in one flat pass, a thread a corner;
//   3. cells of 4 samples (17 x 17 corners): a flat loop of constant shape;
//   4. cells of 2 samples (33 x 33 corners): a warp a corner row, a lane a
//      column (column 32 by the lanes of warps 1 to 3), with x's LCG step
//      taken once per lane and y's once per row.
template <int METHOD, bool kUnit = false>
__device__ __forceinline__ void stage_corners(const FieldPlan& P, float4* __restrict__ corners, int j0x, int j0y)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int s = P.s, N = P.N;
    {  // 1. octaves i <= s - 6
        int n6 = s - 5;
        n6 = n6 < 0 ? 0 : (n6 < P.nst ? n6 : P.nst);
        const int e = kThreads - 1 - tid;
        if (e < 4 * n6) {
            const int i = e >> 2, c = e & 3;
            const OctPlan& op = P.oct[i];
            uint32_t x = op.ox + ((uint32_t)j0x >> op.k) + (uint32_t)(c & 1);
            uint32_t y = op.oy + ((uint32_t)j0y >> op.k) + (uint32_t)(c >> 1);
            uint32_t z = op.key;
            pcg3d(x, y, z);
            sst(kSiteStage, &corners[4 * i + c],
                corner_data<METHOD>(x, y, z, kUnit ? 1.0f : op.amp, kUnit ? P.grad_w : op.ampw));
        }
    }
    {  // 2. cells of 32, 16 and 8 samples
        const int n5 = (s >= 5 && s - 5 < N) ? corner_ncx2(5) * corner_ncx2(5) : 0;
        const int n4 = (s >= 4 && s - 4 < N) ? corner_ncx2(4) * corner_ncx2(4) : 0;
        const int n3 = (s >= 3 && s - 3 < N) ? corner_ncx2(3) * corner_ncx2(3) : 0;
        static_assert(corner_ncx2(5) * corner_ncx2(5) + corner_ncx2(4) * corner_ncx2(4) +
                          corner_ncx2(3) * corner_ncx2(3) <= kThreads, "one corner a thread");
        int e = tid, K = 5;
        if (e >= n5) {
            e -= n5;
            K = 4;
            if (e >= n4) {
                e -= n4;
                K = 3;
            }
        }
        if (K > 3 || e < n3) {
            const OctPlan& op = P.oct[s - K];
            const int cy = (int)__umulhi((uint32_t)e, op.magic);
            const int cx = e - cy * op.ncx;
            uint32_t x = op.ox + ((uint32_t)j0x >> K) + (uint32_t)cx;
            uint32_t y = op.oy + ((uint32_t)j0y >> K) + (uint32_t)cy;
            uint32_t z = op.key;
            pcg3d(x, y, z);
            if (bounds_ok(kSiteStage, cy * op.rowlen + corner_slot(cx), op.rowlen * op.ncy))
                sst(kSiteStage, &corners[op.coff + cy * op.rowlen + corner_slot(cx)],
                    corner_data<METHOD>(x, y, z, kUnit ? 1.0f : op.amp, kUnit ? P.grad_w : op.ampw));
        }
    }
    if (s >= 2 && s - 2 < N) {  // 3. cells of 4 samples
        const OctPlan& op = P.oct[s - 2];
        constexpr int NC = corner_ncx2(2), RL = corner_rowlen2(2);
        const uint32_t bx = op.ox + ((uint32_t)j0x >> 2), by = op.oy + ((uint32_t)j0y >> 2);
        float4* cg = corners + op.coff;
        const float amp = kUnit ? 1.0f : op.amp, ampw = kUnit ? P.grad_w : op.ampw;
        const uint32_t key = op.key;
        for (int e = tid; e < NC * NC; e += kThreads) {
            const int cy = e / NC, cx = e - cy * NC;
            uint32_t x = bx + (uint32_t)cx, y = by + (uint32_t)cy, z = key;
            pcg3d(x, y, z);
            sst(kSiteStage, &cg[cy * RL + corner_slot(cx)], corner_data<METHOD>(x, y, z, amp, ampw));
        }
    }
    if (s >= 1 && s - 1 < N) {  // 4. cells of 2 samples
        const OctPlan& op = P.oct[s - 1];
        constexpr int NC = corner_ncx2(1), RL = corner_rowlen2(1);
        static_assert(NC == 33, "33 corners a row: 32 lanes and one extra column");
        const uint32_t bx = op.ox + ((uint32_t)j0x >> 1), by = op.oy + ((uint32_t)j0y >> 1);
        float4* cg = corners + op.coff;
        const float amp = kUnit ? 1.0f : op.amp, ampw = kUnit ? P.grad_w : op.ampw;
        const uint32_t z1 = pcg_lcg(op.key), x1 = pcg_lcg(bx + (uint32_t)lane);
        float4* dst = cg + corner_slot(lane);
#pragma unroll 3
        for (int cy = warp; cy < NC; cy += kThreads / 32) {
            uint32_t x = x1, y = pcg_lcg(by + (uint32_t)cy), z = z1;
            pcg3d_post(x, y, z);
            sst(kSiteStage, &dst[cy * RL], corner_data<METHOD>(x, y, z, amp, ampw));
        }
        if (warp > 0 && lane < 11) {  // column 32: rows 11 (warp - 1) + lane
            const int cy = 11 * (warp - 1) + lane;
            uint32_t x = bx + 32u, y = by + (uint32_t)cy, z = op.key;
            pcg3d(x, y, z);
            sst(kSiteStage, &cg[cy * RL + corner_slot(NC - 1)], corner_data<METHOD>(x, y, z, amp, ampw));
        }
    }
}

// kGen: the field may have generic run octaves (n_generic > 0); kernels of
// fields without them are compiled without that path.
template <int METHOD, int RW, bool kGen = true>
__device__ __forceinline__ void stage_tile(const FieldPlan& P, float4* sm, int j0x, int j0y)
{
    using SH = Shape<RW>;
    constexpr int D = Deg<METHOD>::value, NN = D + 1;
    const int tid = threadIdx.x, s = P.s, nt = n_tile<METHOD>(P), ng = kGen ? n_generic<METHOD>(P) : 0;
    float4* xnode = sm;
    float4* ylut = sm + xnode_words<METHOD, RW>(ng);
    float4* rbase = ylut + ng * 64;
    const int nrb = run_basis_words<METHOD, RW>(P);
    float4* corners = rbase + nrb;
    {  // constant tables, global -> shared (latency hidden by the hashing below)
        const float4* src = reinterpret_cast<const float4*>(&kRunBasis<METHOD, RW>);
        for (int e = tid; e < nrb; e += kThreads)
            sst(kSiteStage, &rbase[e], gld(kSiteConst, src, e, (int)sizeof(RunBasis<METHOD, RW>) / 16));
    }
    for (int e = tid; e < ng * NN * SH::TXN; e += kThreads) {
        const int i = e / (NN * SH::TXN), rem = e - i * (NN * SH::TXN);
        const int q = rem / SH::TXN, tx = rem % SH::TXN;
        const int col = tx * RW + node_col<D, RW>(q);
        sst(kSiteStage, &xnode[e], axis_basis<METHOD>(axis_t((uint32_t)(j0x + col), nt + i, s)));
    }
    for (int e = tid; e < ng * 64; e += kThreads) {  // stored in table order: conflict-free
        const int i = e >> 6, slot = e & 63;
        const int row = (slot % SH::TYN) * SH::RR + slot / SH::TYN;
        sst(kSiteStage, &ylut[e], axis_basis<METHOD>(axis_t((uint32_t)(j0y + row), nt + i, s)));
    }
    if (D <= 4 && nt > 0) {  // weights of the tile nodes, global -> shared (latency hidden by the hashing below)
        constexpr int NW = (int)sizeof(TileWeights<D, RW>) / 16;
        const float4* src = reinterpret_cast<const float4*>(&kTileWeights<D, RW>);
        float4* dst = corners + P.ncorner + NN * TileWeights<D, RW>::LW / 4;
        for (int e = tid; e < NW; e += kThreads) sst(kSiteStage, &dst[e], gld(kSiteConst, src, e, NW));
    }
    stage_corners<METHOD>(P, corners, j0x, j0y);
}

// Corner s of a row of a staged octave's block (slot `at` of the block's
// nslots slots, checked in the debug build).
__device__ __forceinline__ float4 corner_at(const float4* __restrict__ row, int s, int at, int nslots)
{
    if (!bounds_ok(kSiteCorner, at, nslots)) return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    return sld(kSiteCorner, &row[s]);
}

__device__ __forceinline__ Cell load_cell(const float4* __restrict__ cg, int rowlen, int lcx, int lcy, int nslots)
{
    const float4* row0 = cg + lcy * rowlen;
    const float4* row1 = row0 + rowlen;
    const int s0 = corner_slot(lcx), s1 = corner_slot(lcx + 1);
    Cell c;
    c.c00 = corner_at(row0, s0, lcy * rowlen + s0, nslots);
    c.c10 = corner_at(row0, s1, lcy * rowlen + s1, nslots);
    c.c01 = corner_at(row1, s0, (lcy + 1) * rowlen + s0, nslots);
    c.c11 = corner_at(row1, s1, (lcy + 1) * rowlen + s1, nslots);
    return c;
}

// A run octave: node columns only.  A collapsed row's V0 term is the same at
// every node, so it is summed once per row (vacc) and the nodes take the rest.
// i = octave, ti = its slot in the basis tables (i minus the tile octaves).
template <int METHOD, int RW>
__device__ __forceinline__ void run_octave(float (&nacc)[n_rows<METHOD, RW>()][Deg<METHOD>::value + 1],
                                           float (&vacc)[n_rows<METHOD, RW>()],
                                           const float4* __restrict__ sm, const float4* __restrict__ corners,
                                           const FieldPlan& P, int i, int ti, int tx, int ty, int ng, int par)
{
    using SH = Shape<RW>;
    constexpr int NN = Deg<METHOD>::value + 1, NRW = n_rows<METHOD, RW>();
    const OctPlan& op = P.oct[i];
    const float4* ylut = sm + xnode_words<METHOD, RW>(ng);
    const float4* cg = corners + op.coff;
    const Cell c = load_cell(cg, op.rowlen, (tx * RW) >> op.k, (ty * SH::RR) >> op.k, op.rowlen * op.ncy);
    float4 xb[NN];
#pragma unroll
    for (int q = 0; q < NN; ++q) xb[q] = sld(kSiteTable, &sm[(ti * NN + q) * SH::TXN + tx]);
#pragma unroll
    for (int r = 0; r < NRW; ++r) {
        const float4 yb = sld(kSiteTable, &ylut[ti * 64 + eval_row<METHOD, RW>(r, par) * SH::TYN + ty]);
        const Row R = Model<METHOD>::row(c, yb);
        vacc[r] += R.V0;
#pragma unroll
        for (int q = 0; q < NN; ++q) nacc[r][q] = Model<METHOD>::eval_add(R, xb[q], nacc[r][q]);
    }
}

// A run octave with cells of 2^K samples, RW <= 2^K <= 64: the same work as
// run_octave, with the corner block, its row length and the cell index
// shifts known at compile time and the bases read from the constant tables.
template <int METHOD, int RW, int K>
__device__ __forceinline__ void run_octave_k(float (&nacc)[n_rows<METHOD, RW>()][Deg<METHOD>::value + 1],
                                             float (&vacc)[n_rows<METHOD, RW>()],
                                             const float4* __restrict__ fine, const float4* __restrict__ rb,
                                             int tx, int ty, int par)
{
    using SH = Shape<RW>;
    using RB = RunBasis<METHOD, RW>;
    constexpr int NN = Deg<METHOD>::value + 1, NXK = (1 << K) / RW, NRW = n_rows<METHOD, RW>();
    const Cell c = load_cell(fine + fine_off2(K), corner_rowlen2(K), (tx * RW) >> K, (ty * SH::RR) >> K, corner_size2(K));
    const float4* tb = shared_run_basis<METHOD>() ? rb : reinterpret_cast<const float4*>(&kRunBasis<METHOD, RW>);
    const float4* xt = tb + RB::xoff(K) + (tx & (NXK - 1));
    const float4* yt = tb + RB::NX + RB::yoff(K);
    float4 xb[NN];
#pragma unroll
    for (int q = 0; q < NN; ++q)
        xb[q] = !bounds_ok(kSiteConst, RB::xoff(K) + (tx & (NXK - 1)) + q * NXK, RB::NX) ? make_float4(0.f, 0.f, 0.f, 0.f)
                : shared_run_basis<METHOD>() ? sld(kSiteTable, &xt[q * NXK]) : __ldg(xt + q * NXK);
#pragma unroll
    for (int r = 0; r < NRW; ++r) {
        // (ty RR) mod 2^K is a multiple of RR, so the row adds without a carry
        const float4* yp = yt + ((ty * SH::RR) & ((1 << K) - 1)) + eval_row<METHOD, RW>(r, par);
        const float4 yb = !bounds_ok(kSiteConst, (int)(yp - tb), RB::NX + RB::NY) ? make_float4(0.f, 0.f, 0.f, 0.f)
                          : shared_run_basis<METHOD>() ? sld(kSiteTable, yp) : __ldg(yp);
        const Row R = Model<METHOD>::row(c, yb);
        vacc[r] += R.V0;
#pragma unroll
        for (int q = 0; q < NN; ++q) nacc[r][q] = Model<METHOD>::eval_add(R, xb[q], nacc[r][q]);
    }
}

template <int METHOD, int RW, int K>
__device__ __forceinline__ void run_fine(float (&nacc)[n_rows<METHOD, RW>()][Deg<METHOD>::value + 1],
                                         float (&vacc)[n_rows<METHOD, RW>()], const float4* __restrict__ fine,
                                         const float4* __restrict__ rb, int s, int N, int nt, int tx, int ty, int par)
{
    if constexpr (K >= Shape<RW>::LOG) {
        const int i = s - K;  // the octave with cells of 2^K samples, if it is a run octave of this field
        if (i >= nt && i >= 0 && i < N) run_octave_k<METHOD, RW, K>(nacc, vacc, fine, rb, tx, ty, par);
    }
}

// Cells of CW = 8, 4 or 2 samples (CW < RW): the in-cell position of column c
// is (c mod CW) / CW, a constant.  Row positions are constants too when a
// thread's rows cover whole cells (RR >= CW); otherwise (RR < CW) they depend
// on the thread's row and the row basis is evaluated once per octave.  Each
// pair of neighbouring columns is added to the sums by one paired add.
template <int METHOD, int RW, int CW>
__device__ __forceinline__ void small_octave(float (&acc)[Shape<RW>::RR][RW], const float4* __restrict__ fine,
                                             int tx, int ty)
{
    using SH = Shape<RW>;
    constexpr int RR = SH::RR, NXC = RW / CW, RPC = RR < CW ? RR : CW, NYC = RR / RPC;
    constexpr int K = CW == 8 ? 3 : (CW == 4 ? 2 : 1);
    constexpr bool kConstRows = RR >= CW;
    const float4* cg = fine + fine_off2(K);
    constexpr float inv = 1.0f / CW;
    float4 yb[RPC];
#pragma unroll
    for (int rr = 0; rr < RPC; ++rr)
        yb[rr] = axis_basis<METHOD>(kConstRows ? rr * inv : (float)(((ty * RR) & (CW - 1)) + rr) * inv);
#pragma unroll
    for (int yq = 0; yq < NYC; ++yq) {
        const int lcy = (ty * RR + yq * RPC) / CW;
#pragma unroll
        for (int xq = 0; xq < NXC; ++xq) {
            const int lcx = (tx * RW + xq * CW) / CW;
            const Cell c = load_cell(cg, corner_rowlen2(K), lcx, lcy, corner_size2(K));
#pragma unroll
            for (int rr = 0; rr < RPC; ++rr) {
                const Row R = (kConstRows && rr == 0) ? Model<METHOD>::row0(c) : Model<METHOD>::row(c, yb[rr]);
#pragma unroll
                for (int q = 0; q < CW; q += 2) {
                    const float h0 = q == 0 ? R.V0 : Model<METHOD>::eval(R, axis_basis<METHOD>(q * inv));
                    const float h1 = Model<METHOD>::eval(R, axis_basis<METHOD>((q + 1) * inv));
                    float& a0 = acc[yq * RPC + rr][xq * CW + q];
                    float& a1 = acc[yq * RPC + rr][xq * CW + q + 1];
                    const float2 a = __fadd2_rn(make_float2(a0, a1), make_float2(h0, h1));
                    a0 = a.x;
                    a1 = a.y;
                }
            }
        }
    }
}

// Tile octaves, CTA part: the sum of octaves 0 .. nt-1 at the (d+1)^2 tile
// nodes, into G[q][r] (row stride LW).  Each node is summed by PARTS lanes,
// octaves dealt round-robin, then added across the lanes with a fixed
// butterfly (the same bits in every lane and on every run).  Degree 3: warp w
// takes tile-node column q = w, lane 4 part + r, so that the 8 lanes of a
// shared-memory load phase read the corners of two octaves (distinct banks);
// otherwise a node's PARTS lanes are consecutive.
template <int METHOD, int RW>
__device__ __forceinline__ void tile_grid(const FieldPlan& P, const float4* __restrict__ corners, float* G,
                                          int j0x, int j0y, int nt)
{
    constexpr int D = Deg<METHOD>::value, NN = D + 1, NG = NN * NN, LW = TileWeights<D, 8>::LW;
    constexpr int PARTS = NG <= 16 ? 8 : (NG <= 32 ? 4 : 2);
    static_assert(NG <= kThreads / PARTS, "one lane group per node");
    const int tid = threadIdx.x;
    const int node = D == 3 ? (tid >> 5) * NN + (tid & 3) : tid / PARTS;
    const int part = D == 3 ? (tid & 31) >> 2 : tid % PARTS;
    const int q = node / NN, r = node - q * NN;
    float v = 0.0f;
    if (node < NG) {
        const uint32_t jx = (uint32_t)(j0x + tile_node<D>(q)), jy = (uint32_t)(j0y + tile_node<D>(r));
        for (int i = part; i < nt; i += PARTS) {
            const OctPlan& op = P.oct[i];
            const Cell c = load_cell(corners + op.coff, op.rowlen, 0, 0, 4);
            const Row R = Model<METHOD>::row(c, axis_basis<METHOD>(axis_t(jy, i, P.s)));
            v += Model<METHOD>::eval(R, axis_basis<METHOD>(axis_t(jx, i, P.s)));
        }
    }
    if constexpr (D == 3) {
#pragma unroll
        for (int o = 16; o >= 4; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    } else {
#pragma unroll
        for (int o = PARTS / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    if constexpr (D == 3) {
        // Warp w holds the tile-node column q = w (node row r = lane mod 4):
        // its lanes carry that column to every tile row y,
        // Tt[q][y] = sum_m ly[y][m] G[q][m], in the order add_tile_grid reads
        // (with node rows, rows 4b + (0, 2, 3, 1) in slots 4b + (0, 1, 2, 3):
        // each thread's two evaluated rows side by side)
        static_assert(NN * PARTS == 32, "one tile-node column a warp");
        float g[NN];
#pragma unroll
        for (int m = 0; m < NN; ++m) g[m] = __shfl_sync(0xffffffffu, v, m);
        const TileWeights<D, RW>& W = *reinterpret_cast<const TileWeights<D, RW>*>(G + NN * LW);
        float* Tt = G + NN * LW + (int)sizeof(TileWeights<D, RW>) / 4;
        const int lane = tid & 31;
#pragma unroll
        for (int h = 0; h < 64 / 32; ++h) {
            const int y = lane + 32 * h;
            const float4 l = sld(kSiteTable, reinterpret_cast<const float4*>(W.ly[y]));
            const int slot = node_rows<METHOD, RW>() ? (y & ~3) | ((0x2130 >> (4 * (y & 3))) & 3) : y;
            sst(kSiteTable, &Tt[q * 64 + slot], fmaf(l.w, g[3], fmaf(l.z, g[2], fmaf(l.y, g[1], l.x * g[0]))));
        }
    } else if (node < NG && part == 0) {
        sst(kSiteTable, &G[q * LW + r], v);
    }
}

// Tile octaves, thread part: the tile polynomial at the thread's rows and
// node columns, added to the node accumulators.  Degree 3 reads its rows from
// the row table; otherwise each thread carries the tile nodes to its rows.
template <int METHOD, int RW>
__device__ __forceinline__ void add_tile_grid(float (&nacc)[n_rows<METHOD, RW>()][Deg<METHOD>::value + 1],
                                              const float* __restrict__ G, int tx, int ty, int par)
{
    using SH = Shape<RW>;
    constexpr int D = Deg<METHOD>::value, NN = D + 1, LW = TileWeights<D, RW>::LW, NRW = n_rows<METHOD, RW>();
    const TileWeights<D, RW>& W = *reinterpret_cast<const TileWeights<D, RW>*>(G + NN * LW);
    float Rq[NRW][NN];  // tile polynomial at the thread's evaluated rows, tile columns q
    if constexpr (D == 3) {
        const float* Tt = G + NN * LW + (int)sizeof(TileWeights<D, RW>) / 4;
#pragma unroll
        for (int q = 0; q < NN; ++q) {
            if constexpr (node_rows<METHOD, RW>()) {
                const float2 t = sld(kSiteTable, reinterpret_cast<const float2*>(Tt + q * 64 + ty * 4 + 2 * par));
                Rq[0][q] = t.x;
                Rq[1][q] = t.y;
            } else if constexpr (SH::RR == 4) {
                const float4 t = sld(kSiteTable, reinterpret_cast<const float4*>(Tt + q * 64 + ty * 4));
                Rq[0][q] = t.x;
                Rq[1][q] = t.y;
                Rq[2][q] = t.z;
                Rq[3][q] = t.w;
            } else {
                const float2 t = sld(kSiteTable, reinterpret_cast<const float2*>(Tt + q * 64 + ty * 2));
                Rq[0][q] = t.x;
                Rq[1][q] = t.y;
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < SH::RR; ++r) {
            const float* ly = W.ly[ty * SH::RR + r];
            float w[NN];
#pragma unroll
            for (int m = 0; m < NN; ++m) w[m] = sld(kSiteTable, &ly[m]);
#pragma unroll
            for (int q = 0; q < NN; ++q) {
                float a = 0.0f;
#pragma unroll
                for (int m = 0; m < NN; ++m) a = fmaf(w[m], sld(kSiteTable, &G[q * LW + m]), a);
                Rq[r][q] = a;
            }
        }
    }
#pragma unroll
    for (int n = 0; n < NN; ++n) {
        const float* lx = W.lx[n][tx];
        float w[NN];
#pragma unroll
        for (int q = 0; q < NN; ++q) w[q] = sld(kSiteTable, &lx[q]);
#pragma unroll
        for (int r = 0; r < NRW; ++r)
#pragma unroll
            for (int q = 0; q < NN; ++q) nacc[r][n] = fmaf(w[q], Rq[r][q], nacc[r][n]);
    }
}

// One lattice octave: every sample sits on a lattice point.  Each adds
// amp unit_mant(h) = amp (unit_value(h) + 3): the -3 amp terms of all lattice
// octaves (FieldPlan::lat_bias) start the rows' sums in fbm2d_tile instead.
// Neighbouring columns share one paired FMA (two FP32 FMAs in one
// instruction, each rounded as fmaf).
template <int RW>
__device__ __forceinline__ void lattice_octave(float (&acc)[Shape<RW>::RR][RW], const OctPlan& op, uint32_t jx,
                                               uint32_t jy)
{
    const int sh = op.k;
    const uint32_t z1 = pcg_lcg(op.key), dx = 1664525u << sh;  // x's LCG step advances by dx a column
    const uint32_t x0 = op.ox + (jx << sh);
    const float2 amp2 = make_float2(op.amp, op.amp);
#pragma unroll
    for (int r = 0; r < Shape<RW>::RR; ++r) {
        const uint32_t y1 = pcg_lcg(op.oy + ((jy + r) << sh));
        const uint32_t base = pcg3d_run_base(x0, y1, z1);
#pragma unroll
        for (int c = 0; c < RW; c += 2) {
            const uint32_t h0 = pcg3d_run_value(base + (uint32_t)c * dx, y1, z1);
            const uint32_t h1 = pcg3d_run_value(base + (uint32_t)(c + 1) * dx, y1, z1);
            const float2 a = __ffma2_rn(make_float2(unit_mant(h0), unit_mant(h1)), amp2,
                                        make_float2(acc[r][c], acc[r][c + 1]));
            acc[r][c] = a.x;
            acc[r][c + 1] = a.y;
        }
    }
}

// Elements [x, x + n) of row y lie inside the W x H output (checked in the
// debug build only).
__device__ __forceinline__ bool out_ok(const FieldPlan& P, int x, int y, int n)
{
    return bounds_ok(kSiteStore, x + n - 1, P.W) && bounds_ok(kSiteStore, (long long)y * P.W + x, (long long)P.W * P.H);
}

template <typename OutT, int RW>
__device__ __forceinline__ void store_tile_as(const FieldPlan& P, const float (&acc)[Shape<RW>::RR][RW], int x0, int y0)
{
    OutT* out = reinterpret_cast<OutT*>(P.out);
    if (P.vec_ok && x0 + RW <= P.W && y0 + Shape<RW>::RR <= P.H) {  // whole run inside: vector stores only
        OutT* row = out + (size_t)y0 * (size_t)P.W + x0;
#pragma unroll
        for (int r = 0; r < Shape<RW>::RR; ++r, row += P.W) {
            if (sizeof(OutT) == 4) {
                float4* p = reinterpret_cast<float4*>(row);
#pragma unroll
                for (int v = 0; v < RW / 4; ++v)
                    if (out_ok(P, x0 + 4 * v, y0 + r, 4))
                        p[v] = make_float4(acc[r][4 * v], acc[r][4 * v + 1], acc[r][4 * v + 2], acc[r][4 * v + 3]);
            } else {
                uint4* p = reinterpret_cast<uint4*>(row);
#pragma unroll
                for (int v = 0; v < RW / 8; ++v) {
                    __half2 h[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        h[q] = __floats2half2_rn(acc[r][8 * v + 2 * q], acc[r][8 * v + 2 * q + 1]);
                    if (out_ok(P, x0 + 8 * v, y0 + r, 8)) p[v] = *reinterpret_cast<const uint4*>(h);
                }
            }
        }
        return;
    }
#pragma unroll
    for (int r = 0; r < Shape<RW>::RR; ++r) {
        const int y = y0 + r;
        if (y >= P.H) break;
        OutT* row = out + (size_t)y * (size_t)P.W;
        if (P.vec_ok && x0 + RW <= P.W) {
            if (sizeof(OutT) == 4) {
                float4* p = reinterpret_cast<float4*>(row + x0);
#pragma unroll
                for (int v = 0; v < RW / 4; ++v)
                    if (out_ok(P, x0 + 4 * v, y, 4))
                        p[v] = make_float4(acc[r][4 * v], acc[r][4 * v + 1], acc[r][4 * v + 2], acc[r][4 * v + 3]);
            } else {
                uint4* p = reinterpret_cast<uint4*>(row + x0);
#pragma unroll
                for (int v = 0; v < RW / 8; ++v) {
                    __half2 h[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        h[q] = __floats2half2_rn(acc[r][8 * v + 2 * q], acc[r][8 * v + 2 * q + 1]);
                    if (out_ok(P, x0 + 8 * v, y, 8)) p[v] = *reinterpret_cast<const uint4*>(h);
                }
            }
        } else {
#pragma unroll
            for (int c = 0; c < RW; ++c)
                if (x0 + c < P.W && out_ok(P, x0 + c, y, 1)) store1(row + x0 + c, acc[r][c]);
        }
    }
}

template <int RW>
__device__ __forceinline__ void store_tile(const FieldPlan& P, const float (&acc)[Shape<RW>::RR][RW], int x0, int y0)
{
    if (P.dtype == 1) store_tile_as<__half, RW>(P, acc, x0, y0);
    else store_tile_as<float, RW>(P, acc, x0, y0);
}

// Whole tile: stage, evaluate all octaves, store.
template <int METHOD, int RW, bool kGen = true>
__device__ __forceinline__ void fbm2d_tile(const FieldPlan& P, float4* sm, int bx, int by)
{
    using SH = Shape<RW>;
    constexpr int D = Deg<METHOD>::value, NN = D + 1, RR = SH::RR;
    const int tid = threadIdx.x, tx = tid % SH::TXN, ty = tid / SH::TXN;
    const int x0 = bx * kTW, y0 = by * kTH;        // output tile origin
    const int j0x = x0 + P.jx0, j0y = y0 + P.jy0;  // sample indices
    const int s = P.s, N = P.N, nt = n_tile<METHOD>(P), ng = kGen ? n_generic<METHOD>(P) : 0;
    stage_tile<METHOD, RW, kGen>(P, sm, j0x, j0y);
    __syncthreads();

    // tile octaves: their sum at the tile nodes (read back after the barrier below)
    const float4* rb = sm + xnode_words<METHOD, RW>(ng) + ng * 64;
    const float4* corners = rb + run_basis_words<METHOD, RW>(P);
    const float4* fine = corners + 4 * n_coarse(P);  // corner blocks of the octaves with cells <= 64 samples
    float* G = reinterpret_cast<float*>(const_cast<float4*>(corners) + P.ncorner);
    if (Deg<METHOD>::value <= 4 && nt > 0) tile_grid<METHOD, RW>(P, corners, G, j0x, j0y, nt);

    // run octaves: node columns, then interpolate the other columns once
    constexpr bool kPerlin = METHOD == kPerlinS5 || METHOD == kPerlinS3;
    constexpr int NRW = n_rows<METHOD, RW>();
    const int par = node_rows<METHOD, RW>() ? (ty & 1) : 0;
    float nacc[NRW][NN], vacc[NRW];
#pragma unroll
    for (int r = 0; r < NRW; ++r) {
        vacc[r] = 0.0f;
#pragma unroll
        for (int q = 0; q < NN; ++q) nacc[r][q] = 0.0f;
    }
    for (int i = 0; i < ng; ++i) run_octave<METHOD, RW>(nacc, vacc, sm, corners, P, nt + i, i, tx, ty, ng, par);
    run_fine<METHOD, RW, 6>(nacc, vacc, fine, rb, s, N, nt, tx, ty, par);
    run_fine<METHOD, RW, 5>(nacc, vacc, fine, rb, s, N, nt, tx, ty, par);
    run_fine<METHOD, RW, 4>(nacc, vacc, fine, rb, s, N, nt, tx, ty, par);
    run_fine<METHOD, RW, 3>(nacc, vacc, fine, rb, s, N, nt, tx, ty, par);
#pragma unroll
    for (int r = 0; r < NRW; ++r)
#pragma unroll
        for (int q = 0; q < NN; ++q) nacc[r][q] += vacc[r];
    if (Deg<METHOD>::value <= 4 && nt > 0) {  // uniform over the CTA
        __syncthreads();
        add_tile_grid<METHOD, RW>(nacc, G, tx, ty, par);
    }
    // the run and tile octaves' sum at the node columns of all RR rows
    float rowv[RR][NN];
    if constexpr (!node_rows<METHOD, RW>()) {
#pragma unroll
        for (int r = 0; r < RR; ++r)
#pragma unroll
            for (int q = 0; q < NN; ++q) rowv[r][q] = nacc[r][q];
    } else {
        // Mirrored block rows (even thread: y; odd thread: 7 - y): own nodes
        // at 0, 2, the partner's at 5, 7; rows 1 and 3 interpolated with the
        // node columns' Lagrange weights (nodes at 0, 2, 5, 7).
#pragma unroll
        for (int q = 0; q < NN; ++q) {
            const float p5 = __shfl_xor_sync(0xffffffffu, nacc[1][q], 8);
            const float p7 = __shfl_xor_sync(0xffffffffu, nacc[0][q], 8);
            float v[4];
            v[0] = nacc[0][q];
            v[2] = nacc[1][q];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int y = 2 * j + 1;
                v[y] = fmaf(lagrange<3, 8>(y, 3), p7, fmaf(lagrange<3, 8>(y, 2), p5,
                           fmaf(lagrange<3, 8>(y, 1), v[2], lagrange<3, 8>(y, 0) * v[0])));
            }
#pragma unroll
            for (int r = 0; r < RR; ++r) rowv[r][q] = par ? v[RR - 1 - r] : v[r];
        }
    }
    // The -3 amp offsets of all lattice octaves (FieldPlan::lat_bias) start
    // every sample's sum: added to the node columns, and the first term of the
    // others' interpolation (so a field of lattice octaves alone is exact).
    const float lat = (!kPerlin && s < N) ? P.lat_bias : 0.0f;
    float acc[RR][RW];
#pragma unroll
    for (int r = 0; r < RR; ++r)
#pragma unroll
        for (int c = 0; c < RW; ++c) {
            const int q = node_of_col<D, RW>(c);
            if (q >= 0) {
                acc[r][c] = rowv[r][q] + lat;
            } else {
                float v = lat;
#pragma unroll
                for (int m = 0; m < NN; ++m) v = fmaf(lagrange<D, RW>(c, m), rowv[r][m], v);
                acc[r][c] = v;
            }
        }

    // cells narrower than the run (8, 4 and 2 samples), then lattice octaves
    if (RW == 16 && s >= 3 && s - 3 < N) small_octave<METHOD, RW, (RW == 16 ? 8 : 4)>(acc, fine, tx, ty);
    if (s >= 2 && s - 2 < N) small_octave<METHOD, RW, 4>(acc, fine, tx, ty);
    if (s >= 1 && s - 1 < N) small_octave<METHOD, RW, 2>(acc, fine, tx, ty);
    if (!kPerlin && s < N) {
        for (int i = s; i < N; ++i)
            lattice_octave<RW>(acc, P.oct[i], (uint32_t)(j0x + tx * RW), (uint32_t)(j0y + ty * RR));
    }
    store_tile<RW>(P, acc, x0 + tx * RW, y0 + ty * RR);
}

// At least five CTAs a SM for Perlin S5 (up to 102 registers), so that its
// degree-6 node accumulators are not squeezed into spills; the other models
// are left to the compiler's own choice (70-96 registers).
template <int METHOD>
constexpr int min_ctas() { return METHOD == kPerlinS5 ? 5 : 0; }

template <int METHOD, int RW, bool kGen>
__global__ void __launch_bounds__(kThreads, min_ctas<METHOD>()) fbm2d_kernel(const __grid_constant__ FieldPlan P)
{
    extern __shared__ float4 sm[];
    fbm2d_tile<METHOD, RW, kGen>(P, sm, blockIdx.x, blockIdx.y);
}

// One tile of a batch field, as a call (not inlined) so that the batch
// kernel's registers are those of its largest path, not of all paths at once.
template <int METHOD>
__device__ __noinline__ void batch_tile(const FieldPlan& P, float4* sm, int bx, int by)
{
    if (P.rw == 16) fbm2d_tile<METHOD, 16>(P, sm, bx, by);
    else fbm2d_tile<METHOD, 8>(P, sm, bx, by);
}

// ---------------------------------------------------------------------------
// Ridged multifractal (PTG_RIDGED), fused 2D form.  The octaves interact:
// octave i adds p^i r_i with r_i = (1 - |h_i|)^2 w_i, h_i the unit-amplitude
// octave and w_{i+1} = clamp(2 r_i, 0, 1), so every octave is evaluated at
// every sample, in octave order, instead of being summed at nodes first.
// The staging is the fBm kernel's corner staging at unit amplitude, plus
// per-CTA tables of the x- and y-bases of the octaves whose cells are at
// least 8 samples wide (one cell a thread); 4- and 2-sample cells take
// constant in-cell positions and lattice octaves one hash word a sample.
// Thread shape 8 x 4.
// ---------------------------------------------------------------------------

// Octaves with cells of 8 samples or more (their basis tables come first in
// shared memory: 64 x-bases, then 64 y-bases an octave).
__host__ __device__ __forceinline__ int n_ridge_tables(const FieldPlan& P)
{
    const int n = P.s - 2;
    return n < 0 ? 0 : (n < P.N ? n : P.N);
}

// Table slot of tile column j's x-basis: groups of 8 rotated, so that the 8
// threads of a quarter warp (runs 8 tx .. 8 tx + 7, one column each) read 8
// bank groups.
__device__ __forceinline__ int ridge_xslot(int j) { return j ^ ((j >> 3) & 7); }

// One octave at two neighbouring samples: each sum gains wgt (1 - |h|)^2 w,
// and each weight becomes that ridge doubled, clamped to [0, 1]; the products
// and the sums as paired FP32 instructions (each half rounded as the scalar
// operation).
__device__ __forceinline__ void ridge2(float& acc0, float& acc1, float& w0, float& w1, float h0, float h1, float wgt)
{
    const float2 a = make_float2(1.0f - fabsf(h0), 1.0f - fabsf(h1));
    const float2 r = __fmul2_rn(__fmul2_rn(a, a), make_float2(w0, w1));
    const float2 ac = __ffma2_rn(make_float2(wgt, wgt), r, make_float2(acc0, acc1));
    acc0 = ac.x;
    acc1 = ac.y;
    w0 = __saturatef(2.0f * r.x);
    w1 = __saturatef(2.0f * r.y);
}

// Cells of CW = 4 or 2 samples (a thread's 4 rows cover whole cells): the
// in-cell positions are constants, as in small_octave.
template <int METHOD, int CW>
__device__ __forceinline__ void small_ridged(float (&acc)[4][8], float (&w)[4][8], const float4* __restrict__ fine,
                                             int tx, int ty, float wgt)
{
    constexpr int K = CW == 4 ? 2 : 1, NXC = 8 / CW, NYC = 4 / CW;
    constexpr float inv = 1.0f / CW;
    const float4* cg = fine + fine_off2(K);
#pragma unroll
    for (int yq = 0; yq < NYC; ++yq) {
#pragma unroll
        for (int xq = 0; xq < NXC; ++xq) {
            const Cell c = load_cell(cg, corner_rowlen2(K), tx * NXC + xq, ty * NYC + yq, corner_size2(K));
#pragma unroll
            for (int rr = 0; rr < CW; ++rr) {
                const Row R = rr == 0 ? Model<METHOD>::row0(c) : Model<METHOD>::row(c, axis_basis<METHOD>(rr * inv));
#pragma unroll
                for (int q = 0; q < CW; q += 2) {
                    const float h0 = q == 0 ? R.V0 : Model<METHOD>::eval(R, axis_basis<METHOD>(q * inv));
                    const float h1 = Model<METHOD>::eval(R, axis_basis<METHOD>((q + 1) * inv));
                    const int y = yq * CW + rr, x = xq * CW + q;
                    ridge2(acc[y][x], acc[y][x + 1], w[y][x], w[y][x + 1], h0, h1, wgt);
                }
            }
        }
    }
}

// A lattice octave: h is the corner value, unit_value of pcg3d word 0 (zero
// for Perlin), with the row-invariant words hoisted as in lattice_octave.
template <int METHOD>
__device__ __forceinline__ void lattice_ridged(float (&acc)[4][8], float (&w)[4][8], const OctPlan& op, uint32_t jx,
                                               uint32_t jy)
{
    const float wgt = op.amp;
    if constexpr (METHOD == kPerlinS5 || METHOD == kPerlinS3) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 8; c += 2) ridge2(acc[r][c], acc[r][c + 1], w[r][c], w[r][c + 1], 0.0f, 0.0f, wgt);
    } else {
        const int sh = op.k;
        const uint32_t z1 = pcg_lcg(op.key), dx = 1664525u << sh, x0 = op.ox + (jx << sh);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint32_t y1 = pcg_lcg(op.oy + ((jy + r) << sh));
            const uint32_t base = pcg3d_run_base(x0, y1, z1);
#pragma unroll
            for (int c = 0; c < 8; c += 2)
                ridge2(acc[r][c], acc[r][c + 1], w[r][c], w[r][c + 1],
                       unit_value(pcg3d_run_value(base + (uint32_t)c * dx, y1, z1)),
                       unit_value(pcg3d_run_value(base + (uint32_t)(c + 1) * dx, y1, z1)), wgt);
        }
    }
}

template <int METHOD>
__device__ __forceinline__ void ridged_tile(const FieldPlan& P, float4* sm, int bx, int by)
{
    using SH = Shape<8>;
    const int tid = threadIdx.x, tx = tid % SH::TXN, ty = tid / SH::TXN;
    const int x0 = bx * kTW, y0 = by * kTH, j0x = x0 + P.jx0, j0y = y0 + P.jy0;
    const int s = P.s, N = P.N, nb = n_ridge_tables(P);
    for (int e = tid; e < nb * 128; e += kThreads) {  // x- and y-bases of the octaves with cells >= 8
        const int i = e >> 7, a = (e >> 6) & 1, j = e & 63;
        const float4 b = axis_basis<METHOD>(axis_t((uint32_t)((a ? j0y : j0x) + j), i, s));
        sst(kSiteStage, &sm[i * 128 + (a ? 64 + j : ridge_xslot(j))], b);
    }
    float4* corners = sm + nb * 128;
    stage_corners<METHOD, true>(P, corners, j0x, j0y);
    __syncthreads();

    float acc[4][8], w[4][8];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            acc[r][c] = 0.0f;
            w[r][c] = 1.0f;
        }
    for (int i = 0; i < nb; ++i) {  // one cell a thread; octaves in order (the weights chain)
        const OctPlan& op = P.oct[i];
        const Cell c = load_cell(corners + op.coff, op.rowlen, (tx * 8) >> op.k, (ty * 4) >> op.k,
                                 op.rowlen * op.ncy);
        const float4* xt = sm + i * 128;
        const float wgt = op.amp;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const Row R = Model<METHOD>::row(c, sld(kSiteTable, &xt[64 + ty * 4 + r]));
#pragma unroll
            for (int q = 0; q < 8; q += 2)
                ridge2(acc[r][q], acc[r][q + 1], w[r][q], w[r][q + 1],
                       Model<METHOD>::eval(R, sld(kSiteTable, &xt[ridge_xslot(tx * 8 + q)])),
                       Model<METHOD>::eval(R, sld(kSiteTable, &xt[ridge_xslot(tx * 8 + q + 1)])), wgt);
        }
    }
    const float4* fine = corners + 4 * n_coarse(P);
    if (s >= 2 && s - 2 < N) small_ridged<METHOD, 4>(acc, w, fine, tx, ty, P.oct[s - 2].amp);
    if (s >= 1 && s - 1 < N) small_ridged<METHOD, 2>(acc, w, fine, tx, ty, P.oct[s - 1].amp);
    for (int i = s; i < N; ++i) lattice_ridged<METHOD>(acc, w, P.oct[i], (uint32_t)(j0x + tx * 8), (uint32_t)(j0y + ty * 4));
    store_tile<8>(P, acc, x0 + tx * 8, y0 + ty * 4);
}

// Bounded to four CTAs a SM (128 registers; the compiler's own choice is 139,
// three CTAs): on the 8192^2, 12-octave field C1 0.9%, C2 1.2% and Perlin S5
// 3.7% faster, zero-gradient unchanged, with a 4-byte spill.  Five CTAs (96
// registers) spill 100 bytes and are 3-4% slower.
template <int METHOD>
__global__ void __launch_bounds__(kThreads, 4) fbm2d_ridged_kernel(const __grid_constant__ FieldPlan P)
{
    extern __shared__ float4 sm[];
    ridged_tile<METHOD>(P, sm, blockIdx.x, blockIdx.y);
}

// Persistent batched generator: resident CTAs pull tiles of many fields from
// one work counter.  Field f owns tiles [tile_start[f], tile_start[f+1]); its
// plan is copied to shared memory when a CTA moves to it.  Every tile runs the
// same code as the single-field kernel, so results are identical.
//
// Bounded to 80 registers (six CTAs a SM): the tile calls would take 96, the
// largest path's allocation, and five CTAs.  By measurement on GB300 (the
// 4096-chunk batch, C1/C2 50/50) the bound is 7.5% faster, with no spill
// beyond 4 bytes in the C1 path; 72 registers (seven CTAs) gained 0.7% more
// but spilled 124 bytes in the C2 path.
__global__ void __launch_bounds__(kThreads, 6) fbm2d_batch_kernel(const FieldPlan* __restrict__ plans,
                                                               const long long* __restrict__ tile_start, int n,
                                                               unsigned long long* __restrict__ counter, int group)
{
    extern __shared__ float4 sm[];
    __shared__ FieldPlan plan;
    __shared__ long long s_tile;
    __shared__ int s_field;
    const long long total = bounds_ok(kSitePlan, n, (long long)n + 1) ? tile_start[n] : 0;
    // The counter hands out groups of `group` consecutive tiles (1, 2 or 4,
    // chosen by the launch from the tiles per resident CTA): the tiles of a
    // group mostly share a field, so its search, plan copy and barrier are
    // paid once a group.
    const long long ngroups = (total + group - 1) / group;
    const int lane = threadIdx.x & 31;
    // Lane 0 of warp 0 holds the group taken for the next round: the atomic
    // for it is issued as soon as the current group is known, so that its
    // latency passes while the group is computed.
    long long next = 0;
    if (threadIdx.x == 0) next = (long long)atomicAdd(counter, 1ULL);
    int cur = -1;
    for (;;) {
        if (threadIdx.x < 32) {
            const long long g = __shfl_sync(0xffffffffu, next, 0);
            const long long t = g < ngroups ? g * group : total;
            if (t < total) {
                // Last field whose first tile is <= t, by warp 0 together:
                // each round the 32 lanes test 32 evenly spaced fields of the
                // range [lo, hi] and the range shrinks to the gap after the
                // last field that passes (tile_start is non-decreasing and
                // tile_start[lo] <= t throughout, so lane 0 always passes).
                // 4096 fields take 3 rounds of loads instead of 12.
                int lo = 0, hi = n - 1;
                while (lo < hi) {
                    const int step = (hi - lo + 32) >> 5;
                    const int idx = lo + lane * step;
                    const bool ok = idx <= hi && bounds_ok(kSitePlan, idx, (long long)n + 1) && tile_start[idx] <= t;
                    const unsigned m = __ballot_sync(0xffffffffu, ok);
                    lo += (31 - __clz(m | 1u)) * step;
                    hi = min(hi, lo + step - 1);
                }
                if (lane == 0) {
                    s_field = lo;
                    next = (long long)atomicAdd(counter, 1ULL);
                }
            }
            if (lane == 0) s_tile = t;
        }
        __syncthreads();
        const long long t0 = s_tile;
        if (t0 >= total) break;
        int f = s_field;
        const long long t1 = t0 + group < total ? t0 + group : total;
        for (long long t = t0; t < t1; ++t) {
            if (t > t0)  // later tiles of the group: the next field(s) where they start
                while (f + 1 < n && tile_start[f + 1] <= t) ++f;
            if (f != cur && bounds_ok(kSitePlan, f, n)) {
                const int4* src = reinterpret_cast<const int4*>(plans + f);
                int4* dst = reinterpret_cast<int4*>(&plan);
                for (int q = threadIdx.x; q < (int)(sizeof(FieldPlan) / 16); q += kThreads) dst[q] = src[q];
                cur = f;
                __syncthreads();
            }
            const long long local = t - (bounds_ok(kSitePlan, f, (long long)n + 1) ? tile_start[f] : t);
            const int bx = (int)(local % plan.tiles_x), by = (int)(local / plan.tiles_x);
            switch (plan.method) {  // the polynomial models (batches are ptg_field calls)
            case kC1: batch_tile<kC1>(plan, sm, bx, by); break;
            case kC2: batch_tile<kC2>(plan, sm, bx, by); break;
            case kPaperGauge: batch_tile<kPaperGauge>(plan, sm, bx, by); break;
            default: batch_tile<kZeroGrad>(plan, sm, bx, by); break;
            }
            __syncthreads();
        }
    }
}

template <int METHOD>
size_t smem_words(const FieldPlan& P)
{
    if (P.ridged) return (size_t)n_ridge_tables(P) * 128 + (size_t)P.ncorner;
    const int nt = n_tile<METHOD>(P), ng = n_generic<METHOD>(P);
    const size_t grid = nt > 0 ? (size_t)(P.rw == 16 ? grid_words<METHOD, 16>() : grid_words<METHOD, 8>()) : 0;
    const size_t xw = P.rw == 16 ? (size_t)xnode_words<METHOD, 16>(ng) : (size_t)xnode_words<METHOD, 8>(ng);
    const size_t rbw = P.rw == 16 ? run_basis_words<METHOD, 16>(P) : run_basis_words<METHOD, 8>(P);
    return xw + (size_t)ng * 64 + rbw + (size_t)P.ncorner + grid;
}

}  // namespace

size_t fbm2d_smem_bytes(const FieldPlan& P)
{
    size_t w = 0;
    switch (P.method) {
    case kC1: w = smem_words<kC1>(P); break;
    case kC2: w = smem_words<kC2>(P); break;
    case kPaperGauge: w = smem_words<kPaperGauge>(P); break;
    case kZeroGrad: w = smem_words<kZeroGrad>(P); break;
    case kPerlinS5: w = smem_words<kPerlinS5>(P); break;
    default: w = smem_words<kPerlinS3>(P); break;
    }
    return sizeof(float4) * w;
}

cudaError_t launch_fbm2d(const FieldPlan& P, int method, int /*s*/, cudaStream_t stream)
{
    const dim3 grid(P.tiles_x, P.tiles_y, 1);
    const size_t smem = fbm2d_smem_bytes(P);
#define PTG_LAUNCH2D_RW(M, RW)                                                                       \
    do {                                                                                             \
        auto kfn = n_generic<M>(P) > 0 ? fbm2d_kernel<M, RW, true> : fbm2d_kernel<M, RW, false>;      \
        cudaError_t e = set_kernel_smem((const void*)kfn, smem);                                     \
        if (e != cudaSuccess) return e;                                                              \
        kfn<<<grid, kThreads, smem, stream>>>(P);                                                    \
        return cudaGetLastError();                                                                   \
    } while (0)
#define PTG_LAUNCH2D(M)                                                                              \
    do {                                                                                             \
        if (P.ridged) {                                                                              \
            auto kfr = fbm2d_ridged_kernel<M>;                                                       \
            cudaError_t e = set_kernel_smem((const void*)kfr, smem);                                 \
            if (e != cudaSuccess) return e;                                                          \
            kfr<<<grid, kThreads, smem, stream>>>(P);                                                \
            return cudaGetLastError();                                                               \
        }                                                                                            \
        if (P.rw == 16) PTG_LAUNCH2D_RW(M, 16);                                                      \
        PTG_LAUNCH2D_RW(M, 8);                                                                       \
    } while (0)
    switch (method) {
    case kC1: PTG_LAUNCH2D(kC1);
    case kC2: PTG_LAUNCH2D(kC2);
    case kPaperGauge: PTG_LAUNCH2D(kPaperGauge);
    case kZeroGrad: PTG_LAUNCH2D(kZeroGrad);
    case kPerlinS5: PTG_LAUNCH2D(kPerlinS5);
    case kPerlinS3: PTG_LAUNCH2D(kPerlinS3);
    default: return cudaErrorInvalidValue;
    }
#undef PTG_LAUNCH2D_RW
#undef PTG_LAUNCH2D
}

// Tiles a CTA takes at a time: 4 from 32 tiles per resident CTA, 2 from 16,
// else 1.  On GB300, groups of 4 make the 4096-chunk batch (206 tiles a CTA)
// 10% faster than single tiles, while 256 chunks (3 tiles a CTA) are 12%
// slower with them (the last groups leave CTAs idle).
static int batch_group(long long total_tiles, int blocks)
{
    return total_tiles >= 32LL * blocks ? 4 : (total_tiles >= 16LL * blocks ? 2 : 1);
}

cudaError_t launch_fbm2d_batch(const FieldPlan* plans, const long long* tile_start, int n,
                               unsigned long long* counter, long long total_tiles, size_t smem, int blocks,
                               cudaStream_t stream)
{
    cudaError_t e = set_kernel_smem((const void*)fbm2d_batch_kernel, smem);
    if (e != cudaSuccess) return e;
    fbm2d_batch_kernel<<<blocks, kThreads, smem, stream>>>(plans, tile_start, n, counter,
                                                           batch_group(total_tiles, blocks));
    return cudaGetLastError();
}

int fbm2d_batch_blocks_per_sm(size_t smem)
{
    int nb = 0;
    set_kernel_smem((const void*)fbm2d_batch_kernel, smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fbm2d_batch_kernel, kThreads, smem) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

}  // namespace ptg
