// ptg_fbm2d.cu -- fused all-octave 2D generator for the polynomial noise of
// Thorimbert & Chopard (arXiv:1610.03525) and for Perlin's polynomial.
//
// One CTA makes a 64 x 64 tile of samples with 128 threads; each thread owns
// 4 rows x 8 consecutive columns and keeps their fractal sums (Sec. 4) in
// registers across all octaves, then writes each sample once.
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
//   spc_i >= 8 ("run8"): a thread's 8-column run lies in one cell, so each of
//     its rows is one polynomial of degree d in the column (d = 3 for C1, 5 for
//     C2, 4 / 6 for Perlin S3 / S5), and so is the sum over all such octaves.
//     The kernel evaluates d + 1 node columns per octave and fills the other
//     columns once, at the end, by exact Lagrange interpolation.
//   spc_i = 4, 2: in-cell positions are the constants q / spc_i; the basis is
//     folded into the code and positions t = 0 take the corner data directly.
//   spc_i <= 1 ("lattice"): every sample is a lattice point, where the cell
//     polynomial equals the corner value: one hash per sample (zero for
//     Perlin, whose value at lattice points is zero).
// Corners of every staged octave (cells >= 2 samples) are hashed once per CTA
// into shared memory, pre-scaled by the octave amplitude (Sec. 4.1's C_init),
// and the per-axis basis of the run8 octaves is tabulated per CTA (the paper's
// precomputed space-only terms, Sec. 5.2).
#include "ptg_device.cuh"
#include "ptg_eval.cuh"
#include "ptg_kernels.h"

namespace ptg {
namespace {

constexpr int kTW = 64, kTH = 64, kThreads = 128;
constexpr int kCols = 8, kRows = 4;  // per thread

// Shared-memory layout (float4 units):
//   x-basis of run8 octaves at node columns [n8][D+1][8 tx],
//   y-basis of run8 octaves [n8][4 rows][16 ty],
//   staged corners of every staged octave (rows swizzled by corner_slot).
template <int METHOD>
__host__ __device__ constexpr int xnode_words(int n8) { return n8 * (Deg<METHOD>::value + 1) * 8; }

__device__ __forceinline__ int n_run8(const FieldPlan& P)
{
    const int n = P.s - 2;
    return n < 0 ? 0 : (n < P.N ? n : P.N);
}

template <int METHOD>
__device__ __forceinline__ void stage_tile(const FieldPlan& P, float4* sm, int j0x, int j0y)
{
    constexpr int NN = Deg<METHOD>::value + 1;
    const int tid = threadIdx.x, s = P.s, n8 = n_run8(P);
    float4* xnode = sm;
    float4* ylut = sm + xnode_words<METHOD>(n8);
    float4* corners = ylut + n8 * 64;
    for (int e = tid; e < n8 * NN * 8; e += kThreads) {
        const int i = e / (NN * 8), rem = e - i * (NN * 8);
        const int q = rem >> 3, tx = rem & 7;
        const int col = tx * 8 + node_col<Deg<METHOD>::value>(q);
        xnode[e] = axis_basis<METHOD>(axis_t((uint32_t)(j0x + col), i, s));
    }
    for (int e = tid; e < n8 * 64; e += kThreads) {  // stored in table order: conflict-free
        const int i = e >> 6, slot = e & 63;
        const int row = (slot & 15) * 4 + (slot >> 4);
        ylut[e] = axis_basis<METHOD>(axis_t((uint32_t)(j0y + row), i, s));
    }
    // Corners, octave by octave (uniform loops: every lane of a warp reads the
    // same octave parameters).  Octaves with at most 32 corners go to one warp
    // each, in turn, so that no warp carries all the small octaves.
    const int warp = tid >> 5, lane = tid & 31;
    int small = 0;
    for (int i = 0; i < P.nst; ++i) {
        const OctPlan& op = P.oct[i];
        const int n = op.ncx * op.ncy;
        int e0 = tid, step = kThreads;
        if (n <= 32) {
            if ((small++ & 3) != warp) continue;
            e0 = lane;
            step = 32;
        }
        const uint32_t bx = op.ox + ((uint32_t)j0x >> op.k), by = op.oy + ((uint32_t)j0y >> op.k);
        float4* cg = corners + op.coff;
        for (int e = e0; e < n; e += step) {
            const int cy = (int)__umulhi((uint32_t)e, op.magic);
            const int cx = e - cy * op.ncx;
            uint32_t x = bx + (uint32_t)cx, y = by + (uint32_t)cy, z = op.key;
            pcg3d(x, y, z);
            float4 c;
            if (METHOD == kZeroGrad)  // corner values only (Eq. zg has zero gradients)
                c = make_float4(unit_value(x) * op.amp, 0.0f, 0.0f, 0.0f);
            else if (METHOD == kC1 || METHOD == kC2 || METHOD == kPaperGauge)
                c = make_float4(unit_value(x) * op.amp, unit_value(y) * op.ampw, unit_value(z) * op.ampw, 0.0f);
            else
                c = make_float4(0.0f, unit_value(y) * op.amp, unit_value(z) * op.amp, 0.0f);
            cg[cy * op.rowlen + corner_slot(cx)] = c;
        }
    }
}

__device__ __forceinline__ Cell load_cell(const float4* __restrict__ cg, int rowlen, int lcx, int lcy)
{
    const float4* row0 = cg + lcy * rowlen;
    const float4* row1 = row0 + rowlen;
    const int s0 = corner_slot(lcx), s1 = corner_slot(lcx + 1);
    Cell c;
    c.c00 = row0[s0];
    c.c10 = row0[s1];
    c.c01 = row1[s0];
    c.c11 = row1[s1];
    return c;
}

// A run8 octave: node columns only.
template <int METHOD>
__device__ __forceinline__ void run8_octave(float (&nacc)[kRows][Deg<METHOD>::value + 1],
                                            const float4* __restrict__ sm, const FieldPlan& P, int i, int tx,
                                            int ty, int n8)
{
    constexpr int NN = Deg<METHOD>::value + 1;
    const OctPlan& op = P.oct[i];
    const float4* ylut = sm + xnode_words<METHOD>(n8);
    const float4* cg = ylut + n8 * 64 + op.coff;
    const Cell c = load_cell(cg, op.rowlen, (tx * kCols) >> op.k, (ty * kRows) >> op.k);
    float4 xb[NN];
#pragma unroll
    for (int q = 0; q < NN; ++q) xb[q] = sm[(i * NN + q) * 8 + tx];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const float4 yb = ylut[i * 64 + r * 16 + ty];
        const Row R = Model<METHOD>::row(c, yb);
#pragma unroll
        for (int q = 0; q < NN; ++q) nacc[r][q] += Model<METHOD>::eval(R, xb[q]);
    }
}

// Cells of spc_i = 4 (CW = 4) or 2 (CW = 2) samples: the in-cell position of
// column c is (c mod CW) / CW, of row r (r mod CW) / CW -- constants.
template <int METHOD, int CW>
__device__ __forceinline__ void small_octave(float (&acc)[kRows][kCols], const float4* __restrict__ sm,
                                             const FieldPlan& P, int i, int tx, int ty, int n8)
{
    const OctPlan& op = P.oct[i];
    const float4* cg = sm + xnode_words<METHOD>(n8) + n8 * 64 + op.coff;
    constexpr float inv = 1.0f / CW;
#pragma unroll
    for (int yq = 0; yq < kRows / CW; ++yq) {
        const int lcy = (ty * kRows + yq * CW) / CW;
#pragma unroll
        for (int xq = 0; xq < kCols / CW; ++xq) {
            const int lcx = (tx * kCols + xq * CW) / CW;
            const Cell c = load_cell(cg, op.rowlen, lcx, lcy);
#pragma unroll
            for (int rr = 0; rr < CW; ++rr) {
                const Row R = rr == 0 ? Model<METHOD>::row0(c) : Model<METHOD>::row(c, axis_basis<METHOD>(rr * inv));
#pragma unroll
                for (int q = 0; q < CW; ++q) {
                    const float h = q == 0 ? R.V0 : Model<METHOD>::eval(R, axis_basis<METHOD>(q * inv));
                    acc[yq * CW + rr][xq * CW + q] += h;
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
__device__ __forceinline__ void fbm2d_tile(const FieldPlan& P, float4* sm, int bx, int by)
{
    constexpr int D = Deg<METHOD>::value, NN = D + 1;
    const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
    const int x0 = bx * kTW, y0 = by * kTH;        // output tile origin
    const int j0x = x0 + P.jx0, j0y = y0 + P.jy0;  // sample indices
    const int s = P.s, N = P.N, n8 = n_run8(P);
    stage_tile<METHOD>(P, sm, j0x, j0y);
    __syncthreads();

    // run8 octaves: node columns, then interpolate the other columns once
    float nacc[kRows][NN];
#pragma unroll
    for (int r = 0; r < kRows; ++r)
#pragma unroll
        for (int q = 0; q < NN; ++q) nacc[r][q] = 0.0f;
    for (int i = 0; i < n8; ++i) run8_octave<METHOD>(nacc, sm, P, i, tx, ty, n8);
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

    // cells of 4 and 2 samples, then lattice octaves
    if (s >= 2 && s - 2 < N) small_octave<METHOD, 4>(acc, sm, P, s - 2, tx, ty, n8);
    if (s >= 1 && s - 1 < N) small_octave<METHOD, 2>(acc, sm, P, s - 1, tx, ty, n8);
    if (METHOD != kPerlinS5 && METHOD != kPerlinS3)
        for (int i = s; i < N; ++i)
            lattice_octave(acc, P.oct[i], (uint32_t)(j0x + tx * kCols), (uint32_t)(j0y + ty * kRows));
    store_tile<OutT>(P, acc, x0 + tx * kCols, y0 + ty * kRows);
}

template <int METHOD, typename OutT>
__global__ void __launch_bounds__(kThreads) fbm2d_kernel(const __grid_constant__ FieldPlan P)
{
    extern __shared__ float4 sm[];
    fbm2d_tile<METHOD, OutT>(P, sm, blockIdx.x, blockIdx.y);
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
        const bool f16 = plan.dtype == 1;
        switch (plan.method) {
        case kC1:
            if (f16) fbm2d_tile<kC1, __half>(plan, sm, bx, by);
            else fbm2d_tile<kC1, float>(plan, sm, bx, by);
            break;
        case kC2:
            if (f16) fbm2d_tile<kC2, __half>(plan, sm, bx, by);
            else fbm2d_tile<kC2, float>(plan, sm, bx, by);
            break;
        case kPaperGauge:
            if (f16) fbm2d_tile<kPaperGauge, __half>(plan, sm, bx, by);
            else fbm2d_tile<kPaperGauge, float>(plan, sm, bx, by);
            break;
        case kZeroGrad:
            if (f16) fbm2d_tile<kZeroGrad, __half>(plan, sm, bx, by);
            else fbm2d_tile<kZeroGrad, float>(plan, sm, bx, by);
            break;
        case kPerlinS5:
            if (f16) fbm2d_tile<kPerlinS5, __half>(plan, sm, bx, by);
            else fbm2d_tile<kPerlinS5, float>(plan, sm, bx, by);
            break;
        default:
            if (f16) fbm2d_tile<kPerlinS3, __half>(plan, sm, bx, by);
            else fbm2d_tile<kPerlinS3, float>(plan, sm, bx, by);
            break;
        }
        __syncthreads();
    }
}

template <int METHOD>
size_t smem_words(const FieldPlan& P)
{
    int n8 = P.s - 2;
    n8 = n8 < 0 ? 0 : (n8 < P.N ? n8 : P.N);
    return (size_t)xnode_words<METHOD>(n8) + (size_t)n8 * 64 + (size_t)P.ncorner;
}

template <typename K>
cudaError_t set_smem(K kfn, size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kfn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    return e;
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
    const bool f16 = P.dtype == 1;
#define PTG_LAUNCH2D(M, T)                                                                           \
    do {                                                                                             \
        auto kfn = fbm2d_kernel<M, T>;                                                               \
        cudaError_t e = set_smem(kfn, smem);                                                         \
        if (e != cudaSuccess) return e;                                                              \
        kfn<<<grid, kThreads, smem, stream>>>(P);                                                    \
        return cudaGetLastError();                                                                   \
    } while (0)
    switch (method) {
    case kC1: if (f16) PTG_LAUNCH2D(kC1, __half); else PTG_LAUNCH2D(kC1, float);
    case kC2: if (f16) PTG_LAUNCH2D(kC2, __half); else PTG_LAUNCH2D(kC2, float);
    case kPaperGauge: if (f16) PTG_LAUNCH2D(kPaperGauge, __half); else PTG_LAUNCH2D(kPaperGauge, float);
    case kZeroGrad: if (f16) PTG_LAUNCH2D(kZeroGrad, __half); else PTG_LAUNCH2D(kZeroGrad, float);
    case kPerlinS5: if (f16) PTG_LAUNCH2D(kPerlinS5, __half); else PTG_LAUNCH2D(kPerlinS5, float);
    case kPerlinS3: if (f16) PTG_LAUNCH2D(kPerlinS3, __half); else PTG_LAUNCH2D(kPerlinS3, float);
    default: return cudaErrorInvalidValue;
    }
#undef PTG_LAUNCH2D
}

cudaError_t launch_fbm2d_batch(const FieldPlan* plans, const long long* tile_start, int n,
                               unsigned long long* counter, size_t smem, int blocks, cudaStream_t stream)
{
    cudaError_t e = set_smem(fbm2d_batch_kernel, smem);
    if (e != cudaSuccess) return e;
    fbm2d_batch_kernel<<<blocks, kThreads, smem, stream>>>(plans, tile_start, n, counter);
    return cudaGetLastError();
}

int fbm2d_batch_blocks_per_sm(size_t smem)
{
    int nb = 0;
    set_smem(fbm2d_batch_kernel, smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fbm2d_batch_kernel, kThreads, smem) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

}  // namespace ptg
