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
// Gradient staging: for octaves whose lattice spacing is at least a sample
// (up to one lattice unit a sample, while the boxes fit in 96 KB), the CTA
// hashes every vertex of the stretched-plane box that its 64 x 64 tile can
// touch into shared memory once; samples then read their four gradients.
// Finer octaves hash the four vertices per sample directly.  The tile spans
// L = 64 x (lattice units a sample) in real space, i.e.
// [s0 + r L, s0 + (1 + r) L] in each stretched coordinate (s0 the tile's first
// sample); two vertices of margin below and three above cover the extra
// vertices (offsets -1..2) and rounding.
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

// Thread layout: the 32 lanes of a warp cover an 8 x 4 block of samples at a
// time (lane = x + 8 y), so that the gradients they gather from a staged box at
// one instruction lie close together.  A thread takes the columns lx + 8 c
// (c < 8) and the rows 16 w + ly + 4 r (r < 4) of warp w's 16 rows, one row at
// a time through all octaves: the row loop stays rolled, so that the octave
// bodies (8 samples x 4 vertices each) fit the instruction cache.
constexpr int kTW = 64, kTH = 64, kThreads = 128, kCols = 8, kRows = 4;
constexpr float kSquish = 0.36602540378443865f;   // (sqrt(3) - 1) / 2
constexpr double kStretchD = -0.21132486540518713; // (1/sqrt(3) - 1) / 2
constexpr float kStretchHi = (float)kStretchD;
constexpr float kStretchLo = (float)(kStretchD - (double)kStretchHi);
constexpr float kScale = 0.125f;

struct TileOctave {
    int32_t a0, b0;      // integer stretched vertex of the tile's first sample
    float fx, fy;        // its fractional stretched coordinates
    float fxl, fyl;      // their rounding residuals (used when steps are not powers of two)
    int32_t amin, bmin;  // staged: first vertex of the gradient box
    int32_t w, h;        // staged: box extent actually filled (<= plan bound)
};

// a + b = s + err exactly (Knuth's two-sum).
__device__ __forceinline__ float two_sum_err(float a, float b, float s)
{
    const float bv = s - a;
    return (a - (s - bv)) + (b - bv);
}

__device__ __forceinline__ float kernel_term(float gx, float gy, float dx, float dy)
{
    const float k = fmaxf(0.0f, 2.0f - fmaf(dx, dx, dy * dy));
    const float k2 = k * k;
    return (k2 * k2) * fmaf(gx, dx, gy * dy);
}

// Gradient of vertex (a, b): read from the staged box, or hashed.
template <bool kStaged>
struct Grad {
    const float2* box;
    int32_t amin, bmin, wb, size;
    uint32_t key;
    __device__ __forceinline__ float2 at(int32_t a, int32_t b) const
    {
        if (kStaged) {
            int idx = (b - bmin) * wb + (a - amin);
            // the box covers every reachable vertex: the debug build checks the
            // index before the clamp, which only guards
            if (!bounds_ok(kSiteGradient, idx, size)) return make_float2(0.0f, 0.0f);
            idx = min(max(idx, 0), size - 1);
            return sld(kSiteGradient, &box[idx]);
        }
        uint32_t x = (uint32_t)a, y = (uint32_t)b, z = key;
        pcg3d(x, y, z);
        return make_float2(unit_value(y), unit_value(z));
    }
};

// Contribution of vertex (a + da, b + db) at stretched fraction (xi, yi).
template <bool kStaged>
__device__ __forceinline__ float vertex_at(const Grad<kStaged>& G, int32_t a, int32_t b, int da, int db, float xi,
                                           float yi)
{
    const float u = xi - (float)da, v = yi - (float)db;
    const float s = (u + v) * kSquish;
    const float2 g = G.at(a + da, b + db);
    return kernel_term(g.x, g.y, u + s, v + s);
}

// Branch-free vertex choice (neighbouring samples fall in different
// triangles, so branches would diverge): both triangles share (1,0) and
// (0,1); the third vertex is (0,0) or (1,1); the extra one is selected from
// the barycentric weights.
template <bool kStaged>
__device__ __forceinline__ float sample_noise(const Grad<kStaged>& G, int32_t a, int32_t b, float xi, float yi)
{
    const bool lower = xi + yi < 1.0f;
    const int d3 = lower ? 0 : 1;
    // lower: weights (w00, w10, w01) -> extras (1,1), (-1,1), (1,-1)
    // upper: weights (w11, w10, w01) -> extras (0,0), (0,2), (2,0)
    const float wc = lower ? 1.0f - xi - yi : xi + yi - 1.0f;
    const float wx = lower ? xi : 1.0f - yi;
    const float wy = lower ? yi : 1.0f - xi;
    int ex, ey;
    if (wc <= wx && wc <= wy) { ex = lower ? 1 : 0; ey = lower ? 1 : 0; }
    else if (wx <= wy) { ex = lower ? -1 : 0; ey = lower ? 1 : 2; }
    else { ex = lower ? 1 : 2; ey = lower ? -1 : 0; }
    return vertex_at(G, a, b, 1, 0, xi, yi) + vertex_at(G, a, b, 0, 1, xi, yi) +
           vertex_at(G, a, b, d3, d3, xi, yi) + vertex_at(G, a, b, ex, ey, xi, yi);
}

// One octave for the thread's 8 samples of tile row ly.  kExact: the step is
// a power of two, so the offsets k * step and their sums are exact floats.
template <bool kStaged, bool kExact>
__device__ __forceinline__ void simplex_row(float (&acc)[kCols], const SimplexPlan& P, const TileOctave T,
                                            const float2* boxes, int i, int lx, int ly)
{
    const float step = P.step[i], step_lo = P.step_lo[i], amp = P.amp[i] * kScale;
    Grad<kStaged> G;
    G.key = P.key[i];
    G.wb = P.box_wb[i];
    G.box = boxes + P.box_off[i];
    G.amin = T.amin;
    G.bmin = T.bmin;
    G.size = G.wb * G.wb;
    // Offsets k * step as a float plus its residual (k * step - that float):
    // zero when the step is a power of two, so that the arithmetic below is
    // exact there; otherwise it carries the product and step rounding.
    // Without exact steps every sum below also keeps its rounding residual
    // (two-sums), so that a sample's stretched position is off by about one
    // float rounding, as with exact steps.
    // cse: residual of the product k * step (it enters the stretch); cbe: the
    // residuals of the base fraction and of the sum fxc (they do not).
    float cs[kCols], cse[kCols], cbe[kCols], fxc[kCols];
    int32_t icx[kCols];
#pragma unroll
    for (int c = 0; c < kCols; ++c) {
        const float k = (float)(lx + 8 * c);
        cs[c] = __fmul_rn(k, step);  // rounded and never contracted: cse carries its rounding error
        const float fl = floorf(cs[c]);
        icx[c] = (int32_t)fl;
        fxc[c] = T.fx + (cs[c] - fl);
        cse[c] = kExact ? 0.0f : fmaf(k, step, -cs[c]) + k * step_lo;
        cbe[c] = kExact ? 0.0f : two_sum_err(T.fx, cs[c] - fl, fxc[c]) + T.fxl;
    }
    const float k = (float)ly;
    const float rs = __fmul_rn(k, step);
    const float fl = floorf(rs);
    const int32_t iry = (int32_t)fl;
    const float fyr = T.fy + (rs - fl);
    const float rse = kExact ? 0.0f : fmaf(k, step, -rs) + k * step_lo;
    const float rbe = kExact ? 0.0f : two_sum_err(T.fy, rs - fl, fyr) + T.fyl;
#pragma unroll
    for (int c = 0; c < kCols; ++c) {
        const float K = cs[c] + rs;
        const float p = __fmul_rn(K, kStretchHi);  // e carries its rounding error
        const float e = fmaf(K, kStretchHi, -p);         // exact rounding error of p
        const float ip = floorf(p);
        float t, sx, sy;
        if (kExact) {
            t = (p - ip) + (e + K * kStretchLo);
            sx = fxc[c] + t;
            sy = fyr + t;
        } else {
            const float Ke = two_sum_err(cs[c], rs, K) + (cse[c] + rse);  // K's error and product residuals
            const float small = e + fmaf(Ke, kStretchHi, K * kStretchLo);
            const float pt = p - ip;  // exact
            t = pt + small;
            const float te = two_sum_err(pt, small, t);
            const float ux = fxc[c] + t, uy = fyr + t;
            sx = ux + (two_sum_err(fxc[c], t, ux) + (te + (cse[c] + cbe[c])));
            sy = uy + (two_sum_err(fyr, t, uy) + (te + (rse + rbe)));
        }
        const float flx = floorf(sx), fly = floorf(sy);
        const float xi = sx - flx, yi = sy - fly;
        const int32_t iip = (int32_t)ip;
        const int32_t a = T.a0 + icx[c] + iip + (int32_t)flx;
        const int32_t b = T.b0 + iry + iip + (int32_t)fly;
        acc[c] = fmaf(amp, sample_noise(G, a, b, xi, yi), acc[c]);
    }
}

// kAllExact: every octave's step is a power of two (the dyadic fields), so
// only the exact-offset octave code is compiled into the kernel.
template <typename OutT, bool kAllExact>
__global__ void __launch_bounds__(kThreads) opensimplex2d_kernel(const __grid_constant__ SimplexPlan P)
{
    __shared__ TileOctave tile[kMaxOctaves];
    extern __shared__ float2 boxes[];
    const int tid = threadIdx.x, lx = tid & 7, ly0 = ((tid >> 5) << 4) | ((tid >> 3) & 3);
    const int j0x = blockIdx.x * kTW, j0y = blockIdx.y * kTH;
    if (tid < P.N) {
        const int i = tid;
        const double X = P.base_x[i] + (double)j0x * P.step_d[i];
        const double Y = P.base_y[i] + (double)j0y * P.step_d[i];
        const double sh = (X + Y) * kStretchD;
        const double xs = X + sh, ys = Y + sh;
        const double fa = floor(xs), fb = floor(ys);
        TileOctave T;
        T.a0 = (int32_t)(long long)fa;
        T.b0 = (int32_t)(long long)fb;
        T.fx = (float)(xs - fa);
        T.fy = (float)(ys - fb);
        T.fxl = (float)((xs - fa) - (double)T.fx);
        T.fyl = (float)((ys - fb) - (double)T.fy);
        T.amin = T.bmin = T.w = T.h = 0;
        if (P.box_wb[i] > 0) {
            const double L = 64.0 * P.step_d[i];
            T.amin = (int32_t)(long long)floor(xs + kStretchD * L) - 2;
            T.bmin = (int32_t)(long long)floor(ys + kStretchD * L) - 2;
            T.w = min((int32_t)(long long)floor(xs + (1.0 + kStretchD) * L) + 3 - T.amin + 1, P.box_wb[i]);
            T.h = min((int32_t)(long long)floor(ys + (1.0 + kStretchD) * L) + 3 - T.bmin + 1, P.box_wb[i]);
        }
        if (bounds_ok(kSiteTable, i, kMaxOctaves)) tile[i] = T;
    }
    __syncthreads();
    // hash the gradient boxes of the staged octaves (uniform loop per octave)
    for (int i = 0; i < P.N; ++i) {
        if (P.box_wb[i] <= 0) continue;
        const TileOctave T = tile[i];
        const int n = T.w * T.h, wb = P.box_wb[i];
        const float inv = 1.0f / (float)T.w;
        float2* box = boxes + P.box_off[i];
        for (int v = tid; v < n; v += kThreads) {
            const int vy = (int)(((float)v + 0.5f) * inv);  // exact: v < 2^14, w < 2^7
            const int vx = v - vy * T.w;
            uint32_t x = (uint32_t)(T.amin + vx), y = (uint32_t)(T.bmin + vy), z = P.key[i];
            pcg3d(x, y, z);
            if (bounds_ok(kSiteStage, vy * wb + vx, wb * wb) && bounds_ok(kSiteStage, vx, wb))
                sst(kSiteStage, &box[vy * wb + vx], make_float2(unit_value(y), unit_value(z)));
        }
    }
    __syncthreads();

    OutT* out = reinterpret_cast<OutT*>(P.out);
#pragma unroll 1
    for (int r = 0; r < kRows; ++r) {
        const int ly = ly0 + 4 * r, y = j0y + ly;
        if (y >= P.H) break;  // rows grow with r; no barrier follows
        float acc[kCols];
#pragma unroll
        for (int c = 0; c < kCols; ++c) acc[c] = 0.0f;
        for (int i = 0; i < P.N; ++i) {
            const bool exact = kAllExact || ((P.exact_mask >> i) & 1u);
            if (P.box_wb[i] > 0) {
                if (exact) simplex_row<true, true>(acc, P, tile[i], boxes, i, lx, ly);
                else simplex_row<true, kAllExact>(acc, P, tile[i], boxes, i, lx, ly);
            } else {
                if (exact) simplex_row<false, true>(acc, P, tile[i], boxes, i, lx, ly);
                else simplex_row<false, kAllExact>(acc, P, tile[i], boxes, i, lx, ly);
            }
        }
        OutT* row = out + (size_t)y * (size_t)P.W;
#pragma unroll
        for (int c = 0; c < kCols; ++c) {
            const int x = j0x + lx + 8 * c;
            if (x < P.W && bounds_ok(kSiteStore, (long long)y * P.W + x, (long long)P.W * P.H)) store1(row + x, acc[c]);
        }
    }
}

}  // namespace

cudaError_t launch_opensimplex2d(const SimplexPlan& P, cudaStream_t stream)
{
    const dim3 grid(P.tiles_x, P.tiles_y, 1);
    const size_t smem = sizeof(float2) * (size_t)P.box_words;
    const bool all_exact = P.exact_mask == (P.N >= 32 ? 0xffffffffu : (1u << P.N) - 1u);
#define PTG_LAUNCHOS(T, X)                                                                           \
    do {                                                                                             \
        auto kfn = opensimplex2d_kernel<T, X>;                                                       \
        cudaError_t e = set_kernel_smem((const void*)kfn, smem);                                     \
        if (e != cudaSuccess) return e;                                                              \
        kfn<<<grid, kThreads, smem, stream>>>(P);                                                    \
        return cudaGetLastError();                                                                   \
    } while (0)
    if (P.dtype == 1) {
        if (all_exact) PTG_LAUNCHOS(__half, true);
        PTG_LAUNCHOS(__half, false);
    }
    if (all_exact) PTG_LAUNCHOS(float, true);
    PTG_LAUNCHOS(float, false);
#undef PTG_LAUNCHOS
}

}  // namespace ptg
