// ptg_device.cuh -- device building blocks shared by the generator kernels:
// the corner hash, the hash-word -> [-1, 1) map, the per-axis polynomial
// bases of each method, and the launch plan that the host fills per field.
//
// Method: Thorimbert & Chopard, arXiv:1610.03525.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>

namespace ptg {

// Method codes of the generator kernels.
enum : int {
    kC1 = 1,          // D?M1N3, zero twist: tensor cubic Hermite (Sec. 3.1, 3.4)
    kC2 = 2,          // D?M2N5, zero 2nd derivatives: tensor quintic Hermite (Sec. 3.4)
    kPaperGauge = 3,  // D2M1N3 with the printed coefficients (Sec. 3.1), C0 across faces
    kZeroGrad = 4,    // zero-gradient D2M1N3 (Eq. zg with the -xy term), C0 across faces
    kPerlinS5 = 10,   // Perlin's polynomial, smootherstep blend (Sec. 3.2, 5.1)
    kPerlinS3 = 11    // Perlin's polynomial, smoothstep blend (Sec. 3.2)
};

// Octave modes.  A staged octave (cells at least two samples wide) keeps the
// corner data of the CTA tile's cells in shared memory; the number names how
// many samples of a thread's run share one cell along x.  A lattice octave
// (cells one sample wide or narrower) puts every sample on a lattice point,
// where the cell polynomial equals the corner value (Eq. mixedderiv, d = 0).
enum : int { kModeLattice = 0, kModeRun2 = 2, kModeRun4 = 4, kModeRun8 = 8 };

constexpr int kMaxOctaves = 32;

// Per-octave launch plan (host-filled).
struct OctPlan {
    int32_t mode;           // kMode*
    int32_t k;              // staged: log2(samples per cell); lattice: i - log2(spc)
    int32_t ncx, ncy, ncz;  // staged corner grid of one CTA tile
    int32_t coff;           // staged: first corner (float4 units) in shared memory
    uint32_t key;           // hash word: seed << 8 | octave
    uint32_t ox, oy, oz;    // origin * 2^i (mod 2^32)
    float amp;              // persistence^i
    float ampw;             // persistence^i * grad_weight
    uint32_t magic;         // staged: ceil(2^32 / ncx), so that e / ncx == umulhi(e, magic) for small e
    uint32_t magic2;        // staged 3D: ceil(2^32 / (ncx * ncy))
    int32_t rowlen;         // staged: float4 slots per corner row (rows are swizzled, see corner_slot)
};

// One field (2D or 3D) as the kernels see it.
struct FieldPlan {
    void* out;
    int32_t W, H, D;        // samples along x, y, z (D = 1 in 2D)
    int32_t dtype;          // 0 = FP32, 1 = FP16
    int32_t N;              // octaves
    int32_t nst;            // staged octaves = min(N, log2 spc); they are 0 .. nst-1
    int32_t ncorner;        // staged corner slots of one tile, all octaves (shared memory)
    int32_t ncount;         // staged corners of one tile, all octaves (hash work)
    int32_t vec_ok;         // 16-byte vector stores allowed (alignment, row length)
    int32_t tiles_x, tiles_y, tiles_z;
    int32_t jx0, jy0, jz0;  // sample index of output element 0 (bands of a larger field)
    int32_t method;         // kC1, kC2, kPerlinS5, kPerlinS3
    int32_t s;              // log2(samples per cell)
    int32_t rw;             // 2D thread shape: run width 8 (8 x 4 samples a thread) or 16 (16 x 2)
    int32_t nt;             // 2D: octaves summed at the tile nodes (cells >= 64 samples), 0 = none
    float lat_bias;         // sum over the lattice octaves of -3 amp (see unit_mant)
    float grad_w;           // gradient weight w of Sec. 4 (ridged fields stage unit-amplitude corners)
    int32_t ridged;         // 1: ridged multifractal sum (2D), octave i weighted by oct[i].amp
    OctPlan oct[kMaxOctaves];
};
static_assert(sizeof(FieldPlan) % 16 == 0, "FieldPlan is copied in 16-byte words");

// ---------------------------------------------------------------------------
// Hash: pcg3d and pcg4d of Jarzynski & Olano ("Hash Functions for GPU
// Rendering", JCGT 9(3), 2020): an LCG step per word, cross-word multiply-adds,
// a 16-bit xorshift, and a second round of cross-word multiply-adds.
// ---------------------------------------------------------------------------
// The steps of pcg3d after its LCG step (x, y, z already stepped), for
// callers that take the LCG steps of row- or octave-invariant words once.
__device__ __forceinline__ void pcg3d_post(uint32_t& x, uint32_t& y, uint32_t& z)
{
    x += y * z;
    y += z * x;
    z += x * y;
    x ^= x >> 16;
    y ^= y >> 16;
    z ^= z >> 16;
    x += y * z;
    y += z * x;
    z += x * y;
}

__device__ __forceinline__ void pcg3d(uint32_t& x, uint32_t& y, uint32_t& z)
{
    x = x * 1664525u + 1013904223u;
    y = y * 1664525u + 1013904223u;
    z = z * 1664525u + 1013904223u;
    x += y * z;
    y += z * x;
    z += x * y;
    x ^= x >> 16;
    y ^= y >> 16;
    z ^= z >> 16;
    x += y * z;
    y += z * x;
    z += x * y;
}

// Word 0 of pcg3d only (the corner value); the compiler drops the rest.
__device__ __forceinline__ uint32_t pcg3d_value(uint32_t x, uint32_t y, uint32_t z)
{
    pcg3d(x, y, z);
    return x;
}

// Word 0 of pcg3d along a run of lattice points (x0 + c d, y, z), c = 0, 1, ...
// The LCG steps of y and z and the addend y1 z1 of x's first cross step are
// the same for the whole run, and x's LCG step advances by d * 1664525 per
// point, so a point costs its own cross steps and xorshifts only.
__device__ __forceinline__ uint32_t pcg_lcg(uint32_t u) { return u * 1664525u + 1013904223u; }

// x's state after its first cross step at c = 0: lcg(x0) + y1 z1.
__device__ __forceinline__ uint32_t pcg3d_run_base(uint32_t x0, uint32_t y1, uint32_t z1)
{
    return pcg_lcg(x0) + y1 * z1;
}

// The rest of pcg3d word 0 from that state (x2 = base + c d 1664525).
__device__ __forceinline__ uint32_t pcg3d_run_value(uint32_t x2, uint32_t y1, uint32_t z1)
{
    const uint32_t y2 = y1 + z1 * x2;
    const uint32_t z2 = z1 + x2 * y2;
    const uint32_t x3 = x2 ^ (x2 >> 16), y3 = y2 ^ (y2 >> 16), z3 = z2 ^ (z2 >> 16);
    return x3 + y3 * z3;
}

// pcg4d word 0 likewise, with y1, z1, w1 fixed along the run: lcg(x0) + y1 w1,
// then y, z, w cross steps, xorshifts of x, y, w and x + y w.
__device__ __forceinline__ uint32_t pcg4d_run_base(uint32_t x0, uint32_t y1, uint32_t w1)
{
    return pcg_lcg(x0) + y1 * w1;
}

__device__ __forceinline__ uint32_t pcg4d_run_value(uint32_t x2, uint32_t y1, uint32_t z1, uint32_t w1)
{
    const uint32_t y2 = y1 + z1 * x2;
    const uint32_t z2 = z1 + x2 * y2;
    const uint32_t w2 = w1 + y2 * z2;
    const uint32_t x3 = x2 ^ (x2 >> 16), y3 = y2 ^ (y2 >> 16), w3 = w2 ^ (w2 >> 16);
    return x3 + y3 * w3;
}

// The steps of pcg4d after its LCG step (all four words already stepped).
__device__ __forceinline__ void pcg4d_post(uint32_t& x, uint32_t& y, uint32_t& z, uint32_t& w)
{
    x += y * w;
    y += z * x;
    z += x * y;
    w += y * z;
    x ^= x >> 16;
    y ^= y >> 16;
    z ^= z >> 16;
    w ^= w >> 16;
    x += y * w;
    y += z * x;
    z += x * y;
    w += y * z;
}

__device__ __forceinline__ void pcg4d(uint32_t& x, uint32_t& y, uint32_t& z, uint32_t& w)
{
    x = x * 1664525u + 1013904223u;
    y = y * 1664525u + 1013904223u;
    z = z * 1664525u + 1013904223u;
    w = w * 1664525u + 1013904223u;
    x += y * w;
    y += z * x;
    z += x * y;
    w += y * z;
    x ^= x >> 16;
    y ^= y >> 16;
    z ^= z >> 16;
    w ^= w >> 16;
    x += y * w;
    y += z * x;
    z += x * y;
    w += y * z;
}

__device__ __forceinline__ uint32_t pcg4d_value(uint32_t x, uint32_t y, uint32_t z, uint32_t w)
{
    pcg4d(x, y, z, w);
    return x;
}

// Hash word -> (u >> 9) 2^-22 - 1, exactly: the float with exponent of 2 and
// the top 23 bits of u as mantissa lies in [2, 4); subtracting 3 is exact.
__device__ __forceinline__ float unit_value(uint32_t u)
{
    return __uint_as_float(0x40000000u + (u >> 9)) - 3.0f;
}

// The same float before the subtraction: unit_value(u) + 3, in [2, 4).
__device__ __forceinline__ float unit_mant(uint32_t u) { return __uint_as_float(0x40000000u + (u >> 9)); }

// a * unit_value(u) as one FMA, a m - 3a with m3a = -3a (one rounding of a
// product and sum that are exact when 3a is a float, e.g. a a power of two).
__device__ __forceinline__ float unit_scaled(uint32_t u, float a, float m3a) { return fmaf(unit_mant(u), a, m3a); }

// ---------------------------------------------------------------------------
// Per-axis bases.  Every method's octave term is, inside a cell,
//   sum over corners of  V * A_a(x) A_b(y) [A_c(z)]  plus gradient terms,
// with A_0 = 1 - S, A_1 = S (value blend) and two "slope" functions B0, B1
// that carry the corner gradients.  Returned as (S, B0, B1, 0).
//   C1: cubic Hermite:   S = 3t^2 - 2t^3, B0 = t (1-t)^2, B1 = t^2 (t-1)
//   C2: quintic Hermite: S = 6t^5 - 15t^4 + 10t^3,
//       B0 = t (1-t)^3 (1+3t), B1 = t^3 (t-1) (4-3t)
//   Perlin (Sec. 3.2): v_ab = f (x-a) + g (y-b) blended by S, so along x the
//       gradient f_0b multiplies (1-S) x and f_1b multiplies S (x-1):
//       B0 = (1-S) t, B1 = S (t-1); the corner value is zero.
// ---------------------------------------------------------------------------
//   Zero-gradient (Eq. zg): (S3, t); the paper's D2M1N3: t (monomials).
template <int METHOD>
__device__ __forceinline__ float4 axis_basis(float t)
{
    const float t2 = t * t;
    const float u = t - 1.0f;
    if (METHOD == kZeroGrad) {
        return make_float4(t2 * fmaf(-2.0f, t, 3.0f), t, 0.0f, 0.0f);
    } else if (METHOD == kPaperGauge) {
        return make_float4(t, 0.0f, 0.0f, 0.0f);
    } else if (METHOD == kC1) {
        const float S = t2 * fmaf(-2.0f, t, 3.0f);
        return make_float4(S, t * u * u, t2 * u, 0.0f);
    } else if (METHOD == kC2) {
        const float t3 = t2 * t;
        const float S = t3 * fmaf(t, fmaf(6.0f, t, -15.0f), 10.0f);
        const float B0 = t * (u * u) * (-u) * fmaf(3.0f, t, 1.0f);
        const float B1 = t3 * u * fmaf(-3.0f, t, 4.0f);
        return make_float4(S, B0, B1, 0.0f);
    } else {
        const float S = (METHOD == kPerlinS5) ? t2 * t * fmaf(t, fmaf(6.0f, t, -15.0f), 10.0f)
                                              : t2 * fmaf(-2.0f, t, 3.0f);
        return make_float4(S, (1.0f - S) * t, S * u, 0.0f);
    }
}

// Fixed-point sample -> lattice map of one axis at octave i (Sec. 2.1, Sec. 4):
// sample j lies at (origin + j / spc) 2^i, spc = 2^s.  Cell and position t.
__device__ __forceinline__ uint32_t axis_cell(uint32_t origin_shifted, uint32_t j, int i, int s)
{
    return (i < s) ? origin_shifted + (j >> (s - i)) : origin_shifted + (j << (i - s));
}

__device__ __forceinline__ float axis_t(uint32_t j, int i, int s)
{
    if (i >= s) return 0.0f;
    const int k = s - i;
    const uint32_t r = j & ((1u << k) - 1u);
    return (float)r * __uint_as_float((uint32_t)(127 - k) << 23);  // r * 2^-k, exact
}

// Per-sample generators (any spc or frequency ratio): offset k samples from
// a tile's first sample, in cells of the octave.  fb = the first sample's
// position in its cell, scale = hi + lo cells per sample; returns the whole
// cells n past the first sample's cell and the position t in [0, 1).  k * hi
// keeps its exact rounding error (an FMA), so t is good to about 2^-23.
__device__ __forceinline__ void lattice_split(float k, float shi, float slo, float fb, int& n, float& t)
{
    // __fmul_rn: the rounded product, never contracted into an FMA with a later
    // subtraction (p - pf would then carry the product's rounding error, which
    // e adds again)
    const float p = __fmul_rn(k, shi);
    const float e = fmaf(k, shi, -p);  // k * shi - p, exact
    const float pf = floorf(p);
    float w = (p - pf) + fb;           // p - pf is exact
    w += fmaf(k, slo, e);
    const float wf = floorf(w);
    t = w - wf;
    n = __float2int_rn(pf) + __float2int_rn(wf);
}

// Slot of corner column cx inside a staged 2D corner row: one pad slot after
// every 8 corners, so that the 8 lanes of a quarter warp that read corners 1,
// 2 or 4 apart (cells of 8, 4 or 2 samples) hit 8 different 16-byte bank
// groups.
__host__ __device__ constexpr int corner_slot(int cx) { return cx + (cx >> 3); }

// 2D staged corner layout of a 64 x 64 tile.  Octaves whose cells have 2^K
// samples with K >= 7 come first, 4 slots each, in octave order; then the
// fine octaves K = 6 .. 1 at fixed offsets from the end of that coarse part,
// so that kernels specialised on K address them with constants.  Absent fine
// octaves leave their slots at the end (K small) unused and unreserved.
__host__ __device__ constexpr int corner_ncx2(int K) { return (63 >> K) + 2; }
__host__ __device__ constexpr int corner_rowlen2(int K) { return corner_slot(corner_ncx2(K) - 1) + 1; }
__host__ __device__ constexpr int corner_size2(int K) { return corner_rowlen2(K) * corner_ncx2(K); }
__host__ __device__ constexpr int fine_off2(int K)
{
    int o = 0;
    for (int k = 6; k > K; --k) o += corner_size2(k);
    return o;
}

// Output stores.
__device__ __forceinline__ void store1(float* p, float v) { *p = v; }
__device__ __forceinline__ void store1(__half* p, float v) { *p = __float2half_rn(v); }

// ---------------------------------------------------------------------------
// Bounds checks of the debug build (compiled with -DPTG_DEBUG_BOUNDS, the
// library libptg_debug.so; the regular build has none of this code, and the
// helpers below are plain loads and stores there).  Every shared-memory access
// of the checked kernels is tested against the CTA's dynamic shared memory,
// and every global index against the extent it belongs to.  A violation is
// recorded -- the first one of each translation unit, as (site << 48) | index
// -- and the access is skipped (a load returns zero); nothing traps and no
// thread leaves early, so barriers stay matched.  ptg_debug_bounds() reads
// and clears the records.
// ---------------------------------------------------------------------------
enum BoundsSite : int {
    kSiteStage = 1,      // staging stores: tables, weights, corners
    kSiteCorner = 2,     // corner loads of a cell
    kSiteTable = 3,      // per-CTA basis tables, tile nodes, row table, weights
    kSiteConst = 4,      // compile-time tables in global memory
    kSiteStore = 5,      // output elements
    kSitePlan = 6,       // batch plans and tile offsets
    kSiteGradient = 7,   // OpenSimplex gradient boxes
    kSiteSelfTest = 15   // ptg_debug_bounds_selftest
};

#ifdef PTG_DEBUG_BOUNDS
static __device__ unsigned long long g_ptg_bounds;  // one record per translation unit
#endif

// True if 0 <= idx < n; otherwise records (site, idx) and returns false.
__device__ __forceinline__ bool bounds_ok(int site, long long idx, long long n)
{
#ifdef PTG_DEBUG_BOUNDS
    if (idx >= 0 && idx < n) return true;
    atomicCAS(&g_ptg_bounds, 0ull,
              ((unsigned long long)site << 48) | ((unsigned long long)idx & 0xFFFFFFFFFFFFull));
    return false;
#else
    (void)site, (void)idx, (void)n;
    return true;
#endif
}

// True if `bytes` at p lie inside this CTA's dynamic shared memory.
__device__ __forceinline__ bool smem_ok(int site, const void* p, int bytes)
{
#ifdef PTG_DEBUG_BOUNDS
    extern __shared__ float4 ptg_dynamic_smem[];
    unsigned size;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(size));
    const long long off = (long long)__cvta_generic_to_shared(p) - (long long)__cvta_generic_to_shared(ptg_dynamic_smem);
    return bounds_ok(site, off, (long long)size - bytes + 1);
#else
    (void)site, (void)p, (void)bytes;
    return true;
#endif
}

// Checked shared-memory load and store, and checked read-only global load of
// element i of an array of n.
template <typename T>
__device__ __forceinline__ T sld(int site, const T* p)
{
    if (!smem_ok(site, p, (int)sizeof(T))) return T{};
    return *p;
}

template <typename T>
__device__ __forceinline__ void sst(int site, T* p, const T& v)
{
    if (smem_ok(site, p, (int)sizeof(T))) *p = v;
}

template <typename T, typename I>
__device__ __forceinline__ T gld(int site, const T* p, I i, I n)
{
    if (!bounds_ok(site, (long long)i, (long long)n)) return T{};
    return __ldg(p + i);
}

}  // namespace ptg

#ifdef PTG_DEBUG_BOUNDS
// Host side: each translation unit registers a reader of its record.
#include <cuda_runtime.h>
namespace ptg {
using BoundsReader = cudaError_t (*)(unsigned long long* first);
void register_bounds_reader(BoundsReader fn);
}  // namespace ptg
namespace {
cudaError_t ptg_read_bounds_record(unsigned long long* first)
{
    cudaError_t e = cudaMemcpyFromSymbol(first, ptg::g_ptg_bounds, sizeof(unsigned long long));
    const unsigned long long zero = 0;
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(ptg::g_ptg_bounds, &zero, sizeof zero);
    return e;
}
struct PtgBoundsRegistration {
    PtgBoundsRegistration() { ptg::register_bounds_reader(&ptg_read_bounds_record); }
};
PtgBoundsRegistration ptg_bounds_registration;
}  // namespace
#endif
