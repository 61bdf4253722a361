// ptg_opensimplex3d.cuh -- OpenSimplex-style 3D gradient noise: the
// simplex-lattice comparison point of Thorimbert & Chopard (arXiv:1610.03525,
// Sec. 1, 5.1, 5.2) carried to three dimensions, the 3D baseline their
// conclusion asks for, with the same fractal sum (Sec. 4).
//
// Lattice: integer points (a, b, c) of a stretched space, mapped to real space
// by adding (a + b + c) / 3 to every coordinate (the squish); the result is
// the face-centred cubic lattice with nearest vertices sqrt(2) apart.  A
// point's stretched coordinates are x_k - (x + y + z) / 6.  Every vertex
// within distance sqrt(2) adds (2 - r^2)^4 (g . d), g = pcg4d words 1..3.
//
// Vertex choice.  Let xi in [0, 1)^3 be the point's position in its
// stretched unit cube and u = xi - delta for a vertex at cube offset delta;
// the real displacement is u + (sum u) / 3 per axis, so r^2 = |u|^2 +
// (sum u)^2.  Where sum xi <= 3/2, the vertices that can be within sqrt(2)
// are the nineteen offsets delta with entries in -1..2 listed in kCand (the
// cube corner 0, the three unit steps, the three pairs, the three double
// steps, and the nine mixed ones); they were found by minimising r^2 exactly
// over that half of the cube (a convex quadratic on a polytope, solved over
// every set of active faces) for every delta in -3..4 and keeping those with
// a minimum below 2; the list is the same for sum xi <= 1.6.  The other half maps onto this one by the point
// reflection xi -> 1 - xi, delta -> 1 - delta, which flips the sign of every
// displacement and so of every term.  Nineteen vertices per sample and
// octave, all evaluated (max(0, 2 - r^2) is zero out of range), with no
// branch on the region but the reflection.
//
// Gradient staging: one octave at a time, the CTA hashes every vertex that
// its 32 x 16 x 8 tile can reach into shared memory, while that box holds at
// most 4096 vertices (64 KB); finer octaves hash the nineteen vertices per
// sample.
//
// Precision: the octave-i position of the tile's first sample is formed in
// FP64 once per octave and split into an integer vertex and a fraction per
// stretched axis.  A sample's offsets (o_x, o_y, o_z) from it are exact
// floats when the step is a power of two; the stretch adds K r, K = o_x +
// o_y + o_z, r = -1/6, taken in two pieces r = r_hi + r_lo with the rounding
// of K r_hi recovered by an FMA, and integer parts are removed before
// fractions are summed.  Steps that are not powers of two also carry the
// rounding residuals of every offset and sum (two-sums), as in 2D.
#pragma once

#include <cstdint>

#include "ptg_device.cuh"
#include "ptg_kernels.h"

namespace ptg {
namespace {

constexpr int kTW = kTile3dX, kTH = kTile3dY, kTD = kTile3dZ, kThreads = 128;
// Thread layout: the 32 lanes of a warp cover an 8 x 2 x 2 block of samples
// at a time (lane = x + 8 y + 16 z), so that the gradients they gather from
// the staged box at one instruction lie close together (few distinct words,
// few bank conflicts).  Each thread takes the columns x + 8 c (c < 4) and rows
// y + 2 r (r < 8) of one plane; warp w owns planes 2w and 2w + 1.
constexpr int kCols = 4, kRows = 8;
constexpr double kStretchD = -1.0 / 6.0;
constexpr float kStretchHi = (float)kStretchD;
constexpr float kStretchLo = (float)(kStretchD - (double)kStretchHi);
constexpr float kThird = 1.0f / 3.0f;
constexpr float kScale = 0.125f;
constexpr int kNumCand = 19;

// Cube offsets (stretched) of the vertices that can be within sqrt(2) of a
// point with sum xi <= 3/2.
__host__ __device__ constexpr int cand(int n, int a)
{
    constexpr int t[kNumCand][3] = {
        {0, 0, 0},  {1, 0, 0},  {0, 1, 0},  {0, 0, 1},  {1, 1, 0},  {1, 0, 1},  {0, 1, 1},
        {2, 0, 0},  {0, 2, 0},  {0, 0, 2},  {1, -1, 0}, {-1, 1, 0}, {1, 0, -1}, {-1, 0, 1},
        {0, 1, -1}, {0, -1, 1}, {1, 1, -1}, {1, -1, 1}, {-1, 1, 1},
    };
    return t[n][a];
}

// Displacement constant of candidate n along axis a: delta_a + (sum delta) / 3.
__host__ __device__ constexpr float cand_shift(int n, int a)
{
    return (float)((double)cand(n, a) + (double)(cand(n, 0) + cand(n, 1) + cand(n, 2)) / 3.0);
}

struct TileOctave3 {
    int32_t a0[3];    // integer stretched vertex of the tile's first sample
    float f[3];       // its fractional stretched coordinates
    float fl[3];      // their rounding residuals (used when steps are not powers of two)
    int32_t bmin[3];  // staged: first vertex of the gradient box
    int32_t bw[3];    // staged: box extent per axis (<= plan bound)
};

// a + b = s + err exactly (Knuth's two-sum).
__device__ __forceinline__ float two_sum_err(float a, float b, float s)
{
    const float bv = s - a;
    return (a - (s - bv)) + (b - bv);
}

__device__ __forceinline__ float4 hashed_grad(int32_t a, int32_t b, int32_t c, uint32_t key)
{
    uint32_t x = (uint32_t)a, y = (uint32_t)b, z = (uint32_t)c, w = key;
    pcg4d(x, y, z, w);
    return make_float4(unit_value(y), unit_value(z), unit_value(w), 0.0f);
}

// Sum of the nineteen candidates' terms for a point at stretched fraction
// (x0, x1, x2) of vertex (a, b, c); the caller multiplies by the amplitude.
template <bool kStaged>
__device__ __forceinline__ float sample_noise(const float4* __restrict__ box, int bsx, int bsy, int bsize,
                                              const TileOctave3& T, uint32_t key, int32_t a, int32_t b, int32_t c,
                                              float x0, float x1, float x2)
{
    // reflect the upper half of the cube (sum xi > 3/2) onto the lower one
    const bool refl = (x0 + x1) + x2 > 1.5f;
    const float s = refl ? -1.0f : 1.0f;
    const int is = refl ? -1 : 1;
    if (refl) {
        x0 = 1.0f - x0;
        x1 = 1.0f - x1;
        x2 = 1.0f - x2;
        a += 1;
        b += 1;
        c += 1;
    }
    const float q = ((x0 + x1) + x2) * kThird;
    const float z0 = x0 + q, z1 = x1 + q, z2 = x2 + q;
    int base = 0, sx = 0, sy = 0, sz = 0;
    if (kStaged) {
        base = ((c - T.bmin[2]) * bsy + (b - T.bmin[1])) * bsx + (a - T.bmin[0]);
        sx = is;
        sy = is * bsx;
        sz = is * bsx * bsy;
    }
    float sum = 0.0f;
#pragma unroll
    for (int n = 0; n < kNumCand; ++n) {
        const float d0 = z0 - cand_shift(n, 0), d1 = z1 - cand_shift(n, 1), d2 = z2 - cand_shift(n, 2);
        const float r2 = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
        const float k = fmaxf(0.0f, 2.0f - r2);
        const float k2 = k * k;
        float4 g;
        if (kStaged) {
            int idx = base + cand(n, 0) * sx + cand(n, 1) * sy + cand(n, 2) * sz;
            idx = min(max(idx, 0), bsize - 1);  // the box covers every reachable vertex; the clamp only guards
            g = box[idx];
        } else {
            g = hashed_grad(a + is * cand(n, 0), b + is * cand(n, 1), c + is * cand(n, 2), key);
        }
        sum = fmaf(k2 * k2, fmaf(g.x, d0, fmaf(g.y, d1, g.z * d2)), sum);
    }
    return s * sum;
}

// One octave for the thread's 4 x 8 x 1 samples.  kExact: the step is a
// power of two, so the offsets k * step and their sums are exact floats.
template <bool kStaged, bool kExact>
__device__ __forceinline__ void simplex3_octave(float (&acc)[kRows][kCols], const Simplex3Plan& P,
                                                const TileOctave3& T, const float4* box, int i, int lx, int ly,
                                                int pz)
{
    const float step = P.step[i], step_lo = P.step_lo[i], amp = P.amp[i] * kScale;
    const uint32_t key = P.key[i];
    const int bsx = T.bw[0], bsy = T.bw[1], bsize = bsx * bsy * T.bw[2];

    // per-axis offsets: float, integer part, fraction added to the tile base, residuals
    auto axis = [&](float k, int ax, int32_t& io, float& u, float& o, float& oe, float& be) {
        o = __fmul_rn(k, step);  // rounded and never contracted: oe carries its rounding error
        const float fl = floorf(o);
        io = (int32_t)fl;
        u = T.f[ax] + (o - fl);
        oe = kExact ? 0.0f : fmaf(k, step, -o) + k * step_lo;
        be = kExact ? 0.0f : two_sum_err(T.f[ax], o - fl, u) + T.fl[ax];
    };
    int32_t ioz;
    float uz, oz, oez, bez;
    axis((float)pz, 2, ioz, uz, oz, oez, bez);

#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        int32_t ioy;
        float uy, oy, oey, bey;
        axis((float)(ly + 2 * r), 1, ioy, uy, oy, oey, bey);
        const float oyz = oy + oz;
        const float eyz = kExact ? 0.0f : two_sum_err(oy, oz, oyz) + (oey + oez);
#pragma unroll
        for (int c = 0; c < kCols; ++c) {
            int32_t iox;
            float ux, ox, oex, bex;  // recomputed per row: fewer live registers
            axis((float)(lx + 8 * c), 0, iox, ux, ox, oex, bex);
            const float K = ox + oyz;
            const float p = __fmul_rn(K, kStretchHi);  // e carries its rounding error
            const float e = fmaf(K, kStretchHi, -p);  // exact rounding error of p
            const float ip = floorf(p);
            float s0, s1, s2;
            if (kExact) {
                const float t = (p - ip) + (e + K * kStretchLo);
                s0 = ux + t;
                s1 = uy + t;
                s2 = uz + t;
            } else {
                const float Ke = two_sum_err(ox, oyz, K) + (eyz + oex);
                const float small = e + fmaf(Ke, kStretchHi, K * kStretchLo);
                const float pt = p - ip;  // exact
                const float t = pt + small;
                const float te = two_sum_err(pt, small, t);
                const float v0 = ux + t, v1 = uy + t, v2 = uz + t;
                s0 = v0 + (two_sum_err(ux, t, v0) + (te + (oex + bex)));
                s1 = v1 + (two_sum_err(uy, t, v1) + (te + (oey + bey)));
                s2 = v2 + (two_sum_err(uz, t, v2) + (te + (oez + bez)));
            }
            const float f0 = floorf(s0), f1 = floorf(s1), f2 = floorf(s2);
            const int32_t iip = (int32_t)ip;
            const int32_t a = T.a0[0] + iox + iip + (int32_t)f0;
            const int32_t b = T.a0[1] + ioy + iip + (int32_t)f1;
            const int32_t cc = T.a0[2] + ioz + iip + (int32_t)f2;
            acc[r][c] = fmaf(amp, sample_noise<kStaged>(box, bsx, bsy, bsize, T, key, a, b, cc, s0 - f0,
                                                        s1 - f1, s2 - f2),
                             acc[r][c]);
        }
    }
}

// kAllExact: every octave's step is a power of two (the dyadic fields), so
// only the exact-offset octave code is compiled into the kernel.
template <typename OutT, bool kAllExact>
__global__ void __launch_bounds__(kThreads, 4) opensimplex3d_kernel(const __grid_constant__ Simplex3Plan P)
{
    __shared__ TileOctave3 tile[kMaxOctaves];
    extern __shared__ float4 box[];
    const int tid = threadIdx.x, lx = tid & 7, ly = (tid >> 3) & 1, pz = ((tid >> 5) << 1) | ((tid >> 4) & 1);
    const int j0[3] = {(int)blockIdx.x * kTW, (int)blockIdx.y * kTH, (int)blockIdx.z * kTD};
    if (tid < P.N) {
        const int i = tid;
        double X[3], S[3];
        for (int k = 0; k < 3; ++k) X[k] = P.base[k][i] + (double)j0[k] * P.step_d[i];
        const double sh = (X[0] + X[1] + X[2]) * kStretchD;
        TileOctave3 T;
        for (int k = 0; k < 3; ++k) {
            S[k] = X[k] + sh;
            const double fa = floor(S[k]);
            T.a0[k] = (int32_t)(long long)fa;
            T.f[k] = (float)(S[k] - fa);
            T.fl[k] = (float)((S[k] - fa) - (double)T.f[k]);
            T.bmin[k] = 0;
            T.bw[k] = 0;
        }
        if (P.box_w[0][i] > 0) {
            // stretched range of the tile: [S + r (sum L - L_k), S + (1 + r) L_k], r = -1/6
            const double L[3] = {(kTW - 1) * P.step_d[i], (kTH - 1) * P.step_d[i], (kTD - 1) * P.step_d[i]};
            const double sumL = L[0] + L[1] + L[2];
            // a sample's vertex is floor(s) with s in that range up to float
            // rounding (far below 1e-5); its candidates reach one vertex below
            // and two above
            for (int k = 0; k < 3; ++k) {
                T.bmin[k] = (int32_t)(long long)floor(S[k] + kStretchD * (sumL - L[k]) - 1e-5) - 1;
                const int32_t hi = (int32_t)(long long)floor(S[k] + (1.0 + kStretchD) * L[k] + 1e-5) + 2;
                T.bw[k] = min(hi - T.bmin[k] + 1, P.box_w[k][i]);
            }
        }
        tile[i] = T;
    }
    __syncthreads();

    float acc[kRows][kCols];
#pragma unroll
    for (int r = 0; r < kRows; ++r)
#pragma unroll
        for (int c = 0; c < kCols; ++c) acc[r][c] = 0.0f;

    for (int i = 0; i < P.N; ++i) {
        const TileOctave3 T = tile[i];
        const bool exact = kAllExact || ((P.exact_mask >> i) & 1u);
        if (P.box_w[0][i] > 0) {
            // hash this octave's box (the previous octave's readers are done)
            __syncthreads();
            const int wx = T.bw[0], wxy = T.bw[0] * T.bw[1], n = wxy * T.bw[2];
            const uint32_t key = P.key[i];
            for (int v = tid; v < n; v += kThreads) {
                const int vz = v / wxy, rem = v - vz * wxy;
                const int vy = rem / wx, vx = rem - vy * wx;
                box[v] = hashed_grad(T.bmin[0] + vx, T.bmin[1] + vy, T.bmin[2] + vz, key);
            }
            __syncthreads();
            if (exact) simplex3_octave<true, true>(acc, P, T, box, i, lx, ly, pz);
            else simplex3_octave<true, kAllExact>(acc, P, T, box, i, lx, ly, pz);
        } else {
            if (exact) simplex3_octave<false, true>(acc, P, T, box, i, lx, ly, pz);
            else simplex3_octave<false, kAllExact>(acc, P, T, box, i, lx, ly, pz);
        }
    }

    const int z = j0[2] + pz;
    if (z >= P.D) return;
    OutT* out = reinterpret_cast<OutT*>(P.out);
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const int y = j0[1] + ly + 2 * r;
        if (y >= P.H) break;
        OutT* row = out + ((size_t)z * (size_t)P.H + (size_t)y) * (size_t)P.W;
#pragma unroll
        for (int c = 0; c < kCols; ++c) {
            const int x = j0[0] + lx + 8 * c;
            if (x < P.W) store1(row + x, acc[r][c]);
        }
    }
}

// One kernel instance: OutT is float or __half; kAllExact as above.  Each
// instance is compiled in a translation unit of its own
// (ptg_opensimplex3d_{f32,f16}[_dyadic].cu), which keeps the build parallel.
template <typename OutT, bool kAllExact>
cudaError_t launch_instance(const Simplex3Plan& P, cudaStream_t stream)
{
    const dim3 grid(P.tiles_x, P.tiles_y, P.tiles_z);
    const size_t smem = sizeof(float4) * (size_t)P.box_words;
    auto kfn = opensimplex3d_kernel<OutT, kAllExact>;
    const cudaError_t e = set_kernel_smem((const void*)kfn, smem);
    if (e != cudaSuccess) return e;
    kfn<<<grid, kThreads, smem, stream>>>(P);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_opensimplex3d_f32(const Simplex3Plan& P, cudaStream_t stream);
cudaError_t launch_opensimplex3d_f32_dyadic(const Simplex3Plan& P, cudaStream_t stream);
cudaError_t launch_opensimplex3d_f16(const Simplex3Plan& P, cudaStream_t stream);
cudaError_t launch_opensimplex3d_f16_dyadic(const Simplex3Plan& P, cudaStream_t stream);

}  // namespace ptg
