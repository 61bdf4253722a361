// ptg_kernels.h -- internal launch entry points of the generator kernels
// (host side of the CUDA translation units; not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include "ptg_device.cuh"

namespace ptg {

// Raise a kernel's dynamic shared-memory limit to at least `smem` bytes (and
// prefer the largest shared-memory carveout) on the current device.  The
// attribute calls are made once per kernel, device and larger size; later
// launches skip them.
cudaError_t set_kernel_smem(const void* kfn, size_t smem);

// Tile shapes (samples) of the fused generators.
constexpr int kTile2dX = 64, kTile2dY = 64;
constexpr int kTile3dX = 32, kTile3dY = 16, kTile3dZ = 8;

// Float4 slots per staged corner row of a 3D tile with ncx corners a row.
// Rows longer than two slots take an odd length, so that the corner loads
// of two neighbouring rows (threads ty and ty + 1 of a quarter warp) land
// in different 16-byte bank groups; rows of two (cells that cover the tile)
// keep the x + 2 y + 4 z layout the staging writes.
__host__ __device__ constexpr int corner_rowlen3(int ncx)
{
    return corner_slot(ncx - 1) + 1 > 2 ? ((corner_slot(ncx - 1) + 1) | 1) : 2;
}

size_t fbm2d_smem_bytes(const FieldPlan& P);
cudaError_t launch_fbm2d(const FieldPlan& P, int method, int s, cudaStream_t stream);

// Persistent batched 2D generator over many fields (plans, tile_start and
// counter in device memory; counter must be zero at launch; total_tiles =
// tile_start[n], which sets how many tiles a CTA takes at a time).
cudaError_t launch_fbm2d_batch(const FieldPlan* plans, const long long* tile_start, int n,
                               unsigned long long* counter, long long total_tiles, size_t smem, int blocks,
                               cudaStream_t stream);
int fbm2d_batch_blocks_per_sm(size_t smem);

size_t fbm3d_smem_bytes(const FieldPlan& P);
cudaError_t launch_fbm3d(const FieldPlan& P, int method, int s, cudaStream_t stream);

// OpenSimplex-style baseline (2D).  base[i] = (x0, y0) of sample (0, 0) at
// octave i in lattice units (FP64, computed on the host); step[i] = f^i / spc
// lattice units per sample in FP64 (step_d), and as two floats step + step_lo
// (step_lo = 0 when the step is a power of two).
struct SimplexPlan {
    void* out;
    int32_t W, H, dtype, N, tiles_x, tiles_y;
    double base_x[kMaxOctaves], base_y[kMaxOctaves];
    double step_d[kMaxOctaves];
    float step[kMaxOctaves];
    float step_lo[kMaxOctaves];
    float amp[kMaxOctaves];
    uint32_t key[kMaxOctaves];
    int32_t box_off[kMaxOctaves];  // staged gradient box of octave i: first float2 in shared memory
    int32_t box_wb[kMaxOctaves];   // its side bound (row stride); 0 = hash vertices directly
    int32_t box_words;             // float2 words of shared memory for all boxes
    uint32_t exact_mask;           // bit i: step[i] is a power of two (products k * step exact)
};
cudaError_t launch_opensimplex2d(const SimplexPlan& P, cudaStream_t stream);

// 3D OpenSimplex-style noise.  base[k][i] = real lattice coordinate along
// axis k of the launch's sample (0, 0, 0) at octave i (FP64, host); step_d[i]
// = lattice units per sample (also as float hi + lo).  Octaves whose gradient
// box fits are staged one at a time into one shared buffer of box_words
// float4; box_w[k][i] bounds the box extent along axis k (0 = hash per sample).
struct Simplex3Plan {
    void* out;
    int32_t W, H, D, dtype, N, tiles_x, tiles_y, tiles_z;
    int32_t box_words;
    uint32_t exact_mask;  // bit i: step[i] is a power of two (products k * step exact)
    double base[3][kMaxOctaves];
    double step_d[kMaxOctaves];
    float step[kMaxOctaves], step_lo[kMaxOctaves], amp[kMaxOctaves];
    uint32_t key[kMaxOctaves];
    int32_t box_w[3][kMaxOctaves];
};
cudaError_t launch_opensimplex3d(const Simplex3Plan& P, cudaStream_t stream);

// Polynomial and Perlin fields with any frequency ratio f between octaves
// (2D).  base[i] = lattice coordinate of output sample (0, 0) at octave i
// (FP64, host); scale[i] = f^i / spc lattice units per sample, also split
// into two floats (hi + lo) for the per-sample offsets inside a tile.
// Ridged noise (ridged = 1): the corners carry unit amplitude (amp = 1,
// ampw = w) and wgt[i] = p^i weights octave i's ridge.
struct GeneralPlan {
    void* out;
    int32_t W, H, dtype, N, vec_ok, tiles_x, tiles_y, method;
    int32_t box_words;  // float4 words of shared memory for all staged corner boxes
    int32_t ridged;
    uint32_t lattice_mask;  // bit i: every sample of octave i is a lattice point (integer coordinates)
    int32_t pad;
    double base_x[kMaxOctaves], base_y[kMaxOctaves];
    double scale[kMaxOctaves];
    float scale_hi[kMaxOctaves], scale_lo[kMaxOctaves];
    float amp[kMaxOctaves], ampw[kMaxOctaves], wgt[kMaxOctaves];
    uint32_t key[kMaxOctaves];
    int32_t box_off[kMaxOctaves];  // staged corner box of octave i: first float4 in shared memory
    int32_t box_w[kMaxOctaves];    // its side (cells + 1); 0 = hash the corners of each sample
    uint32_t box_magic[kMaxOctaves];  // ceil(2^32 / box_w)
};
cudaError_t launch_general2d(const GeneralPlan& P, cudaStream_t stream);

// The same in 3D (C1, C2, Perlin): 32 x 16 x 8 tiles, corner boxes of
// box_w[0..2][i] corners along x, y, z (0 = hash each sample's 8 corners).
struct General3Plan {
    void* out;
    int32_t W, H, D, dtype, N, vec_ok, tiles_x, tiles_y, tiles_z, method;
    int32_t box_words;  // float4 words of shared memory for all staged corner boxes
    int32_t ridged;     // as in GeneralPlan
    uint32_t lattice_mask;  // as in GeneralPlan
    int32_t pad;
    double base[3][kMaxOctaves];  // lattice coordinate of output sample (0, 0, 0) at octave i
    double scale[kMaxOctaves];
    float scale_hi[kMaxOctaves], scale_lo[kMaxOctaves];
    float amp[kMaxOctaves], ampw[kMaxOctaves], wgt[kMaxOctaves];
    uint32_t key[kMaxOctaves];
    int32_t box_off[kMaxOctaves];
    int32_t box_w[3][kMaxOctaves];
    uint32_t box_magic[2][kMaxOctaves];  // ceil(2^32 / wx), ceil(2^32 / (wx wy))
};
cudaError_t launch_general3d(const General3Plan& P, cudaStream_t stream);

// Map statistics (Sec. 5): coastline box-count pyramid (buf0 >= (W-1)(H-1)
// bytes, buf1 >= a quarter of that rounded up; counts[levels] zeroed) and the
// height / slope histogram (hist[bins + 2] accumulated).
cudaError_t launch_box_counts(const float* map, long long W, long long H, float level, int levels, uint8_t* buf0,
                              uint8_t* buf1, unsigned long long* counts, int num_sms, cudaStream_t stream);
cudaError_t launch_histogram(const float* maps, long long W, long long H, long long count, float lo, float scale,
                             int bins, int what, unsigned long long* hist, int num_sms, cudaStream_t stream);

// Test hooks.
cudaError_t launch_debug_hash(int dims, const uint32_t* keys, long long n, uint32_t* out, cudaStream_t stream);
cudaError_t launch_bounds_selftest(int site, long long idx, long long n, cudaStream_t stream);
cudaError_t launch_debug_axis(long long origin, int s, int octave, const long long* j, long long n,
                              uint32_t* cell, float* t, cudaStream_t stream);

}  // namespace ptg
