// ptg_internal.h -- host-side state behind the C ABI (not installed).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "ptg.h"
#include "ptg_device.cuh"
#include "ptg_kernels.h"

// Generator kinds behind the ABI calls.
enum { kKindField = 0, kKindPerlin = 1, kKindSimplex = 2 };

struct PtgServer;

// Makes a device current for the duration of a call, then restores the
// caller's device.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

struct ptg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;  // default stream of the context
    uint64_t budget = 0;            // request-loop HBM budget (bytes)
    std::string err;
    int num_sms = 0;
    int max_smem = 0;
    // banded host-output path
    void* stage = nullptr;
    size_t stage_bytes = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_gen[2] = {nullptr, nullptr};
    cudaEvent_t ev_copy[2] = {nullptr, nullptr};
    // batched generation (ptg_batch)
    ptg::FieldPlan* batch_dplans = nullptr;
    long long* batch_dtiles = nullptr;
    unsigned long long* batch_dcounter = nullptr;
    ptg::FieldPlan* batch_hplans = nullptr;  // pinned staging of the plans
    long long* batch_htiles = nullptr;
    int batch_cap = 0;
    cudaEvent_t batch_uploaded = nullptr;
    // request loop
    PtgServer* server = nullptr;
    // map statistics (ptg_box_counts): pyramid bytes and level counters
    uint8_t* stat_buf = nullptr;
    size_t stat_bytes = 0;
    // 2D launch-configuration table filled by ptg_autotune, per [method
    // index][dtype][tile octaves 0..8][16..32-sample-cell octaves 0..2][finer
    // octaves follow]: run width (8 / 16) | 0x80 when the tile octaves are
    // summed at the tile nodes; 0 = untuned
    uint8_t tune[6][2][9][3][2] = {};
    // test hook (ptg_debug_fail_alloc): after alloc_pass more allocations made
    // through ptg_dev_alloc / ptg_pinned_alloc succeed, the next fail_allocs
    // fail as if memory were exhausted
    int alloc_pass = 0;
    int fail_allocs = 0;
};

// Every device (cudaMalloc) and pinned host (cudaMallocHost) allocation the
// library makes goes through these two, so that a test can make them fail on
// the host, without touching the GPU.  cudaErrorMemoryAllocation on failure.
cudaError_t ptg_dev_alloc(ptg_ctx* ctx, void** p, size_t bytes);
cudaError_t ptg_pinned_alloc(ptg_ctx* ctx, void** p, size_t bytes);

// Launch configuration of a 2D polynomial / Perlin field: run width (8 or 16)
// and the number of octaves summed at the tile nodes.  The variant bits of
// desc win, then the context's tuned table, then the fixed rule.
void ptg_pick_config(const ptg_ctx* ctx, const ptg_field_desc* d, int method, int s, int32_t* rw, int32_t* nt);

int ptg_fail(ptg_ctx* ctx, int code, const char* fmt, ...);
int ptg_cuda_fail(ptg_ctx* ctx, cudaError_t e, const char* where);
int ptg_check_desc(ptg_ctx* ctx, const ptg_field_desc* d, int kind, int* spc_log2);
int ptg_make_field_plan(ptg_ctx* ctx, const ptg_field_desc* d, int method, void* out, int s, int64_t band_start,
                        int64_t band_len, ptg::FieldPlan* P);
bool ptg_per_sample(const ptg_field_desc* d, int spc_log2);
// Validates a batch of 2D fields and fills plans[0..n) and the tile prefix
// sums tiles[0..n] with the fields ordered by the batch kernel's code path;
// scratch holds 3 n ints (ptg_batch.cu).
int ptg_build_batch(ptg_ctx* ctx, const ptg_field_desc* descs, void* const* outs, int n, ptg::FieldPlan* plans,
                    long long* tiles, int* scratch, size_t* smem);
bool ptg_fused_ridged(const ptg_field_desc* d, int spc_log2);
int ptg_make_simplex_plan(ptg_ctx* ctx, const ptg_field_desc* d, void* out, int s, int64_t band_start,
                          int64_t band_len, ptg::SimplexPlan* P);
int ptg_make_simplex3_plan(ptg_ctx* ctx, const ptg_field_desc* d, void* out, int64_t band_start, int64_t band_len,
                           ptg::Simplex3Plan* P);
int ptg_make_general_plan(ptg_ctx* ctx, const ptg_field_desc* d, int method, void* out, int s, int64_t band_start,
                          int64_t band_len, ptg::GeneralPlan* P);
int ptg_make_general3_plan(ptg_ctx* ctx, const ptg_field_desc* d, int method, void* out, int64_t band_start,
                           int64_t band_len, ptg::General3Plan* P);
// Rows [band_start, band_start + band_len) of the slowest axis into out (the
// band's first row), as consecutive launches of at most ptg_launch_rows rows.
int ptg_launch_plan(ptg_ctx* ctx, int kind, const ptg_field_desc* d, int s, void* out, int64_t band_start,
                    int64_t band_len, cudaStream_t st);
int64_t ptg_launch_rows(const ptg_field_desc* d);
int ptg_kernel_method(int kind, const ptg_field_desc* d);

void ptg_host_release(ptg_ctx* ctx);
void ptg_batch_release(ptg_ctx* ctx);
void ptg_serve_shutdown(ptg_ctx* ctx);
