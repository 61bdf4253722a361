// ptg_host.cu -- generation into host memory.  The field is cut into bands
// along its slowest axis (whole tile rows / planes); band b is generated into
// one of two context-owned device staging buffers while band b-1 is copied to
// the host on a second stream, so the device-to-host copy hides the compute.
#include <cstring>

#include "ptg_internal.h"

namespace {
constexpr size_t kBandBytes = size_t{32} << 20;  // target bytes per band
}

void ptg_host_release(ptg_ctx* ctx)
{
    if (ctx->stage) cudaFree(ctx->stage);
    ctx->stage = nullptr;
    ctx->stage_bytes = 0;
    for (int b = 0; b < 2; ++b) {
        if (ctx->ev_gen[b]) cudaEventDestroy(ctx->ev_gen[b]);
        if (ctx->ev_copy[b]) cudaEventDestroy(ctx->ev_copy[b]);
        ctx->ev_gen[b] = ctx->ev_copy[b] = nullptr;
    }
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    ctx->copy_stream = nullptr;
}

extern "C" int ptg_generate_host(ptg_ctx* ctx, const ptg_field_desc* d, int32_t method, void* host_out)
{
    if (!ctx) return PTG_ERR_INVALID;
    ctx->err.clear();
    if (method < 0 || method > 2) return ptg_fail(ctx, PTG_ERR_INVALID, "method must be 0, 1 or 2");
    const int kind = method == 0 ? kKindField : (method == 1 ? kKindPerlin : kKindSimplex);
    int s = 0;
    int rc = ptg_check_desc(ctx, d, kind, &s);
    if (rc != PTG_OK) return rc;
    if (!host_out) return ptg_fail(ctx, PTG_ERR_INVALID, "host_out is NULL");
    DeviceGuard g(ctx->device);
    if (!g.ok) return ptg_fail(ctx, PTG_ERR_CUDA, "cudaSetDevice failed");
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ptg_cuda_fail(ctx, e, "earlier asynchronous error");

    const bool is3d = d->dims == 3;
    const size_t esz = d->dtype == PTG_F16 ? 2 : 4;
    const size_t slab = (size_t)d->size[0] * esz * (is3d ? (size_t)d->size[1] : 1);  // bytes per row / plane
    const int64_t total = is3d ? d->size[2] : d->size[1];
    const int64_t tile = is3d ? ptg::kTile3dZ : ptg::kTile2dY;
    int64_t band = (int64_t)(kBandBytes / slab) / tile * tile;
    if (band < tile) band = tile;
    if (band > ptg_launch_rows(d)) band = ptg_launch_rows(d);  // one launch a band
    if (band > total) band = total;
    const size_t need = 2 * (size_t)band * slab;
    if (ctx->stage_bytes < need) {
        if (ctx->stage) cudaFree(ctx->stage);
        ctx->stage = nullptr;
        ctx->stage_bytes = 0;
        if (ptg_dev_alloc(ctx, &ctx->stage, need) != cudaSuccess)
            return ptg_fail(ctx, PTG_ERR_NOMEM, "cannot allocate %zu bytes of staging", need);
        ctx->stage_bytes = need;
    }
    if (!ctx->copy_stream) {
        if (cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
            return ptg_fail(ctx, PTG_ERR_CUDA, "cannot create copy stream");
        for (int b = 0; b < 2; ++b) {
            cudaEventCreateWithFlags(&ctx->ev_gen[b], cudaEventDisableTiming);
            cudaEventCreateWithFlags(&ctx->ev_copy[b], cudaEventDisableTiming);
        }
    }
    char* host = static_cast<char*>(host_out);
    int64_t nb = 0;
    for (int64_t start = 0; start < total; start += band, ++nb) {
        const int64_t len = (total - start) < band ? (total - start) : band;
        const int b = (int)(nb & 1);
        char* buf = static_cast<char*>(ctx->stage) + (size_t)b * (size_t)band * slab;
        if (nb >= 2) cudaStreamWaitEvent(ctx->stream, ctx->ev_copy[b], 0);
        rc = ptg_launch_plan(ctx, kind, d, s, buf, start, len, ctx->stream);
        if (rc != PTG_OK) {
            cudaStreamSynchronize(ctx->copy_stream);
            return rc;
        }
        cudaEventRecord(ctx->ev_gen[b], ctx->stream);
        cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_gen[b], 0);
        e = cudaMemcpyAsync(host + (size_t)start * slab, buf, (size_t)len * slab, cudaMemcpyDeviceToHost,
                            ctx->copy_stream);
        if (e != cudaSuccess) {
            cudaStreamSynchronize(ctx->copy_stream);
            return ptg_cuda_fail(ctx, e, "device-to-host copy");
        }
        cudaEventRecord(ctx->ev_copy[b], ctx->copy_stream);
    }
    e = cudaStreamSynchronize(ctx->copy_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? PTG_OK : ptg_cuda_fail(ctx, e, "host generation");
}
