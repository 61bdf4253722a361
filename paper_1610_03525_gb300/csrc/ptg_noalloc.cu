// ptg_noalloc.cu -- batched generation that allocates no memory.
//
// Some callers cannot call cudaMalloc: an engine that hands all device memory
// out of its own fixed arena, or a real-time loop in which cudaMalloc's
// implicit device synchronisation would stall every other stream.  For them,
// ptg_batch_noalloc runs the persistent batched kernel with its launch plans
// and work counter in a fixed device array that belongs to this file, instead
// of context-owned allocations.  The caller still owns every output buffer.
//
// The array is file-scope and static: every GPU that loads the library holds
// it until the process exits.  In host code its name only stands in for the
// device object; the kernel is given the address that cudaGetSymbolAddress
// returns for the current device, looked up on the first call per device.
// Every call reuses the same array, so calls that overlap on the GPU race; the
// counter is cleared at each call.
#include <mutex>

#include "ptg_internal.h"

using namespace ptg;

namespace {

constexpr int kNoAllocMaxFields = 256;
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
    FieldPlan plans[kNoAllocMaxFields];
    long long tiles[kNoAllocMaxFields + 1];
    unsigned long long counter;
};
// 256 x sizeof(FieldPlan) + 257 x 8 + 8 bytes: the footprint the header states.
static_assert(sizeof(FieldPlan) == 2016, "FieldPlan changed size: update the stated footprint");
static_assert(sizeof(NoAllocScratch) == 518160, "scratch footprint changed: update the stated size");

// Host staging of the plans.  A pageable source of cudaMemcpyAsync is consumed
// before the call returns, so it is free again right after the copies.
NoAllocScratch g_stage;
std::mutex g_mu;
void* g_dev_addr[kMaxDevices];

}  // namespace

// The scratch array: 256 field plans, their tile offsets and the work counter
// (518,160 bytes, about 506 KiB, on each device that loads the library).
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

extern "C" int ptg_batch_noalloc(ptg_ctx* ctx, const ptg_field_desc* descs, void* const* outs, int32_t n,
                                 void* stream)
{
    if (!ctx) return PTG_ERR_INVALID;
    ctx->err.clear();
    if (n < 0 || n > kNoAllocMaxFields)
        return ptg_fail(ctx, PTG_ERR_INVALID, "ptg_batch_noalloc takes 0 to %d fields, got %d", kNoAllocMaxFields, n);
    if (n > 0 && (!descs || !outs)) return ptg_fail(ctx, PTG_ERR_INVALID, "descs or outs is NULL");
    if (n == 0) return PTG_OK;
    if (ctx->device < 0 || ctx->device >= kMaxDevices)
        return ptg_fail(ctx, PTG_ERR_UNSUPPORTED, "device %d out of range", ctx->device);
    DeviceGuard g(ctx->device);
    if (!g.ok) return ptg_fail(ctx, PTG_ERR_CUDA, "cudaSetDevice failed");
    std::lock_guard<std::mutex> lock(g_mu);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ptg_cuda_fail(ctx, e, "earlier asynchronous error");
    if (!g_dev_addr[ctx->device]) {
        void* addr = nullptr;
        e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
        if (e != cudaSuccess || !addr) return ptg_cuda_fail(ctx, e, "cudaGetSymbolAddress(scratch)");
        g_dev_addr[ctx->device] = addr;
    }
    NoAllocScratch* dev = static_cast<NoAllocScratch*>(g_dev_addr[ctx->device]);

    size_t smem = 0;
    int scratch[3 * kNoAllocMaxFields];
    const int rc = ptg_build_batch(ctx, descs, outs, n, g_stage.plans, g_stage.tiles, scratch, &smem);
    if (rc != PTG_OK) return rc;
    const long long acc = g_stage.tiles[n];

    cudaStream_t st = (cudaStream_t)stream;
    e = cudaMemcpyAsync(dev->plans, g_stage.plans, sizeof(FieldPlan) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dev->tiles, g_stage.tiles, sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(&dev->counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return ptg_cuda_fail(ctx, e, "ptg_batch_noalloc upload");
    if (acc == 0) return PTG_OK;
    const long long resident = (long long)ctx->num_sms * fbm2d_batch_blocks_per_sm(smem);
    const int blocks = (int)(acc < resident ? acc : resident);
    e = launch_fbm2d_batch(dev->plans, dev->tiles, n, &dev->counter, acc, smem, blocks, st);
    return e == cudaSuccess ? PTG_OK : ptg_cuda_fail(ctx, e, "ptg_batch_noalloc launch");
}
