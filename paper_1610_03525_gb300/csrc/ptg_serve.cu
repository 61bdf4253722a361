// ptg_serve.cu -- request loop (placeholder until the serving runtime lands).
#include "ptg_internal.h"

void ptg_serve_shutdown(ptg_ctx*) {}

extern "C" {
int ptg_batch(ptg_ctx* ctx, const ptg_field_desc*, void* const*, int32_t, void*)
{
    return ptg_fail(ctx, PTG_ERR_UNSUPPORTED, "batched generation is not built yet");
}
int ptg_submit(ptg_ctx* ctx, const ptg_field_desc*, void*, uint64_t*)
{
    return ptg_fail(ctx, PTG_ERR_UNSUPPORTED, "request loop is not built yet");
}
int ptg_poll(ptg_ctx* ctx, uint64_t, ptg_status*, uint64_t*)
{
    return ptg_fail(ctx, PTG_ERR_UNSUPPORTED, "request loop is not built yet");
}
int ptg_wait(ptg_ctx* ctx, uint64_t, uint64_t)
{
    return ptg_fail(ctx, PTG_ERR_UNSUPPORTED, "request loop is not built yet");
}
}
