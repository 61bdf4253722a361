// ptg_serve.cu -- request loop behind ptg_submit / ptg_poll / ptg_wait.
//
// Requests (2D or 3D polynomial-noise fields into caller-owned device
// buffers) queue in arrival order.  A request is admitted when a worker slot
// is free and the output bytes of all admitted, unfinished requests stay
// within the context's HBM budget; it is then enqueued on that slot's own
// stream, so requests admitted while others run overlap on the device
// (continuous batching: slots and budget free up as requests finish, and the
// queue advances at every call into the loop).  Timestamps: submit, admit and
// end are taken on the host (end = when the loop sees the request's completion
// event); start = end minus the device time between the two timing events
// recorded around the request's kernels.  Nothing but the kernels and the two
// events enters the slot's stream (no host callbacks, which would stall it).
// There is no background thread and no device spin: progress is made inside
// ptg_submit / ptg_poll / ptg_wait.
//
// NVTX annotations (seen by any NVTX tool attached to the process, free
// otherwise): a pushed range around each ptg_submit ("ptg_submit"), around
// each admission ("ptg_admit") and, inside it, around the enqueue of the
// request's kernels ("ptg_launch"); a mark when the loop sees a request
// complete ("ptg_complete"); and one process-wide range per request from its
// submission to its completion or cancellation ("ptg_request").
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "ptg_internal.h"

namespace {

constexpr int kSlots = 16;
constexpr uint64_t kHoldLimitNs = 5ull * 1000 * 1000 * 1000;  // a held stream is released after 5 s

uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Request {
    uint64_t id = 0;
    ptg_field_desc d{};
    void* out = nullptr;
    int s = 0;
    uint64_t bytes = 0;
    int status = PTG_PENDING;
    uint64_t ts[4] = {0, 0, 0, 0};
    nvtxRangeId_t span = 0;  // NVTX range from submission to completion
};

// A pushed NVTX range for the lifetime of a scope.
struct NvtxScope {
    explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
};

// Test hook: blocks a slot's stream on the host (not on the device) until
// released or kHoldLimitNs passes, to simulate a stalled device.
struct Hold {
    std::atomic<int> held{0};
};
void CUDART_CB on_hold(void* p)
{
    Hold* h = static_cast<Hold*>(p);
    const uint64_t t0 = now_ns();
    while (h->held.load() && now_ns() - t0 < kHoldLimitNs) std::this_thread::sleep_for(std::chrono::microseconds(200));
}

}  // namespace

struct PtgServer {
    std::mutex mu;
    std::deque<Request*> pending;
    std::unordered_map<uint64_t, Request*> reqs;
    Request* running[kSlots] = {};
    cudaStream_t streams[kSlots] = {};
    cudaEvent_t begin[kSlots] = {};  // timing events around each slot's current request
    cudaEvent_t done[kSlots] = {};
    uint64_t admitted = 0;
    uint64_t next_id = 1;
    Hold hold;
    int hold_next = 0;
};

namespace {

PtgServer* server(ptg_ctx* ctx)
{
    if (ctx->server) return ctx->server;
    PtgServer* S = new (std::nothrow) PtgServer();
    if (!S) return nullptr;
    for (int k = 0; k < kSlots; ++k) {
        if (cudaStreamCreateWithFlags(&S->streams[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreate(&S->begin[k]) != cudaSuccess || cudaEventCreate(&S->done[k]) != cudaSuccess) {
            cudaGetLastError();
            for (int j = 0; j <= k; ++j) {
                if (S->streams[j]) cudaStreamDestroy(S->streams[j]);
                if (S->begin[j]) cudaEventDestroy(S->begin[j]);
                if (S->done[j]) cudaEventDestroy(S->done[j]);
            }
            delete S;
            return nullptr;
        }
    }
    ctx->server = S;
    return S;
}

void finish(PtgServer* S, int slot, int status)
{
    Request* r = S->running[slot];
    nvtxMarkA("ptg_complete");
    nvtxRangeEnd(r->span);
    r->status = status;
    r->ts[3] = now_ns();
    float ms = 0.0f;
    uint64_t dev_ns = 0;
    if (status == PTG_OK && cudaEventElapsedTime(&ms, S->begin[slot], S->done[slot]) == cudaSuccess && ms > 0.0f)
        dev_ns = (uint64_t)((double)ms * 1e6);
    cudaGetLastError();
    const uint64_t span = r->ts[3] - r->ts[1];
    r->ts[2] = r->ts[3] - (dev_ns < span ? dev_ns : span);
    S->admitted -= r->bytes;
    S->running[slot] = nullptr;
}

// Retire finished requests, then admit queued ones in arrival order.
void progress(ptg_ctx* ctx, PtgServer* S)
{
    for (int k = 0; k < kSlots; ++k) {
        if (!S->running[k]) continue;
        const cudaError_t q = cudaEventQuery(S->done[k]);
        if (q == cudaSuccess) finish(S, k, PTG_OK);
        else if (q != cudaErrorNotReady) {
            cudaGetLastError();
            finish(S, k, PTG_ERR_CUDA);
        }
    }
    while (!S->pending.empty()) {
        Request* r = S->pending.front();
        int slot = -1;
        for (int k = 0; k < kSlots; ++k)
            if (!S->running[k]) {
                slot = k;
                break;
            }
        if (slot < 0 || S->admitted + r->bytes > ctx->budget) break;
        NvtxScope admit("ptg_admit");
        S->pending.pop_front();
        r->ts[1] = now_ns();
        cudaStream_t st = S->streams[slot];
        if (S->hold_next) {
            S->hold_next = 0;
            cudaLaunchHostFunc(st, on_hold, &S->hold);
        }
        cudaEventRecord(S->begin[slot], st);
        const int64_t slow = r->d.dims == 3 ? r->d.size[2] : r->d.size[1];
        int rc;
        {
            NvtxScope launch("ptg_launch");
            rc = ptg_launch_plan(ctx, kKindField, &r->d, r->s, r->out, 0, slow, st);
        }
        if (rc != PTG_OK) {
            r->status = rc;
            r->ts[2] = r->ts[3] = now_ns();
            nvtxMarkA("ptg_complete");
            nvtxRangeEnd(r->span);
            continue;
        }
        cudaEventRecord(S->done[slot], st);
        S->running[slot] = r;
        S->admitted += r->bytes;
    }
}

}  // namespace

void ptg_serve_shutdown(ptg_ctx* ctx)
{
    PtgServer* S = ctx->server;
    if (!S) return;
    S->hold.held.store(0);
    for (int k = 0; k < kSlots; ++k) {
        cudaStreamSynchronize(S->streams[k]);
        cudaStreamDestroy(S->streams[k]);
        cudaEventDestroy(S->begin[k]);
        cudaEventDestroy(S->done[k]);
    }
    for (auto& kv : S->reqs) delete kv.second;
    delete S;
    ctx->server = nullptr;
}

extern "C" {

int ptg_submit(ptg_ctx* ctx, const ptg_field_desc* d, void* out, uint64_t* req_id)
{
    NvtxScope scope("ptg_submit");
    if (!ctx) return PTG_ERR_INVALID;
    ctx->err.clear();
    if (!req_id) return ptg_fail(ctx, PTG_ERR_INVALID, "req_id is NULL");
    int s = 0;
    int rc = ptg_check_desc(ctx, d, kKindField, &s);
    if (rc != PTG_OK) return rc;
    if (!out) return ptg_fail(ctx, PTG_ERR_INVALID, "out is NULL");
    uint64_t bytes = d->dtype == PTG_F16 ? 2 : 4;
    for (int k = 0; k < d->dims; ++k) bytes *= (uint64_t)d->size[k];
    if (bytes > ctx->budget)
        return ptg_fail(ctx, PTG_ERR_BUDGET, "request needs %llu bytes, budget is %llu", (unsigned long long)bytes,
                        (unsigned long long)ctx->budget);
    DeviceGuard g(ctx->device);
    PtgServer* S = server(ctx);
    if (!S) return ptg_fail(ctx, PTG_ERR_NOMEM, "cannot create the request loop");
    std::lock_guard<std::mutex> lock(S->mu);
    Request* r = new (std::nothrow) Request();
    if (!r) return ptg_fail(ctx, PTG_ERR_NOMEM, "out of host memory");
    r->id = S->next_id++;
    r->d = *d;
    r->out = out;
    r->s = s;
    r->bytes = bytes;
    r->ts[0] = now_ns();
    r->span = nvtxRangeStartA("ptg_request");
    S->reqs[r->id] = r;
    S->pending.push_back(r);
    *req_id = r->id;
    progress(ctx, S);
    return PTG_OK;
}

int ptg_poll(ptg_ctx* ctx, uint64_t req_id, ptg_status* st, uint64_t ts_ns[4])
{
    if (!ctx) return PTG_ERR_INVALID;
    PtgServer* S = ctx->server;
    if (!S) return ptg_fail(ctx, PTG_ERR_INVALID, "unknown request %llu", (unsigned long long)req_id);
    DeviceGuard g(ctx->device);
    std::lock_guard<std::mutex> lock(S->mu);
    progress(ctx, S);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return ptg_fail(ctx, PTG_ERR_INVALID, "unknown request %llu", (unsigned long long)req_id);
    Request* r = it->second;
    if (st) *st = (ptg_status)r->status;
    if (ts_ns) memcpy(ts_ns, r->ts, sizeof r->ts);
    if (r->status != PTG_PENDING) {  // final status delivered: release the record
        S->reqs.erase(it);
        delete r;
    }
    return PTG_OK;
}

int ptg_wait(ptg_ctx* ctx, uint64_t req_id, uint64_t timeout_ns)
{
    if (!ctx) return PTG_ERR_INVALID;
    PtgServer* S = ctx->server;
    if (!S) return ptg_fail(ctx, PTG_ERR_INVALID, "unknown request %llu", (unsigned long long)req_id);
    DeviceGuard g(ctx->device);
    const uint64_t deadline = now_ns() + timeout_ns;
    for (;;) {
        {
            std::lock_guard<std::mutex> lock(S->mu);
            progress(ctx, S);
            auto it = S->reqs.find(req_id);
            if (it == S->reqs.end())
                return ptg_fail(ctx, PTG_ERR_INVALID, "unknown request %llu", (unsigned long long)req_id);
            if (it->second->status != PTG_PENDING) return it->second->status;
        }
        if (now_ns() >= deadline) return ptg_fail(ctx, PTG_ERR_TIMEOUT, "request %llu still running",
                                                  (unsigned long long)req_id);
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

int ptg_cancel(ptg_ctx* ctx, uint64_t req_id)
{
    if (!ctx) return PTG_ERR_INVALID;
    PtgServer* S = ctx->server;
    if (!S) return ptg_fail(ctx, PTG_ERR_INVALID, "unknown request");
    std::lock_guard<std::mutex> lock(S->mu);
    for (auto it = S->pending.begin(); it != S->pending.end(); ++it) {
        if ((*it)->id == req_id) {
            nvtxRangeEnd((*it)->span);
            (*it)->status = PTG_ERR_CANCELLED;
            S->pending.erase(it);
            return PTG_OK;
        }
    }
    return ptg_fail(ctx, PTG_ERR_INVALID, "request %llu is not queued", (unsigned long long)req_id);
}

int ptg_debug_hold(ptg_ctx* ctx, int32_t hold)
{
    if (!ctx) return PTG_ERR_INVALID;
    DeviceGuard g(ctx->device);
    PtgServer* S = server(ctx);
    if (!S) return PTG_ERR_NOMEM;
    std::lock_guard<std::mutex> lock(S->mu);
    if (hold) {
        S->hold.held.store(1);
        S->hold_next = 1;
    } else {
        S->hold.held.store(0);
    }
    return PTG_OK;
}

}  // extern "C"
