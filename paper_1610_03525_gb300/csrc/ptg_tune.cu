// ptg_tune.cu -- choice of the 2D thread shape (8 x 4 or 16 x 2 samples per
// thread) and the autotuner that measures it (ptg_autotune).
//
// The key of a choice is what decides the relative cost of the two shapes:
// the kernel method, the output dtype, n16 = the number of octaves whose
// cells are at least 16 samples wide (the octaves the wider run makes
// cheaper; capped at 8) and whether finer octaves follow (where the wider run
// pays for an 8-sample-cell octave evaluated column by column).  The field's
// size and offset are not part of the key, so every chunk of a field takes
// the same shape as the whole and mosaics stay bit-identical.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ptg_internal.h"

using namespace ptg;

namespace {

constexpr int kTuneMaxN16 = 8;
constexpr int kTuneSide = 4096;  // samples per side of the timed field
const int kMethods[6] = {kC1, kC2, kPaperGauge, kZeroGrad, kPerlinS5, kPerlinS3};

int method_index(int method)
{
    for (int m = 0; m < 6; ++m)
        if (kMethods[m] == method) return m;
    return 0;
}

struct TuneKey {
    int n16, tail;
};

TuneKey tune_key(const ptg_field_desc* d, int s)
{
    int n16 = s - 3;
    n16 = n16 < 0 ? 0 : (n16 < d->octaves ? n16 : d->octaves);
    TuneKey k;
    k.tail = d->octaves > n16 ? 1 : 0;
    k.n16 = n16 < kTuneMaxN16 ? n16 : kTuneMaxN16;
    return k;
}

// Untuned choice: the wider run from a per-method number of 16-wide run
// octaves on.  The thresholds are where 16 x 2 overtook 8 x 4 in the tuner's
// timings on a GB300 (4096^2 fields, FP32): the wider run saves work in every
// coarse octave but costs more in the 8-sample-cell octave, in the Lagrange
// fill (16 - d - 1 columns a row instead of 8 - d - 1) and in the stores.
int default_rw(int method, const TuneKey& k)
{
    int n = 5;
    switch (method) {
    case kC2: n = 6; break;
    case kPaperGauge: n = 4; break;
    case kZeroGrad: n = 7; break;
    case kPerlinS5: n = 6; break;
    case kPerlinS3: n = 4; break;
    default: break;
    }
    return k.n16 >= n ? 16 : 8;
}

bool device_identity(int device, std::string* name, int* sms)
{
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return false;
    *name = prop.name;
    *sms = prop.multiProcessorCount;
    return true;
}

// Cache file: {"version": 1, "device": "...", "sms": N, "entries": [{"method":
// M, "dtype": T, "n16": K, "tail": 0|1, "rw": 8|16, "us_rw8": x, "us_rw16": y}, ...]}
// Returns 1 loaded, 0 absent or written for another device, -1 malformed.
int load_cache(ptg_ctx* ctx, const char* path, const std::string& name, int sms)
{
    FILE* f = std::fopen(path, "rb");
    if (!f) return 0;
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
    std::fclose(f);
    int version = 0, fsms = 0;
    const char* v = std::strstr(text.c_str(), "\"version\":");
    const char* dv = std::strstr(text.c_str(), "\"device\": \"");
    const char* sv = std::strstr(text.c_str(), "\"sms\":");
    if (!v || !dv || !sv || std::sscanf(v, "\"version\": %d", &version) != 1 ||
        std::sscanf(sv, "\"sms\": %d", &fsms) != 1 || version != 1)
        return -1;
    dv += std::strlen("\"device\": \"");
    const char* de = std::strchr(dv, '"');
    if (!de) return -1;
    if (std::string(dv, de) != name || fsms != sms) return 0;
    uint8_t table[6][2][9][2] = {};
    int count = 0;
    for (const char* p = std::strstr(de, "{\"method\":"); p; p = std::strstr(p + 1, "{\"method\":")) {
        int m = 0, dt = 0, n16 = 0, tail = 0, rw = 0;
        if (std::sscanf(p, "{\"method\": %d, \"dtype\": %d, \"n16\": %d, \"tail\": %d, \"rw\": %d", &m, &dt, &n16,
                        &tail, &rw) != 5)
            return -1;
        int mi = -1;
        for (int q = 0; q < 6; ++q)
            if (kMethods[q] == m) mi = q;
        if (mi < 0 || dt < 0 || dt > 1 || n16 < 0 || n16 > kTuneMaxN16 || tail < 0 || tail > 1 ||
            (rw != 8 && rw != 16))
            return -1;
        table[mi][dt][n16][tail] = (uint8_t)rw;
        ++count;
    }
    if (count == 0) return -1;
    std::memcpy(ctx->tune_rw, table, sizeof table);
    return 1;
}

struct Timed {
    int method, dtype, n16, tail, rw;
    float us8, us16;
};

bool write_cache(const char* path, const std::string& name, int sms, int reps, const std::vector<Timed>& rows)
{
    FILE* f = std::fopen(path, "wb");
    if (!f) return false;
    std::fprintf(f, "{\"version\": 1, \"device\": \"%s\", \"sms\": %d, \"field\": [%d, %d], \"reps\": %d,\n",
                 name.c_str(), sms, kTuneSide, kTuneSide, reps);
    std::fprintf(f, " \"entries\": [\n");
    for (size_t r = 0; r < rows.size(); ++r) {
        const Timed& t = rows[r];
        std::fprintf(f,
                     "  {\"method\": %d, \"dtype\": %d, \"n16\": %d, \"tail\": %d, \"rw\": %d, \"us_rw8\": %.3f, "
                     "\"us_rw16\": %.3f}%s\n",
                     t.method, t.dtype, t.n16, t.tail, t.rw, t.us8, t.us16, r + 1 < rows.size() ? "," : "");
    }
    std::fprintf(f, " ]}\n");
    return std::fclose(f) == 0;
}

float median(std::vector<float> v)
{
    std::sort(v.begin(), v.end());
    return v.empty() ? 0.0f : v[v.size() / 2];
}

}  // namespace

int ptg_pick_rw(const ptg_ctx* ctx, const ptg_field_desc* d, int method, int s)
{
    const int shape = d->variant & ~0xff;
    if (shape == PTG_SHAPE_8X4) return 8;
    if (shape == PTG_SHAPE_16X2) return 16;
    const TuneKey k = tune_key(d, s);
    const int dt = d->dtype == PTG_F16 ? 1 : 0;
    const int tuned = ctx ? ctx->tune_rw[method_index(method)][dt][k.n16][k.tail] : 0;
    return tuned ? tuned : default_rw(method, k);
}

extern "C" {

int ptg_thread_shape(ptg_ctx* ctx, const ptg_field_desc* desc, int32_t method, int32_t* rw)
{
    if (!ctx || !rw) return PTG_ERR_INVALID;
    ctx->err.clear();
    if (method != 0 && method != 1) return ptg_fail(ctx, PTG_ERR_INVALID, "method must be 0 (field) or 1 (Perlin)");
    const int kind = method == 1 ? kKindPerlin : kKindField;
    int s = 0;
    const int rc = ptg_check_desc(ctx, desc, kind, &s);
    if (rc != PTG_OK) return rc;
    *rw = desc->dims == 2 ? ptg_pick_rw(ctx, desc, ptg_kernel_method(kind, desc), s) : 8;
    return PTG_OK;
}

int ptg_autotune(ptg_ctx* ctx, int32_t effort, const char* cache_path)
{
    if (!ctx) return PTG_ERR_INVALID;
    ctx->err.clear();
    if (effort < 0 || effort > 100) return ptg_fail(ctx, PTG_ERR_INVALID, "effort must be in [0, 100]");
    const int reps = effort ? effort : 5;
    DeviceGuard g(ctx->device);
    if (!g.ok) return ptg_fail(ctx, PTG_ERR_CUDA, "cannot select device %d", ctx->device);
    std::string name;
    int sms = 0;
    if (!device_identity(ctx->device, &name, &sms)) return ptg_fail(ctx, PTG_ERR_CUDA, "cudaGetDeviceProperties");
    if (cache_path) {
        const int lc = load_cache(ctx, cache_path, name, sms);
        if (lc > 0) return PTG_OK;
        if (lc < 0) return ptg_fail(ctx, PTG_ERR_INVALID, "autotune cache %s is not a thread-shape table", cache_path);
    }

    void* out = nullptr;
    cudaError_t e = cudaMalloc(&out, (size_t)kTuneSide * kTuneSide * sizeof(float));
    if (e != cudaSuccess) return ptg_cuda_fail(ctx, e, "cudaMalloc (autotune field)");
    std::vector<cudaEvent_t> ev(4 * (size_t)reps, nullptr);
    for (auto& x : ev)
        if (e == cudaSuccess) e = cudaEventCreate(&x);
    uint8_t table[6][2][9][2] = {};
    std::vector<Timed> rows;
    for (int mi = 0; mi < 6 && e == cudaSuccess; ++mi) {
        const int method = kMethods[mi];
        for (int dt = 0; dt < 2 && e == cudaSuccess; ++dt)
            for (int n16 = 0; n16 <= kTuneMaxN16 && e == cudaSuccess; ++n16)
                for (int tail = 0; tail < 2 && e == cudaSuccess; ++tail) {
                    if (n16 == 0 && tail == 0) continue;  // no octave at all
                    ptg_field_desc d;
                    std::memset(&d, 0, sizeof d);
                    d.struct_size = sizeof d;
                    d.dims = 2;
                    d.size[0] = d.size[1] = kTuneSide;
                    d.size[2] = 1;
                    d.spc = int64_t{1} << (n16 + 3);
                    d.octaves = n16 + (tail ? 4 : 0);
                    d.smoothness = method == kC2 ? PTG_C2 : method == kPaperGauge ? PTG_PAPER_D2M1N3
                                 : method == kZeroGrad ? PTG_ZERO_GRADIENT : PTG_C1;
                    d.persistence = 0.5f;
                    d.lacunarity = 2.0f;
                    d.grad_weight = 1.0f;
                    d.dtype = dt;
                    FieldPlan P[2];
                    int rc = PTG_OK;
                    for (int v = 0; v < 2 && rc == PTG_OK; ++v) {
                        d.variant = (method == kPerlinS3 ? PTG_PERLIN_S3 : 0) | (v ? PTG_SHAPE_16X2 : PTG_SHAPE_8X4);
                        rc = ptg_make_field_plan(ctx, &d, method, out, n16 + 3, 0, kTuneSide, &P[v]);
                    }
                    if (rc != PTG_OK) {
                        cudaFree(out);
                        for (auto& x : ev)
                            if (x) cudaEventDestroy(x);
                        return rc;
                    }
                    for (int w = 0; w < 2 && e == cudaSuccess; ++w)  // warm-up
                        for (int v = 0; v < 2 && e == cudaSuccess; ++v)
                            e = launch_fbm2d(P[v], method, n16 + 3, ctx->stream);
                    for (int r = 0; r < reps && e == cudaSuccess; ++r)
                        for (int v = 0; v < 2 && e == cudaSuccess; ++v) {
                            cudaEventRecord(ev[4 * r + 2 * v], ctx->stream);
                            e = launch_fbm2d(P[v], method, n16 + 3, ctx->stream);
                            cudaEventRecord(ev[4 * r + 2 * v + 1], ctx->stream);
                        }
                    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
                    std::vector<float> t8, t16;
                    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
                        float a = 0.0f, b = 0.0f;
                        e = cudaEventElapsedTime(&a, ev[4 * r], ev[4 * r + 1]);
                        if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[4 * r + 2], ev[4 * r + 3]);
                        t8.push_back(a * 1e3f);
                        t16.push_back(b * 1e3f);
                    }
                    if (e != cudaSuccess) break;
                    Timed t;
                    t.method = method;
                    t.dtype = dt;
                    t.n16 = n16;
                    t.tail = tail;
                    t.us8 = median(t8);
                    t.us16 = median(t16);
                    t.rw = t.us16 < t.us8 ? 16 : 8;
                    table[mi][dt][n16][tail] = (uint8_t)t.rw;
                    rows.push_back(t);
                }
    }
    for (auto& x : ev)
        if (x) cudaEventDestroy(x);
    cudaFree(out);
    if (e != cudaSuccess) return ptg_cuda_fail(ctx, e, "autotune");
    std::memcpy(ctx->tune_rw, table, sizeof table);
    if (cache_path && !write_cache(cache_path, name, sms, reps, rows))
        return ptg_fail(ctx, PTG_ERR_INVALID, "cannot write autotune cache %s", cache_path);
    return PTG_OK;
}

}  // extern "C"
