// ptg_tune.cu -- the 2D launch configuration (thread shape 8 x 4 or 16 x 2;
// coarse octaves per run or summed at the tile nodes) and the autotuner that
// measures it (ptg_autotune).
//
// The key of a choice is what decides the relative cost of the variants: the
// kernel method, the output dtype and the octave structure -- nt = octaves
// whose cells cover a whole 64-sample tile (capped at 8), mid = octaves with
// cells of 16 or 32 samples (0..2), and whether finer octaves follow (cells
// of 8 samples and less, where the 16-wide run pays more).  The field's size
// and offset are not part of the key, so every chunk of a field takes the
// same configuration as the whole and mosaics stay bit-identical.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ptg_internal.h"

using namespace ptg;

namespace {

constexpr int kTuneMaxNt = 8;
constexpr int kTuneSide = 8192;  // samples per side of the timed field (the 2D headline size)
const int kMethods[6] = {kC1, kC2, kPaperGauge, kZeroGrad, kPerlinS5, kPerlinS3};
constexpr uint8_t kTileBit = 0x80;

int method_index(int method)
{
    for (int m = 0; m < 6; ++m)
        if (kMethods[m] == method) return m;
    return 0;
}

bool tile_capable(int method) { return method != kC2 && method != kPerlinS5; }  // degree <= 4

struct TuneKey {
    int nt_all;   // octaves with cells >= 64 samples (uncapped)
    int nt, mid, tail;
};

TuneKey tune_key(const ptg_field_desc* d, int s)
{
    const int N = d->octaves;
    int n16 = s - 3, n64 = s - 5;
    n16 = n16 < 0 ? 0 : (n16 < N ? n16 : N);
    n64 = n64 < 0 ? 0 : (n64 < N ? n64 : N);
    TuneKey k;
    k.nt_all = n64;
    k.nt = n64 < kTuneMaxNt ? n64 : kTuneMaxNt;
    k.mid = n16 - n64;
    k.tail = N > n16 ? 1 : 0;
    return k;
}

// Untuned choice, from the tuner's timings on a GB300 (FP32): the tile nodes
// once at least three octaves cover the tile and five have cells of 16
// samples or more (the CTA-wide pass and its extra barrier cost about one
// octave's work), and then the 8 x 4 shape; without them, the 16-wide run for
// the degree-5 and -6 models once six octaves have cells of 16 samples or
// more (it saves work in each of them but costs more in the 8-sample-cell
// octave, in the Lagrange fill and in the stores).
uint8_t default_config(int method, const TuneKey& k)
{
    if (tile_capable(method) && k.nt >= 3 && k.nt + k.mid >= 5) return (uint8_t)(8 | kTileBit);
    const bool wide = (method == kC2 || method == kPerlinS5) && k.nt + k.mid >= 6;
    return wide ? 16 : 8;
}

bool device_identity(int device, std::string* name, int* sms)
{
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return false;
    *name = prop.name;
    *sms = prop.multiProcessorCount;
    return true;
}

typedef uint8_t Table[6][2][kTuneMaxNt + 1][3][2];

// Cache file: {"version": 2, "device": "...", "sms": N, ..., "entries":
// [{"method": M, "dtype": T, "nt": K, "mid": J, "tail": 0|1, "rw": 8|16,
// "tile": 0|1, "us": [rw8, rw16, rw8 tile, rw16 tile]}, ...]} (-1 = not timed).
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
        std::sscanf(sv, "\"sms\": %d", &fsms) != 1)
        return -1;
    dv += std::strlen("\"device\": \"");
    const char* de = std::strchr(dv, '"');
    if (!de) return -1;
    if (version != 2 || std::string(dv, de) != name || fsms != sms) return 0;  // re-time
    Table table = {};
    int count = 0;
    for (const char* p = std::strstr(de, "{\"method\":"); p; p = std::strstr(p + 1, "{\"method\":")) {
        int m = 0, dt = 0, nt = 0, mid = 0, tail = 0, rw = 0, tile = 0;
        if (std::sscanf(p, "{\"method\": %d, \"dtype\": %d, \"nt\": %d, \"mid\": %d, \"tail\": %d, \"rw\": %d, \"tile\": %d",
                        &m, &dt, &nt, &mid, &tail, &rw, &tile) != 7)
            return -1;
        int mi = -1;
        for (int q = 0; q < 6; ++q)
            if (kMethods[q] == m) mi = q;
        if (mi < 0 || dt < 0 || dt > 1 || nt < 0 || nt > kTuneMaxNt || mid < 0 || mid > 2 || tail < 0 ||
            tail > 1 || (rw != 8 && rw != 16) || tile < 0 || tile > 1 || (tile && !tile_capable(m)))
            return -1;
        table[mi][dt][nt][mid][tail] = (uint8_t)(rw | (tile ? kTileBit : 0));
        ++count;
    }
    if (count == 0) return -1;
    std::memcpy(ctx->tune, table, sizeof table);
    return 1;
}

struct Timed {
    int method, dtype, nt, mid, tail;
    uint8_t best;
    float us[4];  // rw8, rw16, rw8 + tile nodes, rw16 + tile nodes (-1 = not timed)
};

bool write_cache(const char* path, const std::string& name, int sms, int reps, const std::vector<Timed>& rows)
{
    FILE* f = std::fopen(path, "wb");
    if (!f) return false;
    std::fprintf(f, "{\"version\": 2, \"device\": \"%s\", \"sms\": %d, \"field\": [%d, %d], \"reps\": %d,\n",
                 name.c_str(), sms, kTuneSide, kTuneSide, reps);
    std::fprintf(f, " \"entries\": [\n");
    for (size_t r = 0; r < rows.size(); ++r) {
        const Timed& t = rows[r];
        std::fprintf(f,
                     "  {\"method\": %d, \"dtype\": %d, \"nt\": %d, \"mid\": %d, \"tail\": %d, \"rw\": %d, "
                     "\"tile\": %d, \"us\": [%.3f, %.3f, %.3f, %.3f]}%s\n",
                     t.method, t.dtype, t.nt, t.mid, t.tail, t.best & 0x7f, (t.best & kTileBit) ? 1 : 0, t.us[0],
                     t.us[1], t.us[2], t.us[3], r + 1 < rows.size() ? "," : "");
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

void ptg_pick_config(const ptg_ctx* ctx, const ptg_field_desc* d, int method, int s, int32_t* rw, int32_t* nt)
{
    const TuneKey k = tune_key(d, s);
    const int dt = d->dtype == PTG_F16 ? 1 : 0;
    uint8_t c = ctx ? ctx->tune[method_index(method)][dt][k.nt][k.mid][k.tail] : 0;
    if (!c) c = default_config(method, k);
    const int shape = d->variant & 0x300, coarse = d->variant & 0xc00;
    if (shape == PTG_SHAPE_8X4) c = (uint8_t)((c & kTileBit) | 8);
    if (shape == PTG_SHAPE_16X2) c = (uint8_t)((c & kTileBit) | 16);
    if (coarse == PTG_COARSE_RUNS) c &= (uint8_t)~kTileBit;
    if (coarse == PTG_COARSE_TILE) c |= kTileBit;
    if (!tile_capable(method)) c &= (uint8_t)~kTileBit;
    *rw = c & 0x7f;
    *nt = (c & kTileBit) ? k.nt_all : 0;
}

extern "C" {

int ptg_launch_config(ptg_ctx* ctx, const ptg_field_desc* desc, int32_t method, int32_t* rw, int32_t* tile_octaves)
{
    if (!ctx) return PTG_ERR_INVALID;
    ctx->err.clear();
    if (method != 0 && method != 1) return ptg_fail(ctx, PTG_ERR_INVALID, "method must be 0 (field) or 1 (Perlin)");
    const int kind = method == 1 ? kKindPerlin : kKindField;
    int s = 0;
    const int rc = ptg_check_desc(ctx, desc, kind, &s);
    if (rc != PTG_OK) return rc;
    int32_t w = 8, t = 0;  // (the per-sample generator of other spc and frequency ratios has no choice)
    if (desc->dims == 2 && s >= 0 && desc->lacunarity == 2.0f)
        ptg_pick_config(ctx, desc, ptg_kernel_method(kind, desc), s, &w, &t);
    if (rw) *rw = w;
    if (tile_octaves) *tile_octaves = t;
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
        if (lc < 0) return ptg_fail(ctx, PTG_ERR_INVALID, "autotune cache %s is not a launch-config table", cache_path);
    }

    void* out = nullptr;
    cudaError_t e = ptg_dev_alloc(ctx, &out, (size_t)kTuneSide * kTuneSide * sizeof(float));
    if (e != cudaSuccess) return ptg_fail(ctx, PTG_ERR_NOMEM, "cannot allocate the autotune field");
    std::vector<cudaEvent_t> ev(8 * (size_t)reps, nullptr);
    for (auto& x : ev)
        if (e == cudaSuccess) e = cudaEventCreate(&x);
    Table table = {};
    std::vector<Timed> rows;
    int rc = PTG_OK;
    for (int mi = 0; mi < 6 && e == cudaSuccess && rc == PTG_OK; ++mi) {
        const int method = kMethods[mi];
        for (int dt = 0; dt < 2 && e == cudaSuccess && rc == PTG_OK; ++dt)
            for (int nt = 0; nt <= kTuneMaxNt && e == cudaSuccess && rc == PTG_OK; ++nt)
                for (int mid = 0; mid < 3 && e == cudaSuccess && rc == PTG_OK; ++mid)
                    for (int tail = 0; tail < 2 && e == cudaSuccess && rc == PTG_OK; ++tail) {
                        // a field with this octave structure: with finer octaves, the
                        // structure fixes spc (mid < 2 only without tile octaves) and
                        // four finer octaves follow; without, N = nt + mid, spc = 2^(nt+5)
                        int s = 0, N = 0;
                        if (tail) {
                            if (nt > 0 && mid < 2) continue;
                            s = nt > 0 ? nt + 5 : mid + 3;
                            N = nt + mid + 4;
                        } else {
                            s = nt + 5;
                            N = nt + mid;
                            if (N < 1) continue;
                        }
                        ptg_field_desc d;
                        std::memset(&d, 0, sizeof d);
                        d.struct_size = sizeof d;
                        d.dims = 2;
                        d.size[0] = d.size[1] = kTuneSide;
                        d.size[2] = 1;
                        d.spc = int64_t{1} << s;
                        d.octaves = N;
                        d.smoothness = method == kC2 ? PTG_C2 : method == kPaperGauge ? PTG_PAPER_D2M1N3
                                     : method == kZeroGrad ? PTG_ZERO_GRADIENT : PTG_C1;
                        d.persistence = 0.5f;
                        d.lacunarity = 2.0f;
                        d.grad_weight = 1.0f;
                        d.dtype = dt;
                        const int nv = (nt > 0 && tile_capable(method)) ? 4 : 2;
                        FieldPlan P[4];
                        for (int v = 0; v < nv && rc == PTG_OK; ++v) {
                            d.variant = (method == kPerlinS3 ? PTG_PERLIN_S3 : 0) |
                                        ((v & 1) ? PTG_SHAPE_16X2 : PTG_SHAPE_8X4) |
                                        ((v & 2) ? PTG_COARSE_TILE : PTG_COARSE_RUNS);
                            rc = ptg_make_field_plan(ctx, &d, method, out, s, 0, kTuneSide, &P[v]);
                        }
                        for (int v = 0; v < nv && e == cudaSuccess && rc == PTG_OK; ++v)  // warm-up
                            e = launch_fbm2d(P[v], method, s, ctx->stream);
                        for (int r = 0; r < reps && e == cudaSuccess && rc == PTG_OK; ++r)
                            for (int v = 0; v < nv && e == cudaSuccess; ++v) {
                                cudaEventRecord(ev[8 * r + 2 * v], ctx->stream);
                                e = launch_fbm2d(P[v], method, s, ctx->stream);
                                cudaEventRecord(ev[8 * r + 2 * v + 1], ctx->stream);
                            }
                        if (e == cudaSuccess && rc == PTG_OK) e = cudaStreamSynchronize(ctx->stream);
                        if (e != cudaSuccess || rc != PTG_OK) break;
                        Timed t;
                        t.method = method;
                        t.dtype = dt;
                        t.nt = nt;
                        t.mid = mid;
                        t.tail = tail;
                        int best = 0;
                        for (int v = 0; v < 4 && e == cudaSuccess; ++v) {
                            t.us[v] = -1.0f;
                            if (v >= nv) continue;
                            std::vector<float> ts;
                            for (int r = 0; r < reps && e == cudaSuccess; ++r) {
                                float a = 0.0f;
                                e = cudaEventElapsedTime(&a, ev[8 * r + 2 * v], ev[8 * r + 2 * v + 1]);
                                ts.push_back(a * 1e3f);
                            }
                            t.us[v] = median(ts);
                            if (t.us[v] < t.us[best]) best = v;
                        }
                        t.best = (uint8_t)(((best & 1) ? 16 : 8) | ((best & 2) ? kTileBit : 0));
                        table[mi][dt][nt][mid][tail] = t.best;  // nt = 8 also stands for more
                        rows.push_back(t);
                    }
    }
    for (auto& x : ev)
        if (x) cudaEventDestroy(x);
    cudaFree(out);
    if (rc != PTG_OK) return rc;
    if (e != cudaSuccess) return ptg_cuda_fail(ctx, e, "autotune");
    std::memcpy(ctx->tune, table, sizeof table);
    if (cache_path && !write_cache(cache_path, name, sms, reps, rows))
        return ptg_fail(ctx, PTG_ERR_INVALID, "cannot write autotune cache %s", cache_path);
    return PTG_OK;
}

}  // extern "C"
