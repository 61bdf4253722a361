// ptg_api.cu -- the C ABI declared in include/ptg.h: argument validation,
// per-field launch plans, contexts, and the banded host-output path.
//
// Method: Thorimbert & Chopard, arXiv:1610.03525 (cell polynomials of
// Sec. 2-3, fractal sum of Sec. 4).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ptg.h"
#include "ptg_internal.h"
#include "ptg_kernels.h"

using namespace ptg;

namespace {

int log2_exact(int64_t v)
{
    if (v <= 0 || (v & (v - 1))) return -1;
    int s = 0;
    while ((int64_t{1} << s) < v) ++s;
    return s;
}

}  // namespace

namespace ptg {

cudaError_t set_kernel_smem(const void* kfn, size_t smem)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> done;  // (device, kernel) -> largest limit set
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    auto it = done.find({dev, kfn});
    if (it != done.end() && it->second >= smem) return cudaSuccess;
    e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kfn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) done[{dev, kfn}] = smem;
    return e;
}

}  // namespace ptg

#ifdef PTG_DEBUG_BOUNDS
// Readers of the bounds records of every translation unit (debug build).
static std::vector<ptg::BoundsReader>& bounds_readers()
{
    static std::vector<ptg::BoundsReader> readers;
    return readers;
}

void ptg::register_bounds_reader(ptg::BoundsReader fn) { bounds_readers().push_back(fn); }
#endif

int ptg_fail(ptg_ctx* ctx, int code, const char* fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

static bool injected_alloc_failure(ptg_ctx* ctx)
{
    if (ctx->fail_allocs <= 0) return false;
    if (ctx->alloc_pass > 0) {
        --ctx->alloc_pass;
        return false;
    }
    --ctx->fail_allocs;
    return true;
}

cudaError_t ptg_dev_alloc(ptg_ctx* ctx, void** p, size_t bytes)
{
    *p = nullptr;
    if (injected_alloc_failure(ctx)) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaSuccess;
}

cudaError_t ptg_pinned_alloc(ptg_ctx* ctx, void** p, size_t bytes)
{
    *p = nullptr;
    if (injected_alloc_failure(ctx)) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMallocHost(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaSuccess;
}

int ptg_cuda_fail(ptg_ctx* ctx, cudaError_t e, const char* where)
{
    return ptg_fail(ctx, PTG_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

// Polynomial / Perlin fields that run the per-sample generators: a frequency
// ratio other than 2, spc not a power of two, or ridged noise.
bool ptg_per_sample(const ptg_field_desc* d, int spc_log2)
{
    return d->lacunarity != 2.0f || spc_log2 < 0 || (d->variant & PTG_RIDGED) != 0;
}

// Ridged fields that the fused generators' ridged kernels take instead:
// frequency ratio 2, spc a power of two and tiles aligned to cells (offsets
// multiples of min(spc, tile side) on every axis), as for the fused fBm kernels.
bool ptg_fused_ridged(const ptg_field_desc* d, int spc_log2)
{
    if (!(d->variant & PTG_RIDGED) || d->lacunarity != 2.0f || spc_log2 < 0) return false;
    static const int64_t tile2[2] = {kTile2dX, kTile2dY}, tile3[3] = {kTile3dX, kTile3dY, kTile3dZ};
    for (int k = 0; k < d->dims; ++k) {
        const int64_t t = d->dims == 3 ? tile3[k] : tile2[k], align = d->spc < t ? d->spc : t;
        if (d->offset[k] % align != 0) return false;
    }
    return true;
}

// Argument checks common to every generator.  On success fills *spc_log2
// (-1 when spc is not a power of two: 2D, per-sample generators).
int ptg_check_desc(ptg_ctx* ctx, const ptg_field_desc* d, int kind, int* spc_log2)
{
    if (!d) return ptg_fail(ctx, PTG_ERR_INVALID, "descriptor is NULL");
    if (d->struct_size != sizeof(ptg_field_desc))
        return ptg_fail(ctx, PTG_ERR_INVALID, "struct_size %u != %zu", d->struct_size, sizeof(ptg_field_desc));
    if (d->dims != 2 && d->dims != 3) return ptg_fail(ctx, PTG_ERR_INVALID, "dims must be 2 or 3");
    const int s = log2_exact(d->spc);
    if (d->spc <= 0 || d->spc > (int64_t{1} << 30)) return ptg_fail(ctx, PTG_ERR_INVALID, "spc out of [1, 2^30]");
    // the fused generators need tiles aligned to cells; the per-sample ones
    // (OpenSimplex, and 2D fields with any other spc or frequency ratio) do not
    const bool fused = kind != kKindSimplex && s >= 0 && d->lacunarity == 2.0f && !(d->variant & PTG_RIDGED);
    static const int tile2[3] = {kTile2dX, kTile2dY, 1}, tile3[3] = {kTile3dX, kTile3dY, kTile3dZ};
    for (int k = 0; k < d->dims; ++k) {
        if (d->size[k] <= 0 || d->size[k] > (int64_t{1} << 30))
            return ptg_fail(ctx, PTG_ERR_INVALID, "size[%d] = %lld out of [1, 2^30]", k, (long long)d->size[k]);
        if (d->offset[k] < 0 || d->offset[k] + d->size[k] > (int64_t{1} << 31))
            return ptg_fail(ctx, PTG_ERR_INVALID, "offset[%d] must be >= 0 with offset + size <= 2^31", k);
        const int64_t tile = d->dims == 3 ? tile3[k] : tile2[k];
        const int64_t align = d->spc < tile ? d->spc : tile;
        if (fused && d->offset[k] % align)
            return ptg_fail(ctx, PTG_ERR_UNSUPPORTED, "offset[%d] must be a multiple of %lld", k, (long long)align);
    }
    if (d->octaves < 1 || d->octaves > kMaxOctaves)
        return ptg_fail(ctx, PTG_ERR_INVALID, "octaves %d out of [1, 32]", d->octaves);
    if (kind == kKindField && (d->smoothness < PTG_C1 || d->smoothness > PTG_ZERO_GRADIENT))
        return ptg_fail(ctx, PTG_ERR_INVALID, "smoothness must be a ptg_smoothness value");
    if (kind == kKindField && d->dims == 3 && d->smoothness != PTG_C1 && d->smoothness != PTG_C2)
        return ptg_fail(ctx, PTG_ERR_UNSUPPORTED, "the paper's D2M1N3 and zero-gradient models are 2D");
    const int blend = d->variant & 0xff, shape = d->variant & 0x300, coarse = d->variant & 0xc00;
    const bool ridged = (d->variant & PTG_RIDGED) != 0;
    if (d->variant & ~0x1fff) return ptg_fail(ctx, PTG_ERR_INVALID, "variant: unknown bits 0x%x", (unsigned)d->variant);
    if (ridged && kind == kKindSimplex)
        return ptg_fail(ctx, PTG_ERR_UNSUPPORTED, "ridged noise is built for the polynomial models and Perlin");
    if (shape == 0x300) return ptg_fail(ctx, PTG_ERR_INVALID, "variant: unknown thread-shape bits");
    if (coarse == 0xc00) return ptg_fail(ctx, PTG_ERR_INVALID, "variant: unknown coarse-octave bits");
    if (kind == kKindPerlin && blend != PTG_PERLIN_S5 && blend != PTG_PERLIN_S3)
        return ptg_fail(ctx, PTG_ERR_INVALID, "Perlin variant must be PTG_PERLIN_S5 or PTG_PERLIN_S3");
    if (kind != kKindPerlin && blend != 0)
        return ptg_fail(ctx, PTG_ERR_INVALID, "variant: the low byte is the Perlin blend, 0 for other generators");
    if ((shape | coarse) != 0 && (kind == kKindSimplex || d->dims != 2) && !ridged)
        return ptg_fail(ctx, PTG_ERR_UNSUPPORTED, "thread shape and coarse-octave mode apply to 2D polynomial and "
                                                  "Perlin fields");
    if (coarse == PTG_COARSE_TILE && !ridged && ((kind == kKindField && d->smoothness == PTG_C2) ||
                                                 (kind == kKindPerlin && blend == PTG_PERLIN_S5)))
        return ptg_fail(ctx, PTG_ERR_UNSUPPORTED, "tile nodes apply to models of degree <= 4 (not C2, not Perlin S5)");
    if (!std::isfinite(d->persistence) || !std::isfinite(d->grad_weight))
        return ptg_fail(ctx, PTG_ERR_INVALID, "persistence and grad_weight must be finite");
    if (!std::isfinite(d->lacunarity) || d->lacunarity < 1.0f || d->lacunarity > 16.0f)
        return ptg_fail(ctx, PTG_ERR_INVALID, "lacunarity (frequency ratio) must be in [1, 16]");
    if (d->lacunarity != 2.0f || s < 0 || ridged) {
        // per-sample generators: every octave's lattice coordinates must stay below 2^30 in magnitude
        const double fN = std::pow((double)d->lacunarity, (double)(d->octaves - 1));
        for (int k = 0; k < d->dims; ++k) {
            const double e = std::fabs((double)d->origin[k]) + (double)(d->offset[k] + d->size[k]) / (double)d->spc;
            if (e * fN >= std::ldexp(1.0, 30))
                return ptg_fail(ctx, PTG_ERR_UNSUPPORTED, "lattice coordinates (origin + extent) * f^(N-1) exceed 2^30");
        }
    }
    if (d->seed >= (1u << 24)) return ptg_fail(ctx, PTG_ERR_INVALID, "seed must be < 2^24");
    if (d->dtype != PTG_F32 && d->dtype != PTG_F16) return ptg_fail(ctx, PTG_ERR_INVALID, "bad dtype");
    *spc_log2 = s;
    return PTG_OK;
}

// Launch plan of a polynomial / Perlin field (or of a band of one: `band`
// rows/planes starting at sample `band_start` along the slowest axis).
int ptg_make_field_plan(ptg_ctx* ctx, const ptg_field_desc* d, int method, void* out, int s, int64_t band_start,
                        int64_t band_len, FieldPlan* P)
{
    memset(P, 0, sizeof *P);
    const bool is3d = d->dims == 3;
    P->out = out;
    P->W = (int32_t)d->size[0];
    P->H = (int32_t)d->size[1];
    P->D = is3d ? (int32_t)d->size[2] : 1;
    P->jx0 = (int32_t)d->offset[0];
    P->jy0 = (int32_t)d->offset[1];
    P->jz0 = is3d ? (int32_t)d->offset[2] : 0;
    if (is3d) {
        P->D = (int32_t)band_len;
        P->jz0 += (int32_t)band_start;
    } else {
        P->H = (int32_t)band_len;
        P->jy0 += (int32_t)band_start;
    }
    P->dtype = d->dtype;
    P->N = d->octaves;
    const int TW = is3d ? kTile3dX : kTile2dX, TH = is3d ? kTile3dY : kTile2dY, TD = is3d ? kTile3dZ : 1;
    P->tiles_x = (P->W + TW - 1) / TW;
    P->tiles_y = (P->H + TH - 1) / TH;
    P->tiles_z = (P->D + TD - 1) / TD;
    if (P->tiles_y > 65535 || P->tiles_z > 65535)
        return ptg_fail(ctx, PTG_ERR_UNSUPPORTED, "%d x %d tiles along y/z: at most 65535 along y in 3D",
                        P->tiles_y, P->tiles_z);
    const int esz = d->dtype == PTG_F16 ? 2 : 4;
    P->vec_ok = ((reinterpret_cast<uintptr_t>(out) & 15) == 0) && ((P->W * esz) % 16 == 0);
    P->nst = d->octaves < s ? d->octaves : s;
    // 2D: coarse octaves (cells >= 128 samples) first, then fine ones at fixed offsets
    int ncoarse = s - 6;
    ncoarse = ncoarse < 0 ? 0 : (ncoarse < d->octaves ? ncoarse : d->octaves);
    int coff = 0, count = 0, cend = 0;
    double amp = 1.0, lat_bias = 0.0;
    const double p = (double)d->persistence, w = (double)d->grad_weight;
    for (int i = 0; i < d->octaves; ++i) {
        OctPlan& o = P->oct[i];
        if (i < s) {
            const int k = s - i;
            o.mode = k >= 3 ? kModeRun8 : (k == 2 ? kModeRun4 : kModeRun2);
            o.k = k;
            o.ncx = ((TW - 1) >> (k < 31 ? k : 31)) + 2;
            o.ncy = ((TH - 1) >> (k < 31 ? k : 31)) + 2;
            o.ncz = is3d ? ((TD - 1) >> (k < 31 ? k : 31)) + 2 : 1;
            o.coff = coff;
            o.magic = (uint32_t)(((uint64_t{1} << 32) + (uint64_t)o.ncx - 1) / (uint64_t)o.ncx);
            o.magic2 = (uint32_t)(((uint64_t{1} << 32) + (uint64_t)(o.ncx * o.ncy) - 1) / (uint64_t)(o.ncx * o.ncy));
            o.rowlen = is3d ? corner_rowlen3(o.ncx) : corner_slot(o.ncx - 1) + 1;
            if (is3d) {
                // blocks of 8 (cells that cover the tile) one slot apart, so that the
                // two octaves a quarter warp reads in the tile-node sum use two bank groups
                coff += o.rowlen * o.ncy * o.ncz + (o.rowlen == 2 ? 1 : 0);
                cend = coff;
            } else {
                o.coff = k >= 7 ? 4 * i : 4 * ncoarse + fine_off2(k);
                const int e = o.coff + o.rowlen * o.ncy;
                cend = e > cend ? e : cend;
            }
            count += o.ncx * o.ncy * o.ncz;
        } else {
            o.mode = kModeLattice;
            o.k = i - s;
        }
        o.key = (d->seed << 8) | (uint32_t)i;
        o.ox = (uint32_t)((uint64_t)d->origin[0] << i);
        o.oy = (uint32_t)((uint64_t)d->origin[1] << i);
        o.oz = is3d ? (uint32_t)((uint64_t)d->origin[2] << i) : 0u;
        o.amp = (float)amp;
        o.ampw = (float)(amp * w);
        if (i >= s) lat_bias -= 3.0 * (double)o.amp;
        amp *= p;
    }
    P->lat_bias = (float)lat_bias;
    P->grad_w = (float)w;
    P->ridged = ptg_fused_ridged(d, s) ? 1 : 0;
    P->ncorner = cend;
    P->ncount = count;
    P->method = method;
    P->s = s;
    P->rw = 8;
    P->nt = 0;
    if (!is3d && !P->ridged) ptg_pick_config(ctx, d, method, s, &P->rw, &P->nt);  // ridged: 8 x 4
    const size_t smem = is3d ? fbm3d_smem_bytes(*P) : fbm2d_smem_bytes(*P);
    if (smem > (size_t)ctx->max_smem)
        return ptg_fail(ctx, PTG_ERR_UNSUPPORTED, "staging needs %zu bytes of shared memory (max %d)", smem,
                        ctx->max_smem);
    return PTG_OK;
}

int ptg_make_simplex_plan(ptg_ctx* ctx, const ptg_field_desc* d, void* out, int s, int64_t band_start,
                          int64_t band_len, SimplexPlan* P)
{
    memset(P, 0, sizeof *P);
    P->out = out;
    P->W = (int32_t)d->size[0];
    P->H = (int32_t)band_len;
    P->dtype = d->dtype;
    P->N = d->octaves;
    P->tiles_x = (P->W + kTile2dX - 1) / kTile2dX;
    P->tiles_y = (P->H + kTile2dY - 1) / kTile2dY;
    if (P->tiles_y > 65535) return ptg_fail(ctx, PTG_ERR_UNSUPPORTED, "field too tall for one launch");
    (void)s;
    const double spc = (double)d->spc, f = (double)d->lacunarity;
    double lim = 0.0;
    for (int k = 0; k < 2; ++k) {
        const double e = std::fabs((double)d->origin[k]) + (double)(d->offset[k] + d->size[k]) / spc;
        if (e > lim) lim = e;
    }
    if (lim * std::pow(f, (double)(d->octaves - 1)) >= std::ldexp(1.0, 30))
        return ptg_fail(ctx, PTG_ERR_UNSUPPORTED, "OpenSimplex lattice coordinates exceed 2^30");
    double amp = 1.0;
    int box = 0;
    for (int i = 0; i < d->octaves; ++i) {
        const double scale = f == 2.0 ? std::ldexp(1.0, i) : std::pow(f, (double)i);
        const double step = scale / spc;
        // stage the tile's vertex gradients while the lattice is no finer than
        // the samples; the box side is bounded by 64 step + 7 vertices
        P->box_wb[i] = 0;
        if (step <= 1.0) {
            const int wb = (int)std::floor(64.0 * step * 1.0001) + 8;
            if ((size_t)(box + wb * wb) * 8 <= (size_t)96 * 1024) {
                P->box_off[i] = box;
                P->box_wb[i] = wb;
                box += wb * wb;
            }
        }
        P->base_x[i] = (double)d->origin[0] * scale + (double)d->offset[0] * step;
        P->base_y[i] = (double)d->origin[1] * scale + (double)(d->offset[1] + band_start) * step;
        P->step_d[i] = step;
        P->step[i] = (float)step;
        P->step_lo[i] = (float)(step - (double)P->step[i]);
        int ex = 0;
        if (std::frexp(step, &ex) == 0.5) P->exact_mask |= 1u << i;
        P->amp[i] = (float)amp;
        P->key[i] = (d->seed << 8) | (uint32_t)i;
        amp *= (double)d->persistence;
    }
    P->box_words = box;
    return PTG_OK;
}

// Launch plan of a 3D OpenSimplex field (or of a band of planes of one).
int ptg_make_simplex3_plan(ptg_ctx* ctx, const ptg_field_desc* d, void* out, int64_t band_start, int64_t band_len,
                           Simplex3Plan* P)
{
    memset(P, 0, sizeof *P);
    P->out = out;
    P->W = (int32_t)d->size[0];
    P->H = (int32_t)d->size[1];
    P->D = (int32_t)band_len;
    P->dtype = d->dtype;
    P->N = d->octaves;
    P->tiles_x = (P->W + kTile3dX - 1) / kTile3dX;
    P->tiles_y = (P->H + kTile3dY - 1) / kTile3dY;
    P->tiles_z = (P->D + kTile3dZ - 1) / kTile3dZ;
    if (P->tiles_y > 65535 || P->tiles_z > 65535) return ptg_fail(ctx, PTG_ERR_UNSUPPORTED, "field too tall");
    const double spc = (double)d->spc, f = (double)d->lacunarity;
    double lim = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double e = std::fabs((double)d->origin[k]) + (double)(d->offset[k] + d->size[k]) / spc;
        if (e > lim) lim = e;
    }
    if (lim * std::pow(f, (double)(d->octaves - 1)) >= std::ldexp(1.0, 30))
        return ptg_fail(ctx, PTG_ERR_UNSUPPORTED, "OpenSimplex lattice coordinates exceed 2^30");
    const double ext[3] = {kTile3dX - 1, kTile3dY - 1, kTile3dZ - 1};
    constexpr int kBoxMax = 4096;  // vertices (float4 each) of the shared gradient box: 64 KB
    double amp = 1.0;
    int box = 0;
    for (int i = 0; i < d->octaves; ++i) {
        const double scale = f == 2.0 ? std::ldexp(1.0, i) : std::pow(f, (double)i);
        const double step = scale / spc;
        for (int k = 0; k < 3; ++k)
            P->base[k][i] = (double)d->origin[k] * scale + (double)(d->offset[k] + (k == 2 ? band_start : 0)) * step;
        P->step_d[i] = step;
        P->step[i] = (float)step;
        P->step_lo[i] = (float)(step - (double)P->step[i]);
        int ex = 0;
        if (std::frexp(step, &ex) == 0.5) P->exact_mask |= 1u << i;
        P->amp[i] = (float)amp;
        P->key[i] = (d->seed << 8) | (uint32_t)i;
        amp *= (double)d->persistence;
        // stage while the lattice is coarser than the samples and the box
        // fits: the tile spans (5/6) L_k + (1/6)(sum L - L_k) stretched units
        // along axis k (L = tile extent), widened by 1e-5 on each side; its
        // floors take at most floor(span) + 2 values, plus one vertex of
        // margin below and two above
        if (step >= 1.0) continue;
        const double L[3] = {ext[0] * step, ext[1] * step, ext[2] * step}, sumL = L[0] + L[1] + L[2];
        int bw[3];
        for (int k = 0; k < 3; ++k) bw[k] = (int)std::floor((5.0 * L[k] + (sumL - L[k])) / 6.0 + 1e-4) + 5;
        const int n = bw[0] * bw[1] * bw[2];
        if (n > kBoxMax) continue;
        for (int k = 0; k < 3; ++k) P->box_w[k][i] = bw[k];
        if (n > box) box = n;
    }
    P->box_words = box;
    return PTG_OK;
}

// Launch plan of a 2D polynomial / Perlin field with a frequency ratio other
// than 2 (or of a band of one), for the per-sample generator.
int ptg_make_general_plan(ptg_ctx* ctx, const ptg_field_desc* d, int method, void* out, int s, int64_t band_start,
                          int64_t band_len, GeneralPlan* P)
{
    memset(P, 0, sizeof *P);
    P->out = out;
    P->W = (int32_t)d->size[0];
    P->H = (int32_t)band_len;
    P->dtype = d->dtype;
    P->N = d->octaves;
    P->method = method;
    P->ridged = (d->variant & PTG_RIDGED) ? 1 : 0;
    P->tiles_x = (P->W + kTile2dX - 1) / kTile2dX;
    P->tiles_y = (P->H + kTile2dY - 1) / kTile2dY;
    if (P->tiles_y > 65535) return ptg_fail(ctx, PTG_ERR_UNSUPPORTED, "field too tall for one launch");
    const int esz = d->dtype == PTG_F16 ? 2 : 4;
    P->vec_ok = ((reinterpret_cast<uintptr_t>(out) & 15) == 0) && ((P->W * esz) % 16 == 0);
    (void)s;
    const double spc = (double)d->spc, f = (double)d->lacunarity;
    const double p = (double)d->persistence, w = (double)d->grad_weight;
    double amp = 1.0;
    int box = 0;
    for (int i = 0; i < d->octaves; ++i) {
        const double fi = f == 2.0 ? std::ldexp(1.0, i) : std::pow(f, (double)i), scale = fi / spc;
        P->base_x[i] = (double)d->origin[0] * fi + (double)d->offset[0] * scale;
        P->base_y[i] = (double)d->origin[1] * fi + (double)(d->offset[1] + band_start) * scale;
        P->scale[i] = scale;
        P->scale_hi[i] = (float)scale;
        P->scale_lo[i] = (float)(scale - (double)P->scale_hi[i]);
        P->amp[i] = P->ridged ? 1.0f : (float)amp;
        P->ampw[i] = P->ridged ? (float)w : (float)(amp * w);
        P->wgt[i] = (float)amp;
        P->key[i] = (d->seed << 8) | (uint32_t)i;
        if (f == 2.0 && s >= 0 && i >= s) P->lattice_mask |= 1u << i;  // integer lattice coordinates
        // stage the corners of the cells a tile spans while cells cover at
        // least one sample: one cell before the base cell, floor(63 scale) + 1
        // after it, one more for rounding, and the corner past the last cell
        P->box_w[i] = 0;
        if (scale <= 1.0 && !((P->lattice_mask >> i) & 1u)) {  // lattice octaves read one corner a sample
            const int bw = (int)std::floor(63.0 * scale) + 5;
            if ((size_t)(box + bw * bw) * sizeof(float4) <= (size_t)96 * 1024) {
                P->box_off[i] = box;
                P->box_w[i] = bw;
                P->box_magic[i] = (uint32_t)(((uint64_t{1} << 32) + (uint64_t)bw - 1) / (uint64_t)bw);
                box += bw * bw;
            }
        }
        amp *= p;
    }
    P->box_words = box;
    return PTG_OK;
}

// The same for a 3D field (or a band of planes of one).
int ptg_make_general3_plan(ptg_ctx* ctx, const ptg_field_desc* d, int method, void* out, int64_t band_start,
                           int64_t band_len, General3Plan* P)
{
    memset(P, 0, sizeof *P);
    P->out = out;
    P->W = (int32_t)d->size[0];
    P->H = (int32_t)d->size[1];
    P->D = (int32_t)band_len;
    P->dtype = d->dtype;
    P->N = d->octaves;
    P->method = method;
    P->ridged = (d->variant & PTG_RIDGED) ? 1 : 0;
    P->tiles_x = (P->W + kTile3dX - 1) / kTile3dX;
    P->tiles_y = (P->H + kTile3dY - 1) / kTile3dY;
    P->tiles_z = (P->D + kTile3dZ - 1) / kTile3dZ;
    if (P->tiles_y > 65535 || P->tiles_z > 65535) return ptg_fail(ctx, PTG_ERR_UNSUPPORTED, "field too tall");
    const int esz = d->dtype == PTG_F16 ? 2 : 4;
    P->vec_ok = ((reinterpret_cast<uintptr_t>(out) & 15) == 0) && ((P->W * esz) % 16 == 0);
    const double spc = (double)d->spc, f = (double)d->lacunarity;
    const double p = (double)d->persistence, w = (double)d->grad_weight;
    const int ext[3] = {kTile3dX - 1, kTile3dY - 1, kTile3dZ - 1};
    const int spc_log2 = log2_exact(d->spc);
    double amp = 1.0;
    int box = 0;
    for (int i = 0; i < d->octaves; ++i) {
        const double fi = f == 2.0 ? std::ldexp(1.0, i) : std::pow(f, (double)i), scale = fi / spc;
        for (int a = 0; a < 3; ++a)
            P->base[a][i] = (double)d->origin[a] * fi + (double)(d->offset[a] + (a == 2 ? band_start : 0)) * scale;
        P->scale[i] = scale;
        P->scale_hi[i] = (float)scale;
        P->scale_lo[i] = (float)(scale - (double)P->scale_hi[i]);
        P->amp[i] = P->ridged ? 1.0f : (float)amp;
        P->ampw[i] = P->ridged ? (float)w : (float)(amp * w);
        P->wgt[i] = (float)amp;
        P->key[i] = (d->seed << 8) | (uint32_t)i;
        if (f == 2.0 && spc_log2 >= 0 && i >= spc_log2) P->lattice_mask |= 1u << i;  // integer lattice coordinates
        if (scale <= 0.5) {  // one cell before the base cell, ext * scale + 1 after it, one for rounding, +1 corner
            int bw[3];
            for (int a = 0; a < 3; ++a) bw[a] = (int)std::floor(ext[a] * scale) + 5;
            const int n = bw[0] * bw[1] * bw[2];
            if ((size_t)(box + n) * sizeof(float4) <= (size_t)96 * 1024) {
                P->box_off[i] = box;
                for (int a = 0; a < 3; ++a) P->box_w[a][i] = bw[a];
                P->box_magic[0][i] = (uint32_t)(((uint64_t{1} << 32) + (uint64_t)bw[0] - 1) / (uint64_t)bw[0]);
                const uint64_t wxy = (uint64_t)bw[0] * (uint64_t)bw[1];
                P->box_magic[1][i] = (uint32_t)(((uint64_t{1} << 32) + wxy - 1) / wxy);
                box += n;
            }
        }
        amp *= p;
    }
    P->box_words = box;
    return PTG_OK;
}

int ptg_kernel_method(int kind, const ptg_field_desc* d)
{
    if (kind == kKindPerlin) return (d->variant & 0xff) == PTG_PERLIN_S3 ? kPerlinS3 : kPerlinS5;
    switch (d->smoothness) {
    case PTG_C2: return kC2;
    case PTG_PAPER_D2M1N3: return kPaperGauge;
    case PTG_ZERO_GRADIENT: return kZeroGrad;
    default: return kC1;
    }
}

// Rows (2D) or planes (3D) of the slowest axis that one launch covers: a
// grid takes at most 65535 tiles along y and z.
int64_t ptg_launch_rows(const ptg_field_desc* d)
{
    return d->dims == 3 ? int64_t{65535} * kTile3dZ : int64_t{65535} * kTile2dY;
}

// One launch: rows [band_start, band_start + band_len) of the slowest axis into
// out (the band's first row), with band_len <= ptg_launch_rows.
static int launch_band(ptg_ctx* ctx, int kind, const ptg_field_desc* d, int s, void* out, int64_t band_start,
                       int64_t band_len, cudaStream_t st)
{
    cudaError_t e;
    if (kind == kKindSimplex && d->dims == 3) {
        Simplex3Plan P;
        int rc = ptg_make_simplex3_plan(ctx, d, out, band_start, band_len, &P);
        if (rc != PTG_OK) return rc;
        e = launch_opensimplex3d(P, st);
    } else if (kind == kKindSimplex) {
        SimplexPlan P;
        int rc = ptg_make_simplex_plan(ctx, d, out, s, band_start, band_len, &P);
        if (rc != PTG_OK) return rc;
        e = launch_opensimplex2d(P, st);
    } else if (ptg_per_sample(d, s) && !ptg_fused_ridged(d, s) && d->dims == 3) {  // any f or spc, ridged: 3D
        General3Plan P;
        int rc = ptg_make_general3_plan(ctx, d, ptg_kernel_method(kind, d), out, band_start, band_len, &P);
        if (rc != PTG_OK) return rc;
        e = launch_general3d(P, st);
    } else if (ptg_per_sample(d, s) && !ptg_fused_ridged(d, s)) {  // any f or spc, unaligned ridged: per sample
        GeneralPlan P;
        int rc = ptg_make_general_plan(ctx, d, ptg_kernel_method(kind, d), out, s, band_start, band_len, &P);
        if (rc != PTG_OK) return rc;
        e = launch_general2d(P, st);
    } else {
        const int method = ptg_kernel_method(kind, d);
        FieldPlan P;
        int rc = ptg_make_field_plan(ctx, d, method, out, s, band_start, band_len, &P);
        if (rc != PTG_OK) return rc;
        e = d->dims == 3 ? launch_fbm3d(P, method, s, st) : launch_fbm2d(P, method, s, st);
    }
    if (e != cudaSuccess) return ptg_cuda_fail(ctx, e, "kernel launch");
    return PTG_OK;
}

int ptg_launch_plan(ptg_ctx* ctx, int kind, const ptg_field_desc* d, int s, void* out, int64_t band_start,
                    int64_t band_len, cudaStream_t st)
{
    // fields taller than one launch's tiles: consecutive launches of whole-tile
    // bands on the same stream (band starts stay multiples of the tile, so the
    // cell alignment of every band is the field's own)
    const int64_t step = ptg_launch_rows(d);
    const size_t esz = d->dtype == PTG_F16 ? 2 : 4;
    const size_t slab = (size_t)d->size[0] * esz * (d->dims == 3 ? (size_t)d->size[1] : 1);
    for (int64_t done = 0; done < band_len; done += step) {
        const int64_t len = band_len - done < step ? band_len - done : step;
        void* o = out ? static_cast<void*>(static_cast<char*>(out) + (size_t)done * slab) : nullptr;
        const int rc = launch_band(ctx, kind, d, s, o, band_start + done, len, st);
        if (rc != PTG_OK) return rc;
    }
    return PTG_OK;
}

static int generate(ptg_ctx* ctx, const ptg_field_desc* d, int kind, void* out, void* stream)
{
    if (!ctx) return PTG_ERR_INVALID;
    ctx->err.clear();
    int s = 0;
    int rc = ptg_check_desc(ctx, d, kind, &s);
    if (rc != PTG_OK) return rc;
    if (!out) return ptg_fail(ctx, PTG_ERR_INVALID, "out is NULL");
    DeviceGuard g(ctx->device);
    if (!g.ok) return ptg_fail(ctx, PTG_ERR_CUDA, "cudaSetDevice(%d) failed", ctx->device);
    cudaError_t pending = cudaGetLastError();
    if (pending != cudaSuccess) return ptg_cuda_fail(ctx, pending, "earlier asynchronous error");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t slow = d->dims == 3 ? d->size[2] : d->size[1];
    return ptg_launch_plan(ctx, kind, d, s, out, 0, slow, st);
}

static ptg_field_desc short_desc(int dims, const int64_t* size, int32_t octaves, int32_t smoothness, float p,
                                 float lac, uint32_t seed)
{
    ptg_field_desc d;
    memset(&d, 0, sizeof d);
    d.struct_size = sizeof d;
    d.dims = dims;
    for (int k = 0; k < 3; ++k) d.size[k] = k < dims ? size[k] : 1;
    d.spc = 64;
    d.octaves = octaves;
    d.smoothness = smoothness;
    d.persistence = p;
    d.lacunarity = lac;
    d.grad_weight = 1.0f;
    d.seed = seed;
    d.dtype = PTG_F32;
    return d;
}

extern "C" {

int ptg_create(ptg_ctx** out, int device, uint64_t hbm_budget_bytes)
{
    if (!out) return PTG_ERR_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) return PTG_ERR_CUDA;
    if (device < 0 || device >= ndev) return PTG_ERR_INVALID;
    ptg_ctx* ctx = new (std::nothrow) ptg_ctx();
    if (!ctx) return PTG_ERR_NOMEM;
    ctx->device = device;
    ctx->budget = hbm_budget_bytes ? hbm_budget_bytes : (uint64_t{40} << 30);
    DeviceGuard g(device);
    if (!g.ok) {
        delete ctx;
        return PTG_ERR_CUDA;
    }
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    ctx->num_sms = v;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    ctx->max_smem = v;
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete ctx;
        return PTG_ERR_CUDA;
    }
    *out = ctx;
    return PTG_OK;
}

int ptg_destroy(ptg_ctx* ctx)
{
    if (!ctx) return PTG_OK;
    DeviceGuard g(ctx->device);
    ptg_serve_shutdown(ctx);
    cudaStreamSynchronize(ctx->stream);
    ptg_host_release(ctx);
    ptg_batch_release(ctx);
    if (ctx->stat_buf) cudaFree(ctx->stat_buf);
    cudaStreamDestroy(ctx->stream);
    delete ctx;
    return PTG_OK;
}

const char* ptg_last_error(ptg_ctx* ctx) { return ctx ? ctx->err.c_str() : "context is NULL"; }

int ptg_field(ptg_ctx* ctx, const ptg_field_desc* d, void* out, void* stream)
{
    return generate(ctx, d, kKindField, out, stream);
}

int ptg_perlin(ptg_ctx* ctx, const ptg_field_desc* d, void* out, void* stream)
{
    return generate(ctx, d, kKindPerlin, out, stream);
}

int ptg_opensimplex(ptg_ctx* ctx, const ptg_field_desc* d, void* out, void* stream)
{
    return generate(ctx, d, kKindSimplex, out, stream);
}

int ptg_heightmap2d(ptg_ctx* ctx, const int64_t size[2], int32_t octaves, int32_t smoothness, float persistence,
                    float lacunarity, uint32_t seed, void* out, void* stream)
{
    if (!size) return ptg_fail(ctx, PTG_ERR_INVALID, "size is NULL");
    ptg_field_desc d = short_desc(2, size, octaves, smoothness, persistence, lacunarity, seed);
    return generate(ctx, &d, kKindField, out, stream);
}

int ptg_volume3d(ptg_ctx* ctx, const int64_t size[3], int32_t octaves, int32_t smoothness, float persistence,
                 float lacunarity, uint32_t seed, void* out, void* stream)
{
    if (!size) return ptg_fail(ctx, PTG_ERR_INVALID, "size is NULL");
    ptg_field_desc d = short_desc(3, size, octaves, smoothness, persistence, lacunarity, seed);
    return generate(ctx, &d, kKindField, out, stream);
}

int ptg_validate(const ptg_field_desc* d, int32_t method, char* msg, int32_t msg_len)
{
    if (msg && msg_len > 0) msg[0] = 0;
    if (method < 0 || method > 2) return PTG_ERR_INVALID;
    const int kind = method == 0 ? kKindField : (method == 1 ? kKindPerlin : kKindSimplex);
    ptg_ctx scratch;  // host-only: collects the message, no device state
    scratch.max_smem = 227 * 1024;
    int s = 0;
    int rc = ptg_check_desc(&scratch, d, kind, &s);
    if (rc == PTG_OK) {
        // the first launch's band (ptg_launch_plan splits taller fields; later bands
        // differ only in their start)
        int64_t slow = d->dims == 3 ? d->size[2] : d->size[1];
        if (slow > ptg_launch_rows(d)) slow = ptg_launch_rows(d);
        if (kind == kKindSimplex && d->dims == 3) {
            Simplex3Plan P;
            rc = ptg_make_simplex3_plan(&scratch, d, nullptr, 0, slow, &P);
        } else if (kind == kKindSimplex) {
            SimplexPlan P;
            rc = ptg_make_simplex_plan(&scratch, d, nullptr, s, 0, slow, &P);
        } else if (ptg_per_sample(d, s) && !ptg_fused_ridged(d, s) && d->dims == 3) {
            General3Plan P;
            rc = ptg_make_general3_plan(&scratch, d, ptg_kernel_method(kind, d), nullptr, 0, slow, &P);
        } else if (ptg_per_sample(d, s) && !ptg_fused_ridged(d, s)) {
            GeneralPlan P;
            rc = ptg_make_general_plan(&scratch, d, ptg_kernel_method(kind, d), nullptr, s, 0, slow, &P);
        } else {
            FieldPlan P;
            rc = ptg_make_field_plan(&scratch, d, ptg_kernel_method(kind, d), nullptr, s, 0, slow, &P);
        }
    }
    if (msg && msg_len > 0) {
        strncpy(msg, scratch.err.c_str(), (size_t)msg_len - 1);
        msg[msg_len - 1] = 0;
    }
    return rc;
}

int ptg_box_counts(ptg_ctx* ctx, const float* map, int64_t W, int64_t H, float level, int32_t levels,
                   uint64_t* counts, void* stream)
{
    if (!ctx) return PTG_ERR_INVALID;
    ctx->err.clear();
    if (!map || !counts) return ptg_fail(ctx, PTG_ERR_INVALID, "map and counts must not be NULL");
    if (W < 2 || H < 2 || W > (int64_t{1} << 30) || H > (int64_t{1} << 30))
        return ptg_fail(ctx, PTG_ERR_INVALID, "map size must be in [2, 2^30] per axis");
    if (levels < 1 || levels > 31) return ptg_fail(ctx, PTG_ERR_INVALID, "levels must be in [1, 31]");
    if (!std::isfinite(level)) return ptg_fail(ctx, PTG_ERR_INVALID, "level must be finite");
    DeviceGuard g(ctx->device);
    if (!g.ok) return ptg_fail(ctx, PTG_ERR_CUDA, "cudaSetDevice(%d) failed", ctx->device);
    const size_t n0 = (size_t)(W - 1) * (size_t)(H - 1), n1 = (size_t)(W / 2) * (size_t)(H / 2);
    const size_t off_counts = (n0 + n1 + 15) & ~size_t{15};
    const size_t need = off_counts + 32 * sizeof(unsigned long long);
    cudaError_t e = cudaSuccess;
    if (ctx->stat_bytes < need) {
        if (ctx->stat_buf) cudaFree(ctx->stat_buf);
        ctx->stat_buf = nullptr;
        ctx->stat_bytes = 0;
        if (ptg_dev_alloc(ctx, (void**)&ctx->stat_buf, need) != cudaSuccess)
            return ptg_fail(ctx, PTG_ERR_NOMEM, "cannot allocate %zu bytes for the box-count pyramid", need);
        ctx->stat_bytes = need;
    }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long* dcounts = reinterpret_cast<unsigned long long*>(ctx->stat_buf + off_counts);
    e = cudaMemsetAsync(dcounts, 0, sizeof(unsigned long long) * (size_t)levels, st);
    if (e == cudaSuccess)
        e = launch_box_counts(map, W, H, level, levels, ctx->stat_buf, ctx->stat_buf + n0, dcounts, ctx->num_sms, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(counts, dcounts, sizeof(unsigned long long) * (size_t)levels, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? PTG_OK : ptg_cuda_fail(ctx, e, "box counts");
}

int ptg_histogram(ptg_ctx* ctx, const float* maps, int64_t W, int64_t H, int64_t count, float lo, float hi,
                  int32_t bins, int32_t what, uint64_t* hist, void* stream)
{
    if (!ctx) return PTG_ERR_INVALID;
    ctx->err.clear();
    if (!maps || !hist) return ptg_fail(ctx, PTG_ERR_INVALID, "maps and hist must not be NULL");
    if (W < 1 || H < 1 || count < 1 || W > (int64_t{1} << 30) || H > (int64_t{1} << 30) ||
        count > (int64_t{1} << 30))
        return ptg_fail(ctx, PTG_ERR_INVALID, "bad map size or count");
    if (bins < 1 || bins > 4096) return ptg_fail(ctx, PTG_ERR_INVALID, "bins must be in [1, 4096]");
    if (what != 0 && what != 1) return ptg_fail(ctx, PTG_ERR_INVALID, "what must be 0 (height) or 1 (slope)");
    if (!std::isfinite(lo) || !std::isfinite(hi) || !(lo < hi)) return ptg_fail(ctx, PTG_ERR_INVALID, "need lo < hi");
    DeviceGuard g(ctx->device);
    if (!g.ok) return ptg_fail(ctx, PTG_ERR_CUDA, "cudaSetDevice(%d) failed", ctx->device);
    const float scale = (float)bins / (hi - lo);
    const cudaError_t e = launch_histogram(maps, W, H, count, lo, scale, bins, what,
                                           reinterpret_cast<unsigned long long*>(hist), ctx->num_sms,
                                           (cudaStream_t)stream);
    return e == cudaSuccess ? PTG_OK : ptg_cuda_fail(ctx, e, "histogram");
}

int ptg_debug_hash(ptg_ctx* ctx, int32_t dims, const uint32_t* keys, int64_t n, uint32_t* out, void* stream)
{
    if (!ctx) return PTG_ERR_INVALID;
    if ((dims != 2 && dims != 3) || n < 0 || (n > 0 && (!keys || !out)))
        return ptg_fail(ctx, PTG_ERR_INVALID, "bad debug_hash arguments");
    if (n == 0) return PTG_OK;
    DeviceGuard g(ctx->device);
    cudaError_t e = launch_debug_hash(dims, keys, n, out, (cudaStream_t)stream);
    return e == cudaSuccess ? PTG_OK : ptg_cuda_fail(ctx, e, "debug_hash");
}

int ptg_debug_axis(ptg_ctx* ctx, int64_t origin, int64_t spc, int32_t octave, const int64_t* j, int64_t n,
                   uint32_t* cell, float* t, void* stream)
{
    if (!ctx) return PTG_ERR_INVALID;
    const int s = log2_exact(spc);
    if (s < 0) return ptg_fail(ctx, PTG_ERR_UNSUPPORTED, "spc must be a power of two");
    if (octave < 0 || octave >= kMaxOctaves || n < 0 || (n > 0 && (!j || !cell || !t)))
        return ptg_fail(ctx, PTG_ERR_INVALID, "bad debug_axis arguments");
    if (n == 0) return PTG_OK;
    DeviceGuard g(ctx->device);
    cudaError_t e = launch_debug_axis((long long)origin, s, octave, (const long long*)j, (long long)n, cell, t,
                                      (cudaStream_t)stream);
    return e == cudaSuccess ? PTG_OK : ptg_cuda_fail(ctx, e, "debug_axis");
}

int ptg_debug_fail_alloc(ptg_ctx* ctx, int32_t after, int32_t n)
{
    if (!ctx) return PTG_ERR_INVALID;
    if (after < 0 || n < 0) return ptg_fail(ctx, PTG_ERR_INVALID, "after and n must be >= 0");
    ctx->alloc_pass = after;
    ctx->fail_allocs = n;
    return PTG_OK;
}

int ptg_debug_bounds(ptg_ctx* ctx, uint64_t* first)
{
    if (!ctx) return PTG_ERR_INVALID;
    if (!first) return ptg_fail(ctx, PTG_ERR_INVALID, "first is NULL");
    *first = 0;
#ifdef PTG_DEBUG_BOUNDS
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return ptg_cuda_fail(ctx, e, "debug_bounds");
    for (ptg::BoundsReader fn : bounds_readers()) {
        unsigned long long v = 0;
        e = fn(&v);
        if (e != cudaSuccess) return ptg_cuda_fail(ctx, e, "debug_bounds");
        if (*first == 0) *first = v;
    }
    return PTG_OK;
#else
    return ptg_fail(ctx, PTG_ERR_UNSUPPORTED, "bounds checks exist in the debug build (libptg_debug.so) only");
#endif
}

int ptg_debug_bounds_selftest(ptg_ctx* ctx, int32_t site, int64_t idx, int64_t n)
{
    if (!ctx) return PTG_ERR_INVALID;
#ifdef PTG_DEBUG_BOUNDS
    DeviceGuard g(ctx->device);
    const cudaError_t e = launch_bounds_selftest(site, (long long)idx, (long long)n, nullptr);
    return e == cudaSuccess ? PTG_OK : ptg_cuda_fail(ctx, e, "debug_bounds_selftest");
#else
    (void)site, (void)idx, (void)n;
    return ptg_fail(ctx, PTG_ERR_UNSUPPORTED, "bounds checks exist in the debug build (libptg_debug.so) only");
#endif
}

}  // extern "C"
