/*
 * ptg.h -- C ABI of the GB300 polynomial terrain-noise library.
 *
 * Method: Thorimbert & Chopard, "Polynomial methods for fast Procedural
 * Terrain Generation", arXiv:1610.03525.  A field is the fractal (fBm) sum of
 * Sec. 4 over N octaves; octave i uses a lattice 2^i times finer than the base
 * lattice and amplitude persistence^i.  In every octave each sample finds its
 * lattice cell (the unit cell of Sec. 2.1), takes pseudo-random values and
 * gradients at the cell's corners and evaluates the cell polynomial of
 * Eq. (polynomial) that meets the corner constraints of Eq. (mixedderiv):
 *   PTG_C1 -- D2M1N3 / D3M1N3 (Sec. 3.1, 3.4) with zero mixed corner
 *             derivatives: the tensor-product cubic Hermite cell, C1 across
 *             cell faces;
 *   PTG_C2 -- the M = 2 analogue (Sec. 3.4) with per-variable degree 5 and
 *             zero second-order corner derivatives: C2 across faces.
 * Perlin's polynomial (Sec. 3.2) and an OpenSimplex-style simplex-lattice
 * gradient noise (the comparison points of Sec. 1 and 5) use the same octave
 * sum.
 *
 * Conventions shared by every call
 *   - Sample j of axis k sits at base-lattice coordinate
 *     origin[k] + (offset[k] + j) / spc: spc samples per base cell (a power of
 *     two, the same on every axis), origin in whole base cells, offset in
 *     samples.  A field is a window of an unbounded world, so chunks of any
 *     size tile it exactly (the locality argument of Sec. 1).  Cell indices
 *     wrap modulo 2^32.
 *   - Corner data comes from a counter-based hash (pcg3d in 2D, pcg4d in 3D;
 *     Jarzynski & Olano, JCGT 9(3) 2020) of (ix, iy[, iz], seed << 8 | i);
 *     each output word u maps to (u >> 9) * 2^-22 - 1 in [-1, 1).  Word 0 is
 *     the corner value, words 1.. the gradient along x, y[, z], scaled by
 *     grad_weight (the weight w of Sec. 4).
 *   - out is row-major: out[y * W + x] in 2D, out[(z * H + y) * W + x] in 3D,
 *     FP32 or FP16 (round to nearest even from the FP32 sum).
 *   - Device pointers are caller-owned device memory of at least
 *     prod(size) * sizeof(dtype) bytes; the library never frees or keeps them
 *     past the completion of the call's work.
 *   - stream is a cudaStream_t; NULL is the CUDA default stream.  Calls
 *     return after enqueueing; results are ready when the stream is.
 *   - Argument errors return synchronously and write nothing.  Asynchronous
 *     CUDA errors are reported as PTG_ERR_CUDA by the next call.
 *   - A context is not thread-safe; use one per host thread.
 */
#ifndef PTG_H
#define PTG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ptg_ctx ptg_ctx;

typedef enum {
    PTG_OK = 0,
    PTG_PENDING = 1,
    PTG_ERR_INVALID = -1,     /* bad argument                                  */
    PTG_ERR_UNSUPPORTED = -2, /* valid but not supported (e.g. a too-tall field) */
    PTG_ERR_NOMEM = -3,       /* an allocation failed                          */
    PTG_ERR_BUDGET = -4,      /* request can never fit the HBM budget          */
    PTG_ERR_CUDA = -5,        /* a CUDA call failed                            */
    PTG_ERR_TIMEOUT = -6,     /* a bounded wait ran out                        */
    PTG_ERR_CANCELLED = -7
} ptg_status;

/* Cell polynomial (Sec. 3).  PTG_C1 and PTG_C2 are the smooth cells of the
 * header comment (2D and 3D).  The two 2D-only models of the paper:
 *   PTG_PAPER_D2M1N3  -- D2M1N3 with the coefficients printed in Sec. 3.1
 *                        (c22 = c33 = c32 = c23 = 0); continuous across cell
 *                        faces, its slope is not;
 *   PTG_ZERO_GRADIENT -- zero-gradient D2M1N3, Eq. (zg), read with the -xy
 *                        term that the Sec. 3.1 coefficients give (the
 *                        printed +xy does not interpolate h11); corner
 *                        values only (words 1.. unused). */
typedef enum { PTG_C1 = 1, PTG_C2 = 2, PTG_PAPER_D2M1N3 = 3, PTG_ZERO_GRADIENT = 4 } ptg_smoothness;

typedef enum { PTG_F32 = 0, PTG_F16 = 1 } ptg_dtype;

/* Perlin blend (Sec. 3.2): smootherstep S5 (default) or smoothstep S3. */
typedef enum { PTG_PERLIN_S5 = 0, PTG_PERLIN_S3 = 1 } ptg_perlin_blend;

/* Thread shape of the 2D polynomial and Perlin generators, or-ed into
 * desc->variant: how many samples of a 64 x 64 output tile each thread owns,
 * as consecutive columns x rows.  8 x 4 evaluates octaves whose cells are at
 * least 8 samples wide at 4 node columns per run; 16 x 2 halves that work per
 * sample for cells at least 16 samples wide and interpolates more columns.
 * AUTO takes the context's tuned choice (ptg_autotune), else a fixed rule.
 * Both shapes compute the same field; results differ only by FP32 rounding
 * (well inside the stated tolerance).  A shape is a function of the method,
 * dtype, spc and octave count only, never of the size or offset, so a field
 * cut into chunks is bit-identical to the whole.  No counterpart in the
 * paper: a GPU tuning choice. */
typedef enum { PTG_SHAPE_AUTO = 0, PTG_SHAPE_8X4 = 0x100, PTG_SHAPE_16X2 = 0x200 } ptg_shape;

/* How the 2D generators evaluate the octaves whose cells cover a whole
 * 64 x 64 tile (cells of at least 64 samples), or-ed into desc->variant.
 * Each such octave is one polynomial of degree d per axis over the tile, and
 * so is their sum (Sec. 2.2: the cell polynomial; Sec. 4: the octave sum).
 * RUNS evaluates each octave at every thread's node columns, as the finer
 * octaves are; TILE evaluates their sum once per tile at (d + 1)^2 nodes and
 * interpolates it (degree <= 4 models: C1, the paper's D2M1N3 and
 * zero-gradient models, Perlin S3).  AUTO: the context's tuned choice, else a
 * fixed rule.  Both compute the same field up to FP32 rounding; like the
 * thread shape, the choice depends on the method, dtype, spc and octave count
 * only.  No counterpart in the paper: a GPU tuning choice. */
typedef enum { PTG_COARSE_AUTO = 0, PTG_COARSE_RUNS = 0x400, PTG_COARSE_TILE = 0x800 } ptg_coarse;

/* Ridged noise, or-ed into desc->variant of ptg_field / ptg_perlin (2D or
 * 3D): the ridged mountains the paper renders (Sec. 5.1, figure of ridged
 * zero-gradient D2M1N3 noise), which it defines only by reference to a noise
 * library.  Read as Musgrave's ridged multifractal (Ebert et al., "Texturing
 * and Modeling", ch. 16) with offset 1 and gain 2: octave i contributes
 * p^i r_i with r_i = (1 - |h_i|)^2 w_i, h_i the unit-amplitude octave field,
 * w_0 = 1 and w_{i+1} = clamp(2 r_i, 0, 1).  The octaves interact, so every
 * octave is evaluated at every sample, in octave order: fields with
 * lacunarity 2, spc a power of two and offsets multiples of min(spc, tile
 * side) run the fused ridged kernels (2D and 3D), the others the per-sample
 * generators (thread-shape and coarse-octave bits are ignored); batches
 * (ptg_batch*) do not take them. */
#define PTG_RIDGED 0x1000

/* Full description of one field (Sec. 2.1 cell lattice, Sec. 4 octaves). */
typedef struct {
    uint32_t struct_size; /* sizeof(ptg_field_desc)                            */
    int32_t dims;         /* 2 or 3                                            */
    int64_t size[3];      /* samples per axis (x, y, z), each in [1, 2^30]; unused = 1.
                             A 3D field takes at most 65535 tiles of 16
                             rows along y (H <= 1048560), else
                             PTG_ERR_UNSUPPORTED.  Fields taller than one
                             launch's 65535 tiles along the slowest axis
                             (2D H > 4194240, 3D D > 524280) run as
                             consecutive launches on the same stream       */
    int64_t spc;          /* samples per base cell, in [1, 2^30]; a value
                             that is not a power of two runs the per-sample
                             generators (see lacunarity)                    */
    int64_t origin[3];    /* base-lattice cell of the window (wraps mod 2^32)  */
    int64_t offset[3];    /* sample offset of the window, offset + size <=
                             2^31; for the fused generators (power-of-two spc,
                             lacunarity 2) a multiple of min(spc, tile) with
                             tile 64 (2D) or 32/16/8 (3D x/y/z)              */
    int32_t octaves;      /* N in [1, 32]                                      */
    int32_t smoothness;   /* ptg_smoothness (ptg_field, ptg_submit)            */
    float persistence;    /* amplitude ratio between octaves (0.5 typical)     */
    float lacunarity;     /* frequency ratio f between octaves, in [1, 16]
                             (Sec. 4: frequency f^i at octave i).  f = 2 runs
                             the fused generators; any other f runs a
                             per-sample generator (2D, or 3D C1/C2/Perlin;
                             OpenSimplex takes any f in 2D and 3D)
                             in which the lattice
                             coordinate (origin + (offset + j)/spc) f^i is
                             formed per tile in FP64 and must stay below 2^30
                             (else PTG_ERR_UNSUPPORTED); thread-shape and
                             coarse-octave bits are ignored there, and
                             batches (ptg_batch*) need f = 2               */
    float grad_weight;    /* w of Sec. 4; 1.0 default, 0.01 = the paper's      */
    uint32_t seed;        /* < 2^24                                            */
    int32_t dtype;        /* ptg_dtype                                         */
    int32_t variant;      /* low byte: ptg_perlin_blend for ptg_perlin, else 0;
                             bits 8..9: ptg_shape, bits 10..11: ptg_coarse
                             (2D field / Perlin only); bit 12: PTG_RIDGED
                             (field / Perlin)                                  */
} ptg_field_desc;

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the
 * output bytes that the request loop (ptg_submit) holds admitted at once;
 * 0 means 40 GiB.  *ctx receives the handle.  Returns PTG_OK,
 * PTG_ERR_INVALID (ctx NULL, bad device) or PTG_ERR_CUDA. */
int ptg_create(ptg_ctx** ctx, int device, uint64_t hbm_budget_bytes);

/* Wait for outstanding work and free the context.  NULL is allowed. */
int ptg_destroy(ptg_ctx* ctx);

/* 2D heightmap of Sec. 4 with the short-form defaults: spc = 64, origin 0,
 * offset 0, grad_weight 1, FP32 output.  size[2] = (W, H).
 * out: device, W*H floats. */
int ptg_heightmap2d(ptg_ctx* ctx, const int64_t size[2], int32_t octaves, int32_t smoothness,
                    float persistence, float lacunarity, uint32_t seed, void* out, void* stream);

/* 3D volume, same defaults (spc = 64, FP32 output).  size[3] = (W, H, D).
 * out: device, W*H*D floats. */
int ptg_volume3d(ptg_ctx* ctx, const int64_t size[3], int32_t octaves, int32_t smoothness,
                 float persistence, float lacunarity, uint32_t seed, void* out, void* stream);

/* Polynomial-noise field from a full descriptor (any ptg_smoothness; C1 and C2
 * in 2D or 3D, the paper's D2M1N3 and zero-gradient models in 2D). */
int ptg_field(ptg_ctx* ctx, const ptg_field_desc* desc, void* out, void* stream);

/* Perlin's polynomial (Sec. 3.2) with the same lattice: at each corner the
 * dot product of its gradient with the offset to the corner, blended by S
 * along every axis.  The gradient is hash words 1..2 (2D, pcg3d) or 1..3
 * (3D, pcg4d), unweighted; desc->variant selects S5 or S3.  2D or 3D. */
int ptg_perlin(ptg_ctx* ctx, const ptg_field_desc* desc, void* out, void* stream);

/* OpenSimplex-style noise (Sec. 1, Sec. 5 baseline): the base lattice is
 * squished into equilateral triangles of edge sqrt(2) (stretch
 * (1/sqrt(3) - 1)/2, squish (sqrt(3) - 1)/2); every vertex (a, b) within
 * distance sqrt(2) of the point adds (2 - r^2)^4 (g . d), g from hash words
 * 1..2 of pcg3d(a, b, seed << 8 | i); the sum is scaled by 1/8.  In 3D the
 * squish is 1/3 and the stretch -1/6 (nearest vertices sqrt(2) apart, the
 * face-centred cubic lattice), g = hash words 1..3 of pcg4d(a, b, c,
 * seed << 8 | i), with the same kernel and scale.  2D or 3D; the finest
 * octave's lattice coordinates must stay below 2^30 in magnitude
 * ((|origin| + (offset + size)/spc) * f^(N-1) < 2^30), else
 * PTG_ERR_UNSUPPORTED. */
int ptg_opensimplex(ptg_ctx* ctx, const ptg_field_desc* desc, void* out, void* stream);

/* Generate into HOST memory: the field is produced in bands on the device and
 * each band is copied to `host_out` while the next is computed.  Blocks until
 * the whole field is in host_out.  host_out should be pinned for full copy
 * bandwidth.  method: 0 = ptg_field, 1 = ptg_perlin, 2 = ptg_opensimplex.
 * Uses context-owned device staging (allocated on first use, kept). */
int ptg_generate_host(ptg_ctx* ctx, const ptg_field_desc* desc, int32_t method, void* host_out);

/* Batched generation: n independent 2D fields (any mix of sizes, octave
 * counts, C1/C2 polynomial noise, seeds, origins, offsets, FP32/FP16) in ONE
 * persistent launch: resident CTAs pull 64 x 64 tiles of all fields from a
 * device work counter.  descs: host array of n descriptors; outs: host array
 * of n device output pointers.  Results equal n separate ptg_field calls
 * bit for bit.  The fields may come in any order: the library lays them out
 * grouped by kernel path (method and thread shape), which keeps one path in
 * the instruction cache at a time.  Uses context-owned device memory for the
 * launch plans and the counter (grown on demand, kept).  Asynchronous on
 * `stream`. */
int ptg_batch(ptg_ctx* ctx, const ptg_field_desc* descs, void* const* outs, int32_t n, void* stream);

/* A prepared batch: plans uploaded once and the launch (counter reset plus
 * the persistent kernel) captured in a CUDA graph, for batches that repeat
 * with the same fields and outputs. */
typedef struct ptg_batch_plan ptg_batch_plan;

/* Validate, upload and capture a batch (blocking).  *plan receives it. */
int ptg_batch_prepare(ptg_ctx* ctx, const ptg_field_desc* descs, void* const* outs, int32_t n,
                      ptg_batch_plan** plan);

/* Launch a prepared batch (one graph launch) on `stream` (NULL = default). */
int ptg_batch_launch(ptg_batch_plan* plan, void* stream);

/* Free a prepared batch after its launches have completed. */
int ptg_batch_free(ptg_batch_plan* plan);

/* Batched generation for callers that cannot allocate device memory -- an
 * engine that hands out all device memory from its own fixed arena, or a
 * real-time loop in which cudaMalloc's implicit device synchronisation would
 * stall every other stream.  Same fields, outputs and results as ptg_batch,
 * but the launch plans and the work counter live in one fixed device array
 * inside the library (file-scope, at most 256 fields; 256 x 2016-byte field
 * plans + 257 x 8-byte tile offsets + an 8-byte counter = 518,160 bytes, held
 * by every device that loads the library until the process exits) instead of
 * context-owned allocations; no cudaMalloc, cudaFree or other allocator is
 * called.  The caller owns every output buffer.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress).  All calls
 * share the array and clear its counter: calls that overlap on the GPU race,
 * so order them (one stream, or events).  n > 256 returns PTG_ERR_INVALID.
 * The paper has no counterpart; this is a deployment aid. */
int ptg_batch_noalloc(ptg_ctx* ctx, const ptg_field_desc* descs, void* const* outs, int32_t n, void* stream);

/* Request loop.  Queue one field for asynchronous generation into device
 * memory `out`.  Requests are admitted in arrival order while the admitted
 * output bytes stay within the context's HBM budget; admitted requests run
 * concurrently on the context's worker streams.  *req_id receives the id.
 * Returns PTG_ERR_BUDGET if the request alone exceeds the budget. */
int ptg_submit(ptg_ctx* ctx, const ptg_field_desc* desc, void* out, uint64_t* req_id);

/* Non-blocking status of a request: *st = PTG_PENDING or its final status;
 * ts_ns (may be NULL) = submit, admit, start and end times in ns of a
 * monotonic host clock (0 where not reached yet).  End is when the request
 * loop saw the request complete; start is end minus the device time between
 * timing events recorded around the request's kernels (not before admit).
 * Returns PTG_OK or PTG_ERR_INVALID (unknown id). */
int ptg_poll(ptg_ctx* ctx, uint64_t req_id, ptg_status* st, uint64_t ts_ns[4]);

/* Wait at most timeout_ns for a request; returns its final status or
 * PTG_ERR_TIMEOUT.  The record stays until ptg_poll has returned the final
 * status (ptg_poll releases it). */
int ptg_wait(ptg_ctx* ctx, uint64_t req_id, uint64_t timeout_ns);

/* Cancel a request that is still queued (not yet admitted): its final status
 * becomes PTG_ERR_CANCELLED.  Returns PTG_OK, or PTG_ERR_INVALID if the
 * request is unknown or already admitted. */
int ptg_cancel(ptg_ctx* ctx, uint64_t req_id);

/* Autotuner for the 2D launch configuration: the thread shape (ptg_shape)
 * and the coarse-octave mode (ptg_coarse).  For every 2D method, dtype and
 * octave structure -- the number of octaves with cells of at least 64
 * samples (capped at 8), of 16 to 32 samples (0..2), and whether finer
 * octaves follow -- time every configuration on an 8192 x 8192 field (effort
 * timed launches each, 0 = 5) and keep the fastest in the context; AUTO
 * fields use the table from then on.  cache_path (may be NULL): if the file
 * exists and was written for this device model and SM count, load the table
 * from it instead of timing; otherwise time and write it (JSON).  Call it
 * before other work on the context.  Blocks (about a second); allocates one
 * 256 MiB scratch field for the duration.  Returns PTG_OK, PTG_ERR_CUDA, or PTG_ERR_INVALID
 * (bad arguments, a cache file that is not a table, a cache that cannot be
 * written).  No counterpart in the paper. */
int ptg_autotune(ptg_ctx* ctx, int32_t effort, const char* cache_path);

/* The launch configuration that generator `method` (0 = ptg_field,
 * 1 = ptg_perlin) would use for desc on this context: *rw = 8 (8 x 4) or
 * 16 (16 x 2); *tile_octaves = how many octaves are summed at the tile nodes
 * (0 = none).  Either pointer may be NULL.  Returns PTG_OK or the validation
 * status of desc. */
int ptg_launch_config(ptg_ctx* ctx, const ptg_field_desc* desc, int32_t method, int32_t* rw,
                      int32_t* tile_octaves);

/* Check a descriptor for generator `method` (0 = ptg_field, 1 = ptg_perlin,
 * 2 = ptg_opensimplex) without touching any device: returns the status the
 * generator would return for its arguments (PTG_OK, PTG_ERR_INVALID or
 * PTG_ERR_UNSUPPORTED) and writes the reason into msg (msg_len bytes, may be
 * NULL). */
int ptg_validate(const ptg_field_desc* desc, int32_t method, char* msg, int32_t msg_len);

/* --- Map statistics (the paper's quality measurements, Sec. 5) ---------- */

/* Coastline box counts for the fractal dimension (Sec. 5.3): squares of side
 * eps = 2^k samples, k = 0 .. levels-1, cover a W x H map (device, row-major
 * FP32); square (bx, by) holds the samples bx eps .. bx eps + eps (inclusive,
 * clipped) along x and likewise along y, and counts when it holds samples
 * below `level` and samples at or above it.  counts: host array of `levels`
 * entries.  D is the slope of log counts against -log eps.  Blocks on
 * `stream`; uses context-owned device memory of about (W-1)(H-1) 1.25 bytes
 * (grown on demand, kept).  Returns PTG_OK, PTG_ERR_INVALID or PTG_ERR_CUDA. */
int ptg_box_counts(ptg_ctx* ctx, const float* map, int64_t W, int64_t H, float level, int32_t levels,
                   uint64_t* counts, void* stream);

/* Frequency distribution of heights (what = 0) or of the slope norm
 * (what = 1) over `count` maps of W x H samples (device, [count][H][W] FP32)
 * (Sec. 5.1).  The slope at an interior sample is |central differences| / 2
 * in height per sample; border samples have none.  Bin of a value v:
 * floor((v - lo) * (bins / (hi - lo))) in FP32, hist[0] below lo, hist[1 + b],
 * hist[bins + 1] at or above hi.  hist: device array of bins + 2 counters,
 * added to (zero it first).  bins in [1, 4096].  Asynchronous on `stream`. */
int ptg_histogram(ptg_ctx* ctx, const float* maps, int64_t W, int64_t H, int64_t count, float lo, float hi,
                  int32_t bins, int32_t what, uint64_t* hist, void* stream);

/* Text of the last error reported on this context ("" if none). */
const char* ptg_last_error(ptg_ctx* ctx);

/* --- Test hooks (same device code as the generators) ------------------- */

/* Hash n keys of dims+1 words (dims 2: pcg3d, 3: pcg4d) on the device.
 * keys, out: device arrays of n*(dims+1) uint32. */
int ptg_debug_hash(ptg_ctx* ctx, int32_t dims, const uint32_t* keys, int64_t n, uint32_t* out, void* stream);

/* Failure-injection hook for the request loop: hold = 1 makes the next
 * admitted request's stream wait on the host (never on the device) until
 * hold = 0 is set or 5 s pass, simulating a stalled device. */
int ptg_debug_hold(ptg_ctx* ctx, int32_t hold);

/* Failure-injection hook for memory exhaustion, on the host.  Of the device
 * or pinned-host allocations the library makes next for this context (staging
 * of ptg_generate_host, ptg_batch buffers, prepared batches, the box-count
 * pyramid, the autotune field), the first `after` succeed and the following n
 * fail as if memory were exhausted: the call that needed them frees what it
 * had allocated, returns PTG_ERR_NOMEM and writes nothing.  n = 0 turns the
 * injection off.  A failed allocation is never attempted, so no GPU fault is
 * involved.  Negative arguments return PTG_ERR_INVALID. */
int ptg_debug_fail_alloc(ptg_ctx* ctx, int32_t after, int32_t n);

/* Bounds-check records of the debug build.  libptg_debug.so (the same sources
 * compiled with -DPTG_DEBUG_BOUNDS, see paper_1610_03525_gb300/build.py)
 * checks every shared-memory access of the fused 2D and 3D generators, the
 * batched 2D generator and the 2D OpenSimplex generator against the CTA's
 * shared memory, and every index of their global accesses against its
 * extent; a violation is skipped (loads read zero) and its first occurrence
 * recorded.  This call synchronizes the context's device, writes the first
 * record to *first ((site << 48) | index, 0 if none; sites 1 staging stores,
 * 2 corner loads, 3 per-tile tables, 4 constant tables, 5 output elements,
 * 6 batch plans, 7 gradient boxes, 15 the self-test) and clears the records.
 * The regular library returns PTG_ERR_UNSUPPORTED with *first = 0. */
int ptg_debug_bounds(ptg_ctx* ctx, uint64_t* first);

/* Debug build: evaluate one bounds check (site, idx against [0, n)) in a
 * kernel, without touching memory at idx, to exercise the recording path.
 * The regular library returns PTG_ERR_UNSUPPORTED. */
int ptg_debug_bounds_selftest(ptg_ctx* ctx, int32_t site, int64_t idx, int64_t n);

/* Cell index and in-cell position of n sample indices j (device int64) on
 * one axis at octave i, with the generators' fixed-point map:
 * cell (device uint32) and t (device float). */
int ptg_debug_axis(ptg_ctx* ctx, int64_t origin, int64_t spc, int32_t octave, const int64_t* j, int64_t n,
                   uint32_t* cell, float* t, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PTG_H */
