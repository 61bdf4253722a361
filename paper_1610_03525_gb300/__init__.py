"""GB300 polynomial terrain noise (Thorimbert & Chopard, arXiv:1610.03525).

Thin ctypes binding of the C ABI in ``include/ptg.h`` (``libptg.so``, built by
``paper_1610_03525_gb300.build``).  Every function keeps the C name and only
marshals arguments: device buffers are torch CUDA tensors (or raw integer
pointers), streams default to torch's current stream.  All generation runs in
the library's CUDA kernels; there is no CPU fallback, and importing a function
that needs the library fails loudly when ``libptg.so`` is missing.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
# PTG_LIBRARY may name another build of the same C ABI, e.g. the bounds-checked
# debug build libptg_debug.so; by default the regular libptg.so is loaded.
LIB_PATH = os.environ.get("PTG_LIBRARY") or os.path.join(_PKG, "libptg.so")
DEBUG_LIB_PATH = os.path.join(_PKG, "libptg_debug.so")

PTG_OK, PTG_PENDING = 0, 1
PTG_ERR_INVALID, PTG_ERR_UNSUPPORTED, PTG_ERR_NOMEM, PTG_ERR_BUDGET = -1, -2, -3, -4
PTG_ERR_CUDA, PTG_ERR_TIMEOUT, PTG_ERR_CANCELLED = -5, -6, -7
PTG_C1, PTG_C2, PTG_PAPER_D2M1N3, PTG_ZERO_GRADIENT = 1, 2, 3, 4
PTG_F32, PTG_F16 = 0, 1
PTG_PERLIN_S5, PTG_PERLIN_S3 = 0, 1
PTG_SHAPE_AUTO, PTG_SHAPE_8X4, PTG_SHAPE_16X2 = 0, 0x100, 0x200
PTG_COARSE_AUTO, PTG_COARSE_RUNS, PTG_COARSE_TILE = 0, 0x400, 0x800
PTG_RIDGED = 0x1000
METHOD_FIELD, METHOD_PERLIN, METHOD_OPENSIMPLEX = 0, 1, 2

STATUS_NAMES = {
    0: "PTG_OK", 1: "PTG_PENDING", -1: "PTG_ERR_INVALID", -2: "PTG_ERR_UNSUPPORTED", -3: "PTG_ERR_NOMEM",
    -4: "PTG_ERR_BUDGET", -5: "PTG_ERR_CUDA", -6: "PTG_ERR_TIMEOUT", -7: "PTG_ERR_CANCELLED",
}


class ptg_field_desc(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("dims", ctypes.c_int32),
        ("size", ctypes.c_int64 * 3),
        ("spc", ctypes.c_int64),
        ("origin", ctypes.c_int64 * 3),
        ("offset", ctypes.c_int64 * 3),
        ("octaves", ctypes.c_int32),
        ("smoothness", ctypes.c_int32),
        ("persistence", ctypes.c_float),
        ("lacunarity", ctypes.c_float),
        ("grad_weight", ctypes.c_float),
        ("seed", ctypes.c_uint32),
        ("dtype", ctypes.c_int32),
        ("variant", ctypes.c_int32),
    ]


class PtgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(code, str(code)), msg))
        self.code = code


_lib = None


def lib():
    """The loaded libptg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libptg.so is not built (run paper_1610_03525_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, I64, U32, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
        F = ctypes.c_float
        sig = {
            "ptg_create": ([ctypes.POINTER(P), ctypes.c_int, U64], ctypes.c_int),
            "ptg_destroy": ([P], ctypes.c_int),
            "ptg_heightmap2d": ([P, P, I32, I32, F, F, U32, P, P], ctypes.c_int),
            "ptg_volume3d": ([P, P, I32, I32, F, F, U32, P, P], ctypes.c_int),
            "ptg_field": ([P, P, P, P], ctypes.c_int),
            "ptg_perlin": ([P, P, P, P], ctypes.c_int),
            "ptg_opensimplex": ([P, P, P, P], ctypes.c_int),
            "ptg_generate_host": ([P, P, I32, P], ctypes.c_int),
            "ptg_batch": ([P, P, P, I32, P], ctypes.c_int),
            "ptg_batch_prepare": ([P, P, P, I32, ctypes.POINTER(P)], ctypes.c_int),
            "ptg_batch_launch": ([P, P], ctypes.c_int),
            "ptg_batch_free": ([P], ctypes.c_int),
            "ptg_batch_noalloc": ([P, P, P, I32, P], ctypes.c_int),
            "ptg_submit": ([P, P, P, ctypes.POINTER(U64)], ctypes.c_int),
            "ptg_poll": ([P, U64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(U64)], ctypes.c_int),
            "ptg_wait": ([P, U64, U64], ctypes.c_int),
            "ptg_cancel": ([P, U64], ctypes.c_int),
            "ptg_debug_hold": ([P, I32], ctypes.c_int),
            "ptg_debug_fail_alloc": ([P, I32, I32], ctypes.c_int),
            "ptg_debug_bounds": ([P, ctypes.POINTER(U64)], ctypes.c_int),
            "ptg_debug_bounds_selftest": ([P, I32, I64, I64], ctypes.c_int),
            "ptg_autotune": ([P, I32, ctypes.c_char_p], ctypes.c_int),
            "ptg_box_counts": ([P, P, I64, I64, F, I32, P, P], ctypes.c_int),
            "ptg_histogram": ([P, P, I64, I64, I64, F, F, I32, I32, P, P], ctypes.c_int),
            "ptg_launch_config": ([P, P, I32, ctypes.POINTER(I32), ctypes.POINTER(I32)], ctypes.c_int),
            "ptg_last_error": ([P], ctypes.c_char_p),
            "ptg_validate": ([P, I32, ctypes.c_char_p, I32], ctypes.c_int),
            "ptg_debug_hash": ([P, I32, P, I64, P, P], ctypes.c_int),
            "ptg_debug_axis": ([P, I64, I64, I32, P, I64, P, P, P], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


class Context:
    """Owning handle of a ptg_ctx."""

    def __init__(self, handle: int, device: int):
        self.handle = handle
        self.device = device

    def close(self):
        if self.handle:
            lib().ptg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _check(ctx: Context, rc: int) -> int:
    if rc < 0:
        msg = lib().ptg_last_error(ctx.handle if ctx else None)
        raise PtgError(rc, msg.decode() if msg else "")
    return rc


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_desc(dims=2, size=(256, 256), spc=64, origin=(0, 0, 0), offset=(0, 0, 0), octaves=6, smoothness=PTG_C1,
              persistence=0.5, lacunarity=2.0, grad_weight=1.0, seed=0, dtype=PTG_F32, variant=0) -> ptg_field_desc:
    d = ptg_field_desc()
    d.struct_size = ctypes.sizeof(ptg_field_desc)
    d.dims = dims
    d.spc = int(spc)
    for k in range(3):
        d.size[k] = int(size[k]) if k < len(size) else 1
        d.origin[k] = int(origin[k]) if k < len(origin) else 0
        d.offset[k] = int(offset[k]) if k < len(offset) else 0
    d.octaves = octaves
    d.smoothness = smoothness
    d.persistence = persistence
    d.lacunarity = lacunarity
    d.grad_weight = grad_weight
    d.seed = seed
    d.dtype = dtype
    d.variant = variant
    return d


def _check_out(desc: ptg_field_desc, out):
    if isinstance(out, int) or out is None:
        return
    import torch
    n = 1
    for k in range(desc.dims):
        n *= desc.size[k]
    want = torch.float16 if desc.dtype == PTG_F16 else torch.float32
    if not out.is_cuda or not out.is_contiguous() or out.dtype != want or out.numel() < n:
        raise ValueError("out must be a contiguous CUDA %s tensor with >= %d elements" % (want, n))


def ptg_create(device: int = 0, hbm_budget_bytes: int = 0) -> Context:
    h = ctypes.c_void_p()
    rc = lib().ptg_create(ctypes.byref(h), device, hbm_budget_bytes)
    if rc != PTG_OK:
        raise PtgError(rc, "ptg_create(device=%d) failed" % device)
    return Context(h.value, device)


def ptg_destroy(ctx: Context) -> None:
    ctx.close()


def ptg_validate(desc: ptg_field_desc, method: int = METHOD_FIELD):
    """(status, message) the generator would return for this descriptor."""
    buf = ctypes.create_string_buffer(512)
    rc = lib().ptg_validate(ctypes.byref(desc), method, buf, 512)
    return rc, buf.value.decode()


def ptg_last_error(ctx: Context) -> str:
    return lib().ptg_last_error(ctx.handle).decode()


def ptg_field(ctx: Context, desc: ptg_field_desc, out, stream=None) -> int:
    _check_out(desc, out)
    return _check(ctx, lib().ptg_field(ctx.handle, ctypes.byref(desc), _ptr(out), _stream(stream)))


def ptg_perlin(ctx: Context, desc: ptg_field_desc, out, stream=None) -> int:
    _check_out(desc, out)
    return _check(ctx, lib().ptg_perlin(ctx.handle, ctypes.byref(desc), _ptr(out), _stream(stream)))


def ptg_opensimplex(ctx: Context, desc: ptg_field_desc, out, stream=None) -> int:
    _check_out(desc, out)
    return _check(ctx, lib().ptg_opensimplex(ctx.handle, ctypes.byref(desc), _ptr(out), _stream(stream)))


def ptg_heightmap2d(ctx: Context, size, octaves, smoothness, persistence, lacunarity, seed, out, stream=None) -> int:
    sz = (ctypes.c_int64 * 2)(*size)
    return _check(ctx, lib().ptg_heightmap2d(ctx.handle, sz, octaves, smoothness, persistence, lacunarity, seed,
                                             _ptr(out), _stream(stream)))


def ptg_volume3d(ctx: Context, size, octaves, smoothness, persistence, lacunarity, seed, out, stream=None) -> int:
    sz = (ctypes.c_int64 * 3)(*size)
    return _check(ctx, lib().ptg_volume3d(ctx.handle, sz, octaves, smoothness, persistence, lacunarity, seed,
                                          _ptr(out), _stream(stream)))


def ptg_generate_host(ctx: Context, desc: ptg_field_desc, method: int, host_out) -> int:
    return _check(ctx, lib().ptg_generate_host(ctx.handle, ctypes.byref(desc), method, _ptr(host_out)))


def ptg_batch(ctx: Context, descs, outs, stream=None) -> int:
    n = len(descs)
    arr = (ptg_field_desc * n)(*descs)
    ptrs = (ctypes.c_void_p * n)(*[_ptr(o) for o in outs])
    return _check(ctx, lib().ptg_batch(ctx.handle, arr, ptrs, n, _stream(stream)))


def ptg_batch_noalloc(ctx: Context, descs, outs, stream=None) -> int:
    """ptg_batch without any allocation: plans and work counter live in the
    library's fixed device array (at most 256 fields; see include/ptg.h)."""
    n = len(descs)
    arr = (ptg_field_desc * max(n, 1))(*descs)
    ptrs = (ctypes.c_void_p * max(n, 1))(*[_ptr(o) for o in outs])
    return _check(ctx, lib().ptg_batch_noalloc(ctx.handle, arr, ptrs, n, _stream(stream)))


class BatchPlan:
    """Prepared batch (ptg_batch_plan): uploaded plans plus a captured graph."""

    def __init__(self, ctx: Context, handle: int):
        self.ctx = ctx
        self.handle = handle


def ptg_batch_prepare(ctx: Context, descs, outs) -> BatchPlan:
    n = len(descs)
    arr = (ptg_field_desc * n)(*descs)
    ptrs = (ctypes.c_void_p * n)(*[_ptr(o) for o in outs])
    h = ctypes.c_void_p()
    _check(ctx, lib().ptg_batch_prepare(ctx.handle, arr, ptrs, n, ctypes.byref(h)))
    return BatchPlan(ctx, h.value)


def ptg_batch_launch(plan: BatchPlan, stream=None) -> int:
    return _check(plan.ctx, lib().ptg_batch_launch(plan.handle, _stream(stream)))


def ptg_batch_free(plan: BatchPlan) -> None:
    if plan.handle:
        lib().ptg_batch_free(plan.handle)
        plan.handle = None


def ptg_submit(ctx: Context, desc: ptg_field_desc, out) -> int:
    rid = ctypes.c_uint64()
    _check(ctx, lib().ptg_submit(ctx.handle, ctypes.byref(desc), _ptr(out), ctypes.byref(rid)))
    return rid.value


def ptg_poll(ctx: Context, req_id: int):
    st = ctypes.c_int()
    ts = (ctypes.c_uint64 * 4)()
    _check(ctx, lib().ptg_poll(ctx.handle, req_id, ctypes.byref(st), ts))
    return st.value, list(ts)


def ptg_wait(ctx: Context, req_id: int, timeout_ns: int) -> int:
    return lib().ptg_wait(ctx.handle, req_id, timeout_ns)


def ptg_cancel(ctx: Context, req_id: int) -> int:
    return _check(ctx, lib().ptg_cancel(ctx.handle, req_id))


def ptg_autotune(ctx: Context, effort: int = 0, cache_path: str | None = None) -> int:
    """Time the 2D launch configurations per octave structure and keep the
    fastest (or load the table from cache_path, writing it after timing)."""
    path = cache_path.encode() if cache_path else None
    return _check(ctx, lib().ptg_autotune(ctx.handle, effort, path))


def ptg_launch_config(ctx: Context, desc: ptg_field_desc, method: int = METHOD_FIELD):
    """(run width 8 or 16, octaves summed at the tile nodes) that generator
    `method` would use for desc on this context."""
    rw, nt = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(ctx, lib().ptg_launch_config(ctx.handle, ctypes.byref(desc), method, ctypes.byref(rw), ctypes.byref(nt)))
    return rw.value, nt.value


def ptg_box_counts(ctx: Context, field, level: float = 0.0, levels: int = 7, stream=None):
    """Coastline box counts of a 2D FP32 device map for squares of 1 .. 2^(levels-1) samples (Sec. 5.3)."""
    import numpy as np
    H, W = field.shape[-2:]
    out = np.zeros(levels, np.uint64)
    _check(ctx, lib().ptg_box_counts(ctx.handle, _ptr(field), W, H, float(level), levels,
                                     out.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    return out


def ptg_histogram(ctx: Context, maps, lo: float, hi: float, bins: int, what: int = 0, hist=None, stream=None):
    """Height (what 0) or slope-norm (what 1) histogram of FP32 device maps [..., H, W] (Sec. 5.1),
    accumulated into the device tensor hist (bins + 2 int64; created zeroed if None)."""
    import torch
    H, W = maps.shape[-2:]
    count = maps.numel() // (H * W)
    if hist is None:
        hist = torch.zeros(bins + 2, dtype=torch.int64, device=maps.device)
    _check(ctx, lib().ptg_histogram(ctx.handle, _ptr(maps), W, H, count, float(lo), float(hi), bins, what,
                                    _ptr(hist), _stream(stream)))
    return hist


def box_dimension(counts, first: int = 1, last: int | None = None) -> float:
    """D of Sec. 5.3 from box counts (N(eps) ~ eps^-D): the least-squares slope of
    log2 N against -k over levels first .. last (host arithmetic on the counts)."""
    import numpy as np
    counts = np.asarray(counts, np.float64)
    last = len(counts) - 1 if last is None else last
    k = np.arange(first, last + 1)
    return float(-np.polyfit(k, np.log2(counts[first:last + 1]), 1)[0])


def ptg_debug_hold(ctx: Context, hold: int) -> int:
    return _check(ctx, lib().ptg_debug_hold(ctx.handle, hold))


def ptg_debug_fail_alloc(ctx: Context, n: int, after: int = 0) -> int:
    return _check(ctx, lib().ptg_debug_fail_alloc(ctx.handle, after, n))


def ptg_debug_bounds(ctx: Context) -> int:
    """First bounds violation recorded by the debug build ((site << 48) | index), 0 if none; clears the records."""
    v = ctypes.c_uint64(0)
    _check(ctx, lib().ptg_debug_bounds(ctx.handle, ctypes.byref(v)))
    return int(v.value)


def ptg_debug_bounds_selftest(ctx: Context, site: int, idx: int, n: int) -> int:
    return _check(ctx, lib().ptg_debug_bounds_selftest(ctx.handle, site, idx, n))


def ptg_debug_hash(ctx: Context, dims: int, keys, out, stream=None) -> int:
    n = keys.numel() // (dims + 1)
    return _check(ctx, lib().ptg_debug_hash(ctx.handle, dims, _ptr(keys), n, _ptr(out), _stream(stream)))


def ptg_debug_axis(ctx: Context, origin: int, spc: int, octave: int, j, cell, t, stream=None) -> int:
    return _check(ctx, lib().ptg_debug_axis(ctx.handle, origin, spc, octave, _ptr(j), j.numel(), _ptr(cell),
                                            _ptr(t), _stream(stream)))
