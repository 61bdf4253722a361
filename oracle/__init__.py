"""FP64 CPU oracle for polynomial terrain noise -- TEST INFRASTRUCTURE ONLY.

Thin ctypes/numpy wrapper over ``ptg_oracle.c`` (plain, slow, FP64).  Only the
test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of the
benchmark may import this package.  It shares no code with the CUDA path.

Method of Thorimbert & Chopard, arXiv:1610.03525: cell polynomials of
Sec. 2-3 (Eq. mixedderiv, Eq. polynomial, Eq. nconstraints), the fractal sum
of Sec. 4, Perlin's polynomial of Sec. 3.2 and an OpenSimplex-style baseline.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ptg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libptg_oracle.so")

C1, C2, PAPER_GAUGE, ZERO_GRAD = 1, 2, 3, 4
PERLIN_S5, PERLIN_S3, OPENSIMPLEX = 10, 11, 12


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add contraction, so that
    x86 and Arm hosts round identically)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Desc(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int32),
        ("method", ctypes.c_int32),
        ("size", ctypes.c_int64 * 3),
        ("cells", ctypes.c_int64 * 3),
        ("origin", ctypes.c_int64 * 3),
        ("octaves", ctypes.c_int32),
        ("ridged", ctypes.c_int32),
        ("persistence", ctypes.c_double),
        ("grad_weight", ctypes.c_double),
        ("seed", ctypes.c_uint32),
        ("pad2", ctypes.c_uint32),
        ("frequency", ctypes.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        L.ptgo_pcg3d.argtypes = [P, P]
        L.ptgo_pcg4d.argtypes = [P, P]
        L.ptgo_unit.argtypes = [ctypes.c_uint32]
        L.ptgo_unit.restype = ctypes.c_double
        L.ptgo_system.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P]
        L.ptgo_system.restype = ctypes.c_int
        L.ptgo_invert.argtypes = [ctypes.c_int, P, P]
        L.ptgo_invert.restype = ctypes.c_int
        L.ptgo_cell_coeffs.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_double, P]
        L.ptgo_cell_coeffs.restype = ctypes.c_int
        L.ptgo_field_samples.argtypes = [P, P, ctypes.c_int64, P, ctypes.c_int]
        L.ptgo_field_samples.restype = ctypes.c_int
        L.ptgo_field_grid.argtypes = [P, P, ctypes.c_int]
        L.ptgo_field_grid.restype = ctypes.c_int
        L.ptgo_octave_at.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint32, ctypes.c_int,
                                     ctypes.c_double, P, P, ctypes.c_int64, P]
        L.ptgo_octave_at.restype = ctypes.c_int
        L.ptgo_opensimplex_points.argtypes = [ctypes.c_uint32, ctypes.c_int, P, ctypes.c_int64, P]
        L.ptgo_opensimplex_points.restype = ctypes.c_int
        L.ptgo_opensimplex3_points.argtypes = [ctypes.c_uint32, ctypes.c_int, P, ctypes.c_int64, P]
        L.ptgo_opensimplex3_points.restype = ctypes.c_int
        L.ptgo_hash_batch.argtypes = [ctypes.c_int, P, ctypes.c_int64, P]
        L.ptgo_axis_batch.argtypes = [ctypes.c_int64, ctypes.c_int64, P, ctypes.c_int64, ctypes.c_int, P, P]
        L.ptgo_axis_freq_batch.argtypes = [ctypes.c_int64, ctypes.c_int64, P, ctypes.c_int64, ctypes.c_double,
                                           ctypes.c_int, P, P]
        L.ptgo_num_threads.restype = ctypes.c_int
        L.ptgo_box_counts.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_float, ctypes.c_int, P]
        L.ptgo_histogram.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_float,
                                     ctypes.c_float, ctypes.c_int, ctypes.c_int, P]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def make_desc(dims, size, cells, origin=(0, 0, 0), octaves=1, method=C1, persistence=0.5,
              grad_weight=1.0, seed=0, frequency=2.0, ridged=False) -> Desc:
    d = Desc()
    d.dims = dims
    d.method = method
    d.ridged = 1 if ridged else 0
    for k in range(3):
        d.size[k] = int(size[k]) if k < len(size) else 1
        d.cells[k] = int(cells[k]) if k < len(cells) else 1
        d.origin[k] = int(origin[k]) if k < len(origin) else 0
    d.octaves = octaves
    # persistence and weight enter as the float32 values the GPU path receives
    d.persistence = float(np.float32(persistence))
    d.grad_weight = float(np.float32(grad_weight))
    d.seed = seed
    # the frequency ratio enters as the float32 value the GPU path receives
    d.frequency = float(np.float32(frequency))
    return d


def field_grid(dims, size, cells, *, nthreads=0, **kw) -> np.ndarray:
    """Whole field, shape size[::-1] (row-major [z][y][x])."""
    d = make_desc(dims, size, cells, **kw)
    n = int(np.prod(size[:dims]))
    out = np.empty(n, np.float64)
    rc = lib().ptgo_field_grid(ctypes.byref(d), _ptr(out), nthreads)
    if rc != 0:
        raise ValueError("oracle rejected descriptor")
    return out.reshape(tuple(reversed(size[:dims])))


def field_samples(dims, size, cells, idx, *, nthreads=0, **kw) -> np.ndarray:
    """Field at explicit sample indices idx (n, dims) int64 = (j_x, j_y[, j_z])."""
    d = make_desc(dims, size, cells, **kw)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    assert idx.ndim == 2 and idx.shape[1] == dims
    out = np.empty(idx.shape[0], np.float64)
    rc = lib().ptgo_field_samples(ctypes.byref(d), _ptr(idx), idx.shape[0], _ptr(out), nthreads)
    if rc != 0:
        raise ValueError("oracle rejected descriptor")
    return out


def hash_batch(dims: int, keys: np.ndarray) -> np.ndarray:
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    assert keys.shape[1] == dims + 1
    out = np.empty_like(keys)
    lib().ptgo_hash_batch(dims, _ptr(keys), keys.shape[0], _ptr(out))
    return out


def unit(u: int) -> float:
    return lib().ptgo_unit(int(u) & 0xFFFFFFFF)


def axis(origin: int, spc: int, j, octave: int):
    j = np.ascontiguousarray(np.atleast_1d(j), dtype=np.int64)
    cell = np.empty(j.shape[0], np.uint32)
    t = np.empty(j.shape[0], np.float64)
    lib().ptgo_axis_batch(origin, spc, _ptr(j), j.shape[0], octave, _ptr(cell), _ptr(t))
    return cell, t


def axis_freq(origin: int, spc: int, j, f: float, octave: int):
    """Cell and in-cell position at octave i for frequency ratio f (any f)."""
    j = np.ascontiguousarray(np.atleast_1d(j), dtype=np.int64)
    cell = np.empty(j.shape[0], np.uint32)
    t = np.empty(j.shape[0], np.float64)
    lib().ptgo_axis_freq_batch(origin, spc, _ptr(j), j.shape[0], float(f), octave, _ptr(cell), _ptr(t))
    return cell, t


def system(dims: int, method: int):
    n = 5 if method == C2 else 3
    K = (n + 1) ** dims
    A = np.zeros((K, K), np.float64)
    rc = np.zeros(K, np.int32)
    rd = np.zeros(K, np.int32)
    got = lib().ptgo_system(dims, method, _ptr(A), _ptr(rc), _ptr(rd))
    if got != K:
        raise ValueError("bad system")
    return A, rc, rd


def invert(A: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    out = np.empty_like(A)
    if lib().ptgo_invert(A.shape[0], _ptr(A), _ptr(out)) != 0:
        raise ValueError("singular")
    return out


def cell_coeffs(dims: int, method: int, corner: np.ndarray, w: float) -> np.ndarray:
    """Coefficients c_a (index sum_k a_k (n+1)^k) of one cell from corner data
    (2^dims, dims+1): value then gradient per corner, corner s = sum_k s_k 2^k."""
    corner = np.ascontiguousarray(corner, dtype=np.float64).reshape(-1)
    n = 5 if method == C2 else 3
    coef = np.empty((n + 1) ** dims, np.float64)
    if lib().ptgo_cell_coeffs(dims, method, _ptr(corner), w, _ptr(coef)) < 0:
        raise ValueError("bad system")
    return coef


def octave_at(dims, method, seed, octave, w, cells, t) -> np.ndarray:
    """One octave (unscaled) at explicit (cell, t) points, t_k in [0, 1]."""
    cells = np.ascontiguousarray(cells, dtype=np.uint32)
    t = np.ascontiguousarray(t, dtype=np.float64)
    n = cells.shape[0]
    out = np.empty(n, np.float64)
    if lib().ptgo_octave_at(dims, method, seed, octave, w, _ptr(cells), _ptr(t), n, _ptr(out)) != 0:
        raise ValueError("bad method")
    return out


def opensimplex_points(seed: int, octave: int, xy: np.ndarray) -> np.ndarray:
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    out = np.empty(xy.shape[0], np.float64)
    lib().ptgo_opensimplex_points(seed, octave, _ptr(xy), xy.shape[0], _ptr(out))
    return out


def opensimplex3_points(seed: int, octave: int, xyz: np.ndarray) -> np.ndarray:
    """3D OpenSimplex-style noise of one octave at real lattice positions
    (n x 3)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    out = np.empty(xyz.shape[0], np.float64)
    lib().ptgo_opensimplex3_points(seed, octave, _ptr(xyz), xyz.shape[0], _ptr(out))
    return out


def num_threads() -> int:
    return lib().ptgo_num_threads()


def box_counts(h: np.ndarray, level: float = 0.0, levels: int = 7) -> np.ndarray:
    """Coastline box counts for squares of 1, 2, .. 2^(levels-1) samples (Sec. 5.3)."""
    h = np.ascontiguousarray(h, dtype=np.float32)
    out = np.zeros(levels, np.uint64)
    lib().ptgo_box_counts(_ptr(h), h.shape[1], h.shape[0], float(np.float32(level)), levels, _ptr(out))
    return out


def histogram(h: np.ndarray, lo: float, hi: float, bins: int, what: int = 0) -> np.ndarray:
    """Height (what 0) or slope-norm (what 1) histogram over maps h[..., H, W]
    (Sec. 5.1); bins + 2 counts (below lo, the bins, at or above hi)."""
    h = np.ascontiguousarray(h, dtype=np.float32)
    H, W = h.shape[-2:]
    count = int(np.prod(h.shape[:-2])) if h.ndim > 2 else 1
    out = np.zeros(bins + 2, np.uint64)
    lib().ptgo_histogram(_ptr(h), W, H, count, float(np.float32(lo)), float(np.float32(hi)), bins, what, _ptr(out))
    return out


def box_dimension(counts, first: int = 1, last: int = None) -> float:
    """D of Sec. 5.3: N(eps) ~ eps^(-D), the least-squares slope of log N
    against log eps over levels first .. last (eps = 2^k)."""
    counts = np.asarray(counts, np.float64)
    last = len(counts) - 1 if last is None else last
    k = np.arange(first, last + 1)
    y = np.log2(counts[first:last + 1])
    return float(-np.polyfit(k, y, 1)[0])
