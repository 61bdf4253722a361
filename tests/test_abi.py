"""C-ABI boundary checks that need no GPU: the library loads, exports every
function include/ptg.h declares, and its host-side argument validation returns
the documented status codes without touching a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ptg.h")


@pytest.fixture(scope="module")
def P():
    from paper_1610_03525_gb300 import build
    build.build()
    import paper_1610_03525_gb300 as P
    return P


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(ptg_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_expected_calls():
    names = _declared_functions()
    for want in ["ptg_create", "ptg_destroy", "ptg_heightmap2d", "ptg_volume3d", "ptg_field", "ptg_perlin",
                 "ptg_opensimplex", "ptg_submit", "ptg_poll", "ptg_wait", "ptg_last_error", "ptg_batch"]:
        assert want in names


def test_library_exports_every_declared_symbol(P):
    L = ctypes.CDLL(P.LIB_PATH)
    for name in _declared_functions():
        assert hasattr(L, name), name
    # the binding wraps each declared call under the same name
    for name in _declared_functions():
        assert hasattr(P, name), name


def test_desc_layout_matches_header(P):
    # struct_size check in the library rejects a mismatched layout
    d = P.make_desc()
    assert d.struct_size == ctypes.sizeof(P.ptg_field_desc) == 120


@pytest.mark.parametrize("kw,method,code", [
    (dict(), 0, 0),
    (dict(size=(0, 5)), 0, -1),
    (dict(size=(5, 5), spc=0), 0, -1),
    (dict(size=(5, 5), spc=3), 0, 0),                 # any spc in 2D (per-sample generator)
    (dict(size=(5, 5), spc=100, offset=(7, 3, 0)), 1, 0),
    (dict(size=(5, 5), spc=3), 2, 0),
    (dict(dims=3, size=(32, 32, 32), spc=3), 0, 0),   # any spc in 3D too
    (dict(dims=3, size=(32, 32, 32), spc=3), 1, 0),
    (dict(octaves=0), 0, -1),
    (dict(octaves=33), 0, -1),
    (dict(smoothness=5), 0, -1),
    (dict(smoothness=3), 0, 0),
    (dict(smoothness=4, dims=3, size=(32, 32, 32)), 0, -2),
    (dict(lacunarity=3.0), 0, 0),                     # any frequency ratio in 2D
    (dict(lacunarity=1.5), 2, 0),
    (dict(lacunarity=3.0, dims=3, size=(32, 32, 32)), 0, 0),   # 3D per-sample generator
    (dict(lacunarity=3.0, dims=3, size=(32, 32, 32), smoothness=4), 0, -2),  # zero-gradient is 2D
    (dict(lacunarity=0.5), 0, -1),
    (dict(lacunarity=17.0), 0, -1),
    (dict(lacunarity=3.0, octaves=20, spc=64, size=(64, 64)), 0, -2),  # 3^19 lattice units
    (dict(seed=1 << 24), 0, -1),
    (dict(dtype=7), 0, -1),
    (dict(dims=4), 0, -1),
    (dict(dims=3, size=(32, 32, 32)), 1, 0),          # Perlin in 3D
    (dict(dims=3, size=(32, 32, 32)), 2, 0),          # OpenSimplex in 3D
    (dict(dims=3, size=(32, 32, 32), spc=12, lacunarity=1.7), 2, 0),
    (dict(dims=3, size=(32, 32, 32), origin=(1 << 25, 0, 0), octaves=8, spc=16), 2, -2),  # 2^32 lattice units
    (dict(variant=0x100, dims=3, size=(32, 32, 32)), 2, -2),
    (dict(variant=5), 1, -1),
    (dict(offset=(32, 0, 0)), 0, -2),
    (dict(offset=(128, 64, 0)), 0, 0),
    (dict(offset=(-64, 0, 0)), 0, -1),
    (dict(persistence=float("nan")), 0, -1),
    (dict(origin=(1 << 40, 0, 0), octaves=12, spc=1024), 2, -2),
    (dict(size=(1, 1), spc=1, octaves=32), 0, 0),
    (dict(variant=0x100), 0, 0),                      # thread shape 8 x 4
    (dict(variant=0x201), 1, 0),                      # Perlin S3, shape 16 x 2
    (dict(variant=0x300), 0, -1),                     # unknown shape bits
    (dict(variant=0x2000), 0, -1),
    (dict(variant=0x1000), 0, 0),                     # ridged C1 (per-sample generator)
    (dict(variant=0x1001), 1, 0),                     # ridged Perlin S3
    (dict(variant=0x1000, dims=3, size=(32, 32, 32)), 0, 0),
    (dict(variant=0x1000), 2, -2),                    # not for OpenSimplex
    (dict(variant=0x1800, smoothness=2), 0, 0),       # coarse bits ignored when ridged
    (dict(variant=0x1000, smoothness=4, dims=3, size=(32, 32, 32)), 0, -2),
    (dict(variant=0x800), 0, 0),                      # C1 at the tile nodes
    (dict(variant=0x801), 1, 0),                      # Perlin S3 at the tile nodes
    (dict(variant=0x800), 1, -2),                     # not Perlin S5 (degree 6)
    (dict(variant=0x800, smoothness=2), 0, -2),       # not C2 (degree 5)
    (dict(variant=0x400, smoothness=2), 0, 0),
    (dict(variant=0xc00), 0, -1),                     # unknown coarse bits
    (dict(variant=1), 0, -1),                         # blend byte on a polynomial field
    (dict(variant=0x100), 2, -2),                     # no shape for OpenSimplex
    (dict(variant=0x200, dims=3, size=(32, 32, 32)), 0, -2),
    # size limits: 2^30 samples per axis and per cell; fields taller than one
    # launch (65535 tiles: 64-row tiles in 2D, 8-plane tiles in 3D) run as
    # several; a 3D field takes at most 65535 16-row tiles along y
    (dict(size=(1 << 31, 1)), 0, -1),
    (dict(size=(5, 5), spc=1 << 31), 0, -1),
    (dict(size=(5, 5), spc=1 << 30), 0, 0),
    (dict(size=(64, 64), offset=((1 << 31) - 32, 0, 0)), 0, -1),
    (dict(size=(64, 64), offset=((1 << 31) - 64, 0, 0)), 0, 0),
    (dict(size=(64, 65535 * 64)), 0, 0),
    (dict(size=(64, 65535 * 64 + 1)), 0, 0),
    (dict(size=(64, 65535 * 64 + 1)), 2, 0),
    (dict(size=(64, 65535 * 64 + 1), spc=3), 0, 0),
    (dict(size=(64, 1 << 30)), 0, 0),
    (dict(dims=3, size=(32, 32, 65535 * 8)), 0, 0),
    (dict(dims=3, size=(32, 32, 65535 * 8 + 1)), 0, 0),
    (dict(dims=3, size=(32, 32, 65535 * 8 + 1)), 2, 0),
    (dict(dims=3, size=(32, 32, 65535 * 8 + 1), spc=3), 0, 0),
    (dict(dims=3, size=(32, 65535 * 16, 8)), 0, 0),
    (dict(dims=3, size=(32, 65535 * 16 + 1, 8)), 0, -2),
    (dict(dims=3, size=(32, 65535 * 16 + 1, 8)), 2, -2),
    (dict(dims=3, size=(32, 65535 * 16 + 1, 8), spc=3), 0, -2),
])
def test_validation_codes(P, kw, method, code):
    d = P.make_desc(**kw)
    rc, msg = P.ptg_validate(d, method)
    assert rc == code, msg
    assert (msg == "") == (code == 0)


def test_struct_size_checked(P):
    d = P.make_desc()
    d.struct_size = 64
    assert P.ptg_validate(d)[0] == -1


def test_create_without_gpu_fails_cleanly(P):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(P.PtgError):
        P.ptg_create(0)


def test_header_is_plain_c(tmp_path):
    """The boundary is a C ABI: the header compiles as strict C99 (no C++ or
    torch types), and as C++ with C linkage."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text('#include "ptg.h"\n'
                   "int main(void) {\n"
                   "    ptg_ctx* c = 0;\n"
                   "    ptg_field_desc d;\n"
                   "    d.struct_size = (uint32_t)sizeof d;\n"
                   "    return ptg_create(&c, 0, 0) + (int)d.struct_size;\n"
                   "}\n")
    flags = ["-Wall", "-Wextra", "-Werror", "-pedantic", "-fsyntax-only", "-I", os.path.dirname(HEADER)]
    r = subprocess.run([cc, "-std=c99", *flags, str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    cxx = shutil.which("g++")
    if cxx:
        r = subprocess.run([cxx, "-std=c++17", "-x", "c++", *flags, str(src)], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
