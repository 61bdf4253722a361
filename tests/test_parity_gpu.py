"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bars (Thorimbert & Chopard, arXiv:1610.03525; fractal sum of Sec. 4):
  - lattice hashes and cell indices: bit-exact;
  - FP32 heights: max |gpu - oracle| <= 2e-6 * A_tot, A_tot = sum_i p^i;
  - FP16 output: the FP32 bound plus half an FP16 ulp of the value;
  - on-lattice octaves (cells one sample wide) are exact corner values.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import errlog  # noqa: E402
import oracle as O  # noqa: E402
import paper_1610_03525_gb300 as P  # noqa: E402
from paper_1610_03525_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

KIND_ORACLE = {"c1": O.C1, "c2": O.C2, "perlin_s5": O.PERLIN_S5, "perlin_s3": O.PERLIN_S3,
               "opensimplex": O.OPENSIMPLEX, "paper_gauge": O.PAPER_GAUGE, "zero_grad": O.ZERO_GRAD}
SMOOTH = {"c2": P.PTG_C2, "paper_gauge": P.PTG_PAPER_D2M1N3, "zero_grad": P.PTG_ZERO_GRADIENT}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03525_gb300 import build
    build.build()
    c = P.ptg_create(0)
    yield c
    c.close()


def gpu_field(ctx, kind, dims=2, size=(256, 256), spc=64, octaves=6, origin=(0, 0, 0), offset=(0, 0, 0),
              seed=0, persistence=0.5, grad_weight=1.0, dtype=P.PTG_F32, shape=P.PTG_SHAPE_AUTO, coarse=0,
              lacunarity=2.0, ridged=False):
    smooth = SMOOTH.get(kind, P.PTG_C1)
    variant = (P.PTG_PERLIN_S3 if kind == "perlin_s3" else P.PTG_PERLIN_S5) | shape | coarse
    if ridged:
        variant |= P.PTG_RIDGED
    d = P.make_desc(dims=dims, size=size, spc=spc, origin=origin, offset=offset, octaves=octaves,
                    smoothness=smooth, persistence=persistence, grad_weight=grad_weight, seed=seed, dtype=dtype,
                    variant=variant, lacunarity=lacunarity)
    shape = tuple(reversed(size[:dims]))
    out = torch.full(shape, float("nan"), dtype=torch.float16 if dtype == P.PTG_F16 else torch.float32,
                     device="cuda")
    if kind in ("c1", "c2", "paper_gauge", "zero_grad"):
        P.ptg_field(ctx, d, out)
    elif kind.startswith("perlin"):
        P.ptg_perlin(ctx, d, out)
    else:
        P.ptg_opensimplex(ctx, d, out)
    torch.cuda.synchronize()
    return out


def oracle_at(kind, idx, dims=2, spc=64, octaves=6, origin=(0, 0, 0), offset=(0, 0, 0), seed=0,
              persistence=0.5, grad_weight=1.0, lacunarity=2.0, ridged=False):
    """Oracle values at sample indices idx (n, dims) of the window."""
    idx = np.asarray(idx, np.int64) + np.asarray(offset[:dims], np.int64)[None, :]
    size = (spc,) * dims
    cells = (1,) * dims
    return O.field_samples(dims, size, cells, idx, octaves=octaves, method=KIND_ORACLE[kind],
                           persistence=persistence, grad_weight=grad_weight, seed=seed, origin=origin,
                           frequency=lacunarity, ridged=ridged)


def tol32(octaves, persistence=0.5, kind="c1"):
    """FP32 bar, one for every method (polynomial models, Perlin, OpenSimplex,
    ridged noise): max |gpu - oracle| <= 2e-6 x A_tot, A_tot = sum_i |p|^i.
    `kind` is accepted for the callers' convenience and changes nothing."""
    return 2e-6 * W.total_amplitude(octaves, abs(persistence))


def half_ulp16(x):
    a = np.maximum(np.abs(x), 2.0 ** -14)
    return 0.5 * 2.0 ** (np.floor(np.log2(a)) - 10)


def gather(out, idx):
    """Values of `out` at sample indices idx (n, 2 or 3), gathered on the device."""
    ti = torch.from_numpy(np.ascontiguousarray(idx, dtype=np.int64)).to(out.device)
    sel = out[ti[:, 1], ti[:, 0]] if idx.shape[1] == 2 else out[ti[:, 2], ti[:, 1], ti[:, 0]]
    return sel.float().cpu().numpy().astype(np.float64)


def dtype_name(dtype):
    return "f16" if dtype == P.PTG_F16 else "f32"


# ---------------------------------------------------------------------------
# bit-exact hash and coordinates
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims", [2, 3])
def test_hash_bit_exact(ctx, dims):
    n = 1 << 24
    rng = np.random.default_rng(7 + dims)
    keys = rng.integers(0, 2**32, size=(n, dims + 1), dtype=np.uint64).astype(np.uint32)
    m = 1 << 16                                      # structured keys: lattice runs, wrap, octave words
    keys[:m, 0] = np.arange(m, dtype=np.uint32) - np.uint32(m // 2)
    keys[:m, 1] = np.uint32(0xFFFFFFF0)
    keys[:m, dims] = (np.arange(m, dtype=np.uint32) % 24) | (np.uint32(5) << 8)
    kd = torch.from_numpy(keys.view(np.int32)).cuda()
    od = torch.empty_like(kd)
    P.ptg_debug_hash(ctx, dims, kd, od)
    torch.cuda.synchronize()
    got = od.cpu().numpy().view(np.uint32)
    want = O.hash_batch(dims, keys)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("spc", [1, 2, 64, 1024])
def test_axis_bit_exact(ctx, spc):
    rng = np.random.default_rng(spc)
    j = np.concatenate([np.arange(4096), rng.integers(0, 1 << 30, 1 << 16)]).astype(np.int64)
    jd = torch.from_numpy(j).cuda()
    cell = torch.empty(j.size, dtype=torch.int32, device="cuda")
    t = torch.empty(j.size, dtype=torch.float32, device="cuda")
    for origin in (0, -5, 1 << 20, -(1 << 31) + 7):
        for octave in (0, 1, 5, 10, 11, 20, 31):
            P.ptg_debug_axis(ctx, origin, spc, octave, jd, cell, t)
            torch.cuda.synchronize()
            oc, ot = O.axis(origin, spc, j, octave)
            assert np.array_equal(cell.cpu().numpy().view(np.uint32), oc)
            assert np.array_equal(t.cpu().numpy().astype(np.float64), ot)


def test_lattice_octaves_are_exact_corner_values(ctx):
    """spc = 1: every octave samples lattice points.  One octave is the
    corner value itself (exact in FP32); several octaves are a sum whose
    FP32 rounding stays inside the tolerance."""
    for dims, size in [(2, (300, 70)), (3, (40, 24, 9))]:
        for octaves in (1, 3):
            out = gpu_field(ctx, "c1", dims=dims, size=size, spc=1, octaves=octaves, origin=(-3, 1 << 20, 7),
                            seed=99)
            idx = W.grid_indices_2d(*size) if dims == 2 else W.grid_indices_3d(*size)
            ref = oracle_at("c1", idx, dims=dims, spc=1, octaves=octaves, origin=(-3, 1 << 20, 7), seed=99)
            if octaves == 1:
                assert np.array_equal(gather(out, idx), ref)
            else:
                assert np.abs(gather(out, idx) - ref).max() <= tol32(octaves)


# ---------------------------------------------------------------------------
# full-field parity, 256^2 6-octave configuration and every method
# ---------------------------------------------------------------------------
ALL_KINDS = ["c1", "c2", "perlin_s5", "perlin_s3", "opensimplex", "paper_gauge", "zero_grad"]


@pytest.mark.parametrize("dtype", [P.PTG_F32, P.PTG_F16])
@pytest.mark.parametrize("kind", ALL_KINDS)
def test_full_field_256(ctx, kind, dtype):
    """The whole 256^2, 6-octave field (spc 64) of every method, FP32 and FP16
    output; the measured errors go to the error report."""
    cfg = W.CONFIGS["2d_256_c1_n6"]
    out = gpu_field(ctx, kind, size=cfg["size"], spc=cfg["spc"], octaves=cfg["octaves"], seed=0, dtype=dtype)
    rw, nt = launch_of(ctx, kind, cfg["size"], cfg["spc"], cfg["octaves"])
    idx = W.grid_indices_2d(*cfg["size"])
    ref = oracle_at(kind, idx, spc=cfg["spc"], octaves=cfg["octaves"], seed=0)
    err = np.abs(gather(out, idx) - ref)
    bound = tol32(cfg["octaves"]) + (half_ulp16(ref) if dtype == P.PTG_F16 else 0.0)
    errlog.record("2d_256_n6", kind, dtype_name(dtype), err.max(), W.total_amplitude(cfg["octaves"]), err.size,
                  launch=rw_nt_name(kind, rw, nt), bound_ratio=float((err / bound).max()))
    assert np.all(err <= bound), err.max()


@pytest.mark.parametrize("kind", ["c1", "c2", "perlin_s5", "opensimplex", "paper_gauge", "zero_grad"])
@pytest.mark.parametrize("size,spc,octaves", [
    ((1, 1), 1, 1), ((3, 5), 1, 4), ((17, 13), 2, 3), ((200, 136), 8, 7), ((65, 130), 32, 9),
    ((64, 64), 64, 1), ((129, 3), 4, 32),
])
def test_ragged_and_tiny(ctx, kind, size, spc, octaves):
    if kind == "opensimplex" and octaves > 20:
        octaves = 20
    origin = (-(1 << 20) + 3, 12345, 0)
    if kind == "opensimplex":
        origin = (-3, 5, 0)
    out = gpu_field(ctx, kind, size=size, spc=spc, octaves=octaves, origin=origin, seed=17, persistence=0.6,
                    grad_weight=0.75)
    idx = W.grid_indices_2d(*size)
    ref = oracle_at(kind, idx, spc=spc, octaves=octaves, origin=origin, seed=17, persistence=0.6,
                    grad_weight=0.75)
    err = np.abs(gather(out, idx) - ref).max()
    assert err <= tol32(octaves, 0.6, kind), err


@pytest.mark.parametrize("kind", ["c1", "c2", "perlin_s5", "perlin_s3"])
@pytest.mark.parametrize("dtype", [P.PTG_F32, P.PTG_F16])
def test_3d_world_offset(ctx, kind, dtype):
    size, spc, N, origin = (48, 40, 24), 8, 6, (1 << 20, 1 << 20, 0)
    out = gpu_field(ctx, kind, dims=3, size=size, spc=spc, octaves=N, origin=origin, seed=5, dtype=dtype)
    idx = W.grid_indices_3d(*size)
    ref = oracle_at(kind, idx, dims=3, spc=spc, octaves=N, origin=origin, seed=5)
    err = np.abs(gather(out, idx) - ref)
    bound = tol32(N) + (half_ulp16(ref) if dtype == P.PTG_F16 else 0.0)
    assert np.all(err <= bound), err.max()


@pytest.mark.parametrize("spc,N", [(1024, 10), (256, 9), (256, 3), (128, 8), (64, 7)])
def test_3d_c1_tile_octave_counts(ctx, spc, N):
    """3D C1 with six, four, three, three and two octaves of cells >= 32
    samples: summed at the tile nodes from four up, else node-row octaves."""
    size, origin = (70, 36, 20), (1 << 12, -77, 5)
    out = gpu_field(ctx, "c1", dims=3, size=size, spc=spc, octaves=N, origin=origin, seed=8)
    idx = W.grid_indices_3d(*size)
    ref = oracle_at("c1", idx, dims=3, spc=spc, octaves=N, origin=origin, seed=8)
    err = np.abs(gather(out, idx) - ref)
    assert np.all(err <= tol32(N)), err.max()


def test_3d_ragged(ctx):
    size, spc, N = (37, 19, 11), 4, 5
    for kind in ("c1", "c2", "perlin_s5", "perlin_s3"):
        out = gpu_field(ctx, kind, dims=3, size=size, spc=spc, octaves=N, origin=(-7, 3, -(1 << 30)), seed=2)
        idx = W.grid_indices_3d(*size)
        ref = oracle_at(kind, idx, dims=3, spc=spc, octaves=N, origin=(-7, 3, -(1 << 30)), seed=2)
        assert np.abs(gather(out, idx) - ref).max() <= tol32(N)


# ---------------------------------------------------------------------------
# every 2D launch configuration (thread shape 8 x 4 or 16 x 2; coarse octaves
# per run or at the tile nodes) against the oracle
# ---------------------------------------------------------------------------
SHAPES = [P.PTG_SHAPE_8X4, P.PTG_SHAPE_16X2]
TILE_KINDS = ("c1", "perlin_s3", "paper_gauge", "zero_grad")  # degree <= 4


@pytest.mark.parametrize("coarse", [P.PTG_COARSE_RUNS, P.PTG_COARSE_TILE])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind", ["c1", "c2", "perlin_s5", "perlin_s3", "paper_gauge", "zero_grad"])
@pytest.mark.parametrize("size,spc,octaves", [
    ((256, 256), 64, 6),      # one tile octave, run octaves of 32/16-sample cells, then 8, 4, 2
    ((200, 136), 16, 7),      # ragged; one 16-wide run octave, 8/4/2, lattice
    ((130, 70), 2048, 13),    # six tile octaves, two run octaves, 8/4/2, lattice
    ((96, 80), 8, 5),         # no 16-wide run octave
    ((100, 70), 1 << 20, 20),  # fifteen tile octaves
])
def test_launch_configs_vs_oracle(ctx, kind, shape, coarse, size, spc, octaves):
    if coarse == P.PTG_COARSE_TILE and kind not in TILE_KINDS:
        pytest.skip("tile nodes are for models of degree <= 4")
    origin = (-(1 << 20) + 3, 12345, 0)
    out = gpu_field(ctx, kind, size=size, spc=spc, octaves=octaves, origin=origin, seed=21, persistence=0.6,
                    grad_weight=0.75, shape=shape, coarse=coarse)
    rw, nt = P.ptg_launch_config(ctx, P.make_desc(dims=2, size=size, spc=spc, octaves=octaves,
                                                  variant=shape | coarse))
    assert rw == (8 if shape == P.PTG_SHAPE_8X4 else 16)
    n64 = max(0, min(octaves, spc.bit_length() - 6))
    assert nt == (n64 if coarse == P.PTG_COARSE_TILE else 0)
    idx = W.grid_indices_2d(*size)
    ref = oracle_at(kind, idx, spc=spc, octaves=octaves, origin=origin, seed=21, persistence=0.6, grad_weight=0.75)
    err = np.abs(gather(out, idx) - ref).max()
    assert err <= tol32(octaves, 0.6), err


@pytest.mark.parametrize("kind", ["c1", "c2", "perlin_s5", "zero_grad"])
def test_launch_configs_agree(ctx, kind):
    """Same field, every configuration: equal up to FP32 rounding (twice the bar)."""
    coarse = [P.PTG_COARSE_RUNS] + ([P.PTG_COARSE_TILE] if kind in TILE_KINDS else [])
    outs = [gpu_field(ctx, kind, size=(1024, 512), spc=1024, octaves=10, seed=3, shape=sh, coarse=co)
            for sh in SHAPES for co in coarse]
    for b in outs[1:]:
        assert float((outs[0] - b).abs().max()) <= 2 * tol32(10)


@pytest.mark.parametrize("coarse", [P.PTG_COARSE_RUNS, P.PTG_COARSE_TILE])
@pytest.mark.parametrize("shape", SHAPES)
def test_launch_config_fp16_and_mosaic(ctx, shape, coarse):
    big = gpu_field(ctx, "c1", size=(512, 384), spc=1024, octaves=9, origin=(11, -4, 0), seed=8,
                    dtype=P.PTG_F16, shape=shape, coarse=coarse)
    idx = W.subsample((512, 384), every=64, n_random=4096, seed=2)
    ref = oracle_at("c1", idx, spc=1024, octaves=9, origin=(11, -4, 0), seed=8)
    assert np.all(np.abs(gather(big, idx) - ref) <= tol32(9) + half_ulp16(ref))
    part = gpu_field(ctx, "c1", size=(256, 192), spc=1024, octaves=9, origin=(11, -4, 0), offset=(256, 192, 0),
                     seed=8, dtype=P.PTG_F16, shape=shape, coarse=coarse)
    assert torch.equal(part, big[192:384, 256:512])


# ---------------------------------------------------------------------------
# any frequency ratio f between octaves (Sec. 4), per-sample generator
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["c1", "c2", "perlin_s5", "perlin_s3", "paper_gauge", "zero_grad", "opensimplex"])
@pytest.mark.parametrize("f", [1.5, 1.93, 3.0])
@pytest.mark.parametrize("size,spc,octaves,origin", [
    ((256, 192), 64, 6, (0, 0, 0)),
    ((130, 70), 16, 9, (-(1 << 10) + 3, 345, 0)),    # ragged, cells down to a fraction of a sample
    ((96, 64), 1024, 8, (1 << 16, -(1 << 16), 0)),   # world offset, coarse cells
])
def test_any_lacunarity_vs_oracle(ctx, kind, f, size, spc, octaves, origin):
    out = gpu_field(ctx, kind, size=size, spc=spc, octaves=octaves, origin=origin, seed=13, persistence=0.6,
                    grad_weight=0.75, lacunarity=f)
    idx = W.grid_indices_2d(*size)
    ref = oracle_at(kind, idx, spc=spc, octaves=octaves, origin=origin, seed=13, persistence=0.6, grad_weight=0.75,
                    lacunarity=f)
    err = np.abs(gather(out, idx) - ref).max()
    errlog.record("2d_any_frequency_ratio", kind, "f32", err, W.total_amplitude(octaves, 0.6), idx.shape[0])
    assert err <= tol32(octaves, 0.6, kind), err


@pytest.mark.parametrize("kind", ["c1", "perlin_s5", "opensimplex"])
@pytest.mark.parametrize("dims", [2, 3])
def test_large_steps_any_frequency(ctx, kind, dims):
    """Frequency ratio 1.8175 and spc 8 over 12 octaves at persistence 1: the
    finest octaves step about 90 lattice units a sample, so a product's
    rounding error (a few 1e-4 units) must be carried exactly once -- a
    multiply contracted into an FMA with the next subtraction carries it twice
    and shows as errors of 1e-4 per octave."""
    size = (45, 121) if dims == 2 else (40, 21, 9)
    origin, offset = (2216, 407, 0), (69, 99, 5)
    out = gpu_field(ctx, kind, dims=dims, size=size, spc=8, octaves=12, origin=origin, offset=offset, seed=783621,
                    persistence=1.0, lacunarity=1.8175)
    idx = W.grid_indices_2d(*size) if dims == 2 else W.grid_indices_3d(*size)
    ref = oracle_at(kind, idx, dims=dims, spc=8, octaves=12, origin=origin, offset=offset, seed=783621,
                    persistence=1.0, lacunarity=1.8175)
    err = np.abs(gather(out, idx) - ref).max()
    assert err <= tol32(12, 1.0, kind), err


@pytest.mark.parametrize("kind", ["c1", "c2", "perlin_s5", "zero_grad", "opensimplex"])
@pytest.mark.parametrize("spc,f", [(3, 2.0), (100, 2.0), (1000, 2.0), (48, 1.7)])
def test_any_spc_vs_oracle(ctx, kind, spc, f):
    """Samples per cell that are not powers of two (2D, per-sample generator),
    with an unaligned window offset."""
    size, N, origin, offset = (150, 90), 7, (-5, 1 << 12, 0), (7, 13, 0)
    out = gpu_field(ctx, kind, size=size, spc=spc, octaves=N, origin=origin, offset=offset, seed=2,
                    persistence=0.55, lacunarity=f)
    idx = W.grid_indices_2d(*size)
    ref = oracle_at(kind, idx, spc=spc, octaves=N, origin=origin, offset=offset, seed=2, persistence=0.55,
                    lacunarity=f)
    err = np.abs(gather(out, idx) - ref).max()
    errlog.record("2d_any_spc", kind, "f32", err, W.total_amplitude(N, 0.55), idx.shape[0])
    assert err <= tol32(N, 0.55, kind), err


@pytest.mark.parametrize("kind", ["c1", "c2", "perlin_s5", "perlin_s3"])
@pytest.mark.parametrize("spc,f,dtype", [(16, 1.7, P.PTG_F32), (12, 2.0, P.PTG_F32), (128, 2.6, P.PTG_F16),
                                         (5, 1.3, P.PTG_F32)])
def test_3d_any_spc_and_lacunarity_vs_oracle(ctx, kind, spc, f, dtype):
    """3D per-sample generator: cells down to a fraction of a sample, world offset,
    unaligned window offset."""
    size, N, origin, offset = (45, 23, 19), 6, (1 << 12, -3, 77), (5, 9, 3)
    out = gpu_field(ctx, kind, dims=3, size=size, spc=spc, octaves=N, origin=origin, offset=offset, seed=6,
                    lacunarity=f, dtype=dtype)
    idx = W.grid_indices_3d(*size)
    ref = oracle_at(kind, idx, dims=3, spc=spc, octaves=N, origin=origin, offset=offset, seed=6, lacunarity=f)
    err = np.abs(gather(out, idx) - ref)
    bound = tol32(N, kind=kind) + (half_ulp16(ref) if dtype == P.PTG_F16 else 0.0)
    assert np.all(err <= bound), err.max()


# ---------------------------------------------------------------------------
# 3D OpenSimplex-style noise (nineteen candidate vertices per sample, staged
# or hashed gradients, exact or compensated stretched positions)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("size,spc,octaves,origin,offset,f,dtype", [
    ((48, 40, 24), 8, 6, (1 << 12, -3, 77), (0, 0, 0), 2.0, P.PTG_F32),     # staged, then hashed octaves
    ((37, 19, 11), 4, 5, (-7, 3, -5), (0, 0, 0), 2.0, P.PTG_F32),           # ragged
    ((64, 32, 16), 256, 8, (0, 0, 0), (0, 0, 0), 2.0, P.PTG_F32),           # every octave staged
    ((40, 24, 16), 128, 8, (1 << 20, 1 << 20, 0), (64, 32, 8), 2.0, P.PTG_F16),  # world offset (3D bench shape)
    ((33, 20, 17), 12, 6, (5, -9, 2), (3, 7, 1), 2.0, P.PTG_F32),           # spc not a power of two
    ((45, 23, 19), 16, 6, (1 << 10, -3, 77), (5, 9, 3), 1.7, P.PTG_F32),    # any frequency ratio
    ((1, 1, 1), 1, 1, (0, 0, 0), (0, 0, 0), 2.0, P.PTG_F32),
])
def test_3d_opensimplex_vs_oracle(ctx, size, spc, octaves, origin, offset, f, dtype):
    out = gpu_field(ctx, "opensimplex", dims=3, size=size, spc=spc, octaves=octaves, origin=origin, offset=offset,
                    seed=11, persistence=0.6, lacunarity=f, dtype=dtype)
    idx = W.grid_indices_3d(*size)
    ref = oracle_at("opensimplex", idx, dims=3, spc=spc, octaves=octaves, origin=origin, offset=offset, seed=11,
                    persistence=0.6, lacunarity=f)
    err = np.abs(gather(out, idx) - ref)
    bound = tol32(octaves, 0.6, "opensimplex") + (half_ulp16(ref) if dtype == P.PTG_F16 else 0.0)
    errlog.record("3d_small_fields", "opensimplex", dtype_name(dtype), err.max(), W.total_amplitude(octaves, 0.6),
                  err.size, bound_ratio=float((err / bound).max()))
    assert np.all(err <= bound), err.max()


def test_3d_opensimplex_windows_and_host(ctx):
    """Windows of a 3D OpenSimplex field equal the whole field (dyadic steps:
    tile bases are exact), and the banded host output equals the device one."""
    big = gpu_field(ctx, "opensimplex", dims=3, size=(64, 32, 16), spc=16, octaves=7, seed=4)
    part = gpu_field(ctx, "opensimplex", dims=3, size=(32, 16, 8), spc=16, octaves=7, offset=(32, 16, 8), seed=4)
    assert torch.equal(part, big[8:16, 16:32, 32:64])
    d = P.make_desc(dims=3, size=(96, 80, 72), spc=32, octaves=6, seed=6, dtype=P.PTG_F16)
    dev = gpu_field(ctx, "opensimplex", dims=3, size=(96, 80, 72), spc=32, octaves=6, seed=6, dtype=P.PTG_F16)
    host = torch.empty(dev.shape, dtype=dev.dtype).pin_memory()
    P.ptg_generate_host(ctx, d, 2, host)
    assert torch.equal(host, dev.cpu())


# ---------------------------------------------------------------------------
# ridged noise (the paper's ridged mountains, Sec. 5.1): the fused ridged kernel
# (2D, f = 2, tiles aligned to cells) and the per-sample generators
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["c1", "c2", "zero_grad", "paper_gauge", "perlin_s5", "perlin_s3"])
@pytest.mark.parametrize("size,spc,octaves,origin,f,dtype", [
    ((256, 192), 64, 8, (0, 0, 0), 2.0, P.PTG_F32),
    ((130, 70), 1024, 12, (-(1 << 10) + 3, 345, 0), 2.0, P.PTG_F32),   # ragged; down to on-lattice octaves
    ((96, 64), 48, 7, (1 << 12, -5, 0), 1.8, P.PTG_F16),
])
def test_ridged_vs_oracle(ctx, kind, size, spc, octaves, origin, f, dtype):
    out = gpu_field(ctx, kind, size=size, spc=spc, octaves=octaves, origin=origin, seed=19, persistence=0.6,
                    lacunarity=f, dtype=dtype, ridged=True)
    idx = W.grid_indices_2d(*size)
    ref = oracle_at(kind, idx, spc=spc, octaves=octaves, origin=origin, seed=19, persistence=0.6, lacunarity=f,
                    ridged=True)
    err = np.abs(gather(out, idx) - ref)
    bound = tol32(octaves, 0.6, "ridged") + (half_ulp16(ref) if dtype == P.PTG_F16 else 0.0)
    errlog.record("2d_ridged", kind, dtype_name(dtype), err.max(), W.total_amplitude(octaves, 0.6), err.size,
                  bound_ratio=float((err / bound).max()))
    assert np.all(err <= bound), err.max()


@pytest.mark.parametrize("kind", ["c1", "c2", "zero_grad", "paper_gauge", "perlin_s5", "perlin_s3"])
@pytest.mark.parametrize("dtype", [P.PTG_F32, P.PTG_F16])
def test_ridged_8192_n12_sampled(ctx, kind, dtype):
    """The 8192^2, 12-octave field (spc 1024) as ridged noise: the fused ridged
    kernel (aligned tiles), sampled on every 64th row, 2^18 random samples and
    the base lattice's columns."""
    cfg = W.CONFIGS["2d_8192_n12"]
    out = gpu_field(ctx, kind, size=cfg["size"], spc=cfg["spc"], octaves=cfg["octaves"], seed=4, persistence=0.5,
                    dtype=dtype, ridged=True)
    idx = W.subsample(cfg["size"], every=64, n_random=1 << 18, seed=4, lattice_spc=cfg["spc"])
    ref = oracle_at(kind, idx, spc=cfg["spc"], octaves=cfg["octaves"], seed=4, persistence=0.5, ridged=True)
    err = np.abs(gather(out, idx) - ref)
    bound = tol32(cfg["octaves"]) + (half_ulp16(ref) if dtype == P.PTG_F16 else 0.0)
    errlog.record("2d_ridged_8192_n12", kind, dtype_name(dtype), err.max(), W.total_amplitude(cfg["octaves"]),
                  err.size, bound_ratio=float((err / bound).max()))
    assert np.all(err <= bound), err.max()
    del out


@pytest.mark.parametrize("kind", ["c1", "perlin_s5"])
@pytest.mark.parametrize("offset", [(0, 0, 0), (64, 128, 0), (3, 5, 0)])
def test_ridged_windows(ctx, kind, offset):
    """Windows of a ridged world: aligned offsets run the fused ridged kernel,
    unaligned ones the per-sample generator; both match the oracle."""
    size, spc, N = (200, 136), 32, 8
    out = gpu_field(ctx, kind, size=size, spc=spc, octaves=N, origin=(9, -2, 0), offset=offset, seed=6,
                    persistence=0.6, ridged=True)
    idx = W.grid_indices_2d(*size)
    ref = oracle_at(kind, idx, spc=spc, octaves=N, origin=(9, -2, 0), offset=offset, seed=6, persistence=0.6,
                    ridged=True)
    err = np.abs(gather(out, idx) - ref)
    assert np.all(err <= tol32(N, 0.6)), err.max()


@pytest.mark.parametrize("kind", ["c1", "c2", "perlin_s5"])
def test_ridged_3d_vs_oracle(ctx, kind):
    size, spc, N, origin = (45, 23, 19), 16, 6, (1 << 12, -3, 77)
    out = gpu_field(ctx, kind, dims=3, size=size, spc=spc, octaves=N, origin=origin, seed=5, ridged=True)
    idx = W.grid_indices_3d(*size)
    ref = oracle_at(kind, idx, dims=3, spc=spc, octaves=N, origin=origin, seed=5, ridged=True)
    err = np.abs(gather(out, idx) - ref).max()
    errlog.record("3d_ridged", kind, "f32", err, W.total_amplitude(N), idx.shape[0])
    assert err <= tol32(N, kind="ridged"), err


@pytest.mark.parametrize("kind", ["c1", "perlin_s5"])
@pytest.mark.parametrize("offset", [(0, 0, 0), (32, 16, 8), (3, 1, 2)])
def test_ridged_3d_windows(ctx, kind, offset):
    """3D ridged windows: aligned offsets run the fused ridged kernel, unaligned
    ones the per-sample generator; both match the oracle."""
    size, spc, N, origin = (40, 20, 12), 8, 5, (77, -5, 3)
    out = gpu_field(ctx, kind, dims=3, size=size, spc=spc, octaves=N, origin=origin, offset=offset, seed=2,
                    persistence=0.6, ridged=True)
    idx = W.grid_indices_3d(*size)
    ref = oracle_at(kind, idx, dims=3, spc=spc, octaves=N, origin=origin, offset=offset, seed=2, persistence=0.6,
                    ridged=True)
    err = np.abs(gather(out, idx) - ref)
    assert np.all(err <= tol32(N, 0.6)), err.max()


@pytest.mark.parametrize("kind", ["c1", "c2", "perlin_s5"])
def test_ridged_3d_512_n8_sampled(ctx, kind):
    """The 512^3, 8-octave volume (spc 128, origin (2^20, 2^20, 0)) as ridged
    noise, FP16 out, through the fused ridged kernel: every 64th plane, 2^18
    random samples and the base lattice's lines."""
    cfg = W.CONFIGS["3d_512_n8"]
    origin = cfg["origin"]
    out = gpu_field(ctx, kind, dims=3, size=cfg["size"], spc=cfg["spc"], octaves=cfg["octaves"], origin=origin,
                    seed=3, dtype=P.PTG_F16, ridged=True)
    idx = W.subsample(cfg["size"], every=64, n_random=1 << 18, seed=3, lattice_spc=cfg["spc"])
    ref = oracle_at(kind, idx, dims=3, spc=cfg["spc"], octaves=cfg["octaves"], origin=origin, seed=3, ridged=True)
    err = np.abs(gather(out, idx) - ref)
    bound = tol32(cfg["octaves"]) + half_ulp16(ref)
    errlog.record("3d_ridged_512_n8", kind, "f16", err.max(), W.total_amplitude(cfg["octaves"]), err.size,
                  bound_ratio=float((err / bound).max()))
    assert np.all(err <= bound), err.max()
    del out


def test_ridged_is_not_batched(ctx):
    d = P.make_desc(dims=2, size=(64, 64), spc=64, octaves=4, variant=P.PTG_RIDGED)
    out = torch.empty((64, 64), device="cuda")
    with pytest.raises(P.PtgError) as e:
        P.ptg_batch(ctx, [d], [out])
    assert e.value.code == P.PTG_ERR_UNSUPPORTED


@pytest.mark.parametrize("kind", ["c1", "perlin_s5"])
def test_any_lacunarity_fp16_host_and_chunks(ctx, kind):
    f, size, spc, N = 1.75, (1000, 777), 128, 10
    out = gpu_field(ctx, kind, size=size, spc=spc, octaves=N, seed=4, lacunarity=f, dtype=P.PTG_F16)
    idx = W.subsample(size, every=97, n_random=8192, seed=3)
    ref = oracle_at(kind, idx, spc=spc, octaves=N, seed=4, lacunarity=f)
    assert np.all(np.abs(gather(out, idx) - ref) <= tol32(N) + half_ulp16(ref))
    # banded host output equals the device field
    d = P.make_desc(dims=2, size=size, spc=spc, octaves=N, seed=4, lacunarity=f, dtype=P.PTG_F16,
                    variant=P.PTG_PERLIN_S5 if kind == "perlin_s5" else 0)
    host = torch.empty(out.shape, dtype=out.dtype).pin_memory()
    P.ptg_generate_host(ctx, d, 1 if kind == "perlin_s5" else 0, host)
    assert torch.equal(host, out.cpu()) or float((host.float() - out.float().cpu()).abs().max()) <= 2 * tol32(N) + 1e-3
    # a window of the field: the same values to rounding (tile bases are formed per tile in FP64)
    big = gpu_field(ctx, kind, size=(512, 384), spc=spc, octaves=N, seed=4, lacunarity=f)
    part = gpu_field(ctx, kind, size=(256, 192), spc=spc, octaves=N, seed=4, lacunarity=f, offset=(256, 128, 0))
    assert float((part - big[128:320, 256:512]).abs().max()) <= 2 * tol32(N)


# ---------------------------------------------------------------------------
# full-size configurations in the benchmark's launch configuration, sampled
# ---------------------------------------------------------------------------
def launch_of(ctx, kind, size, spc, octaves, shape=P.PTG_SHAPE_AUTO, coarse=0):
    """(run width, tile octaves) a 2D field of this kind gets; (0, 0) for
    OpenSimplex, which has one launch configuration."""
    if kind == "opensimplex":
        return 0, 0
    smooth = SMOOTH.get(kind, P.PTG_C1)
    variant = (P.PTG_PERLIN_S3 if kind == "perlin_s3" else P.PTG_PERLIN_S5) | shape | coarse
    d = P.make_desc(dims=2, size=size, spc=spc, octaves=octaves, smoothness=smooth, variant=variant)
    return P.ptg_launch_config(ctx, d, P.METHOD_PERLIN if kind.startswith("perlin") else P.METHOD_FIELD)


def rw_nt_name(kind, rw, nt):
    if kind == "opensimplex":
        return "opensimplex2d"
    return "%dx%d%s" % (rw, 32 // rw, " tile%d" % nt if nt else "")


def configs_of(kind):
    """Every 2D launch configuration of a kind: thread shapes 8 x 4 and 16 x 2,
    coarse octaves per run, and (degree <= 4) at the tile nodes."""
    if kind == "opensimplex":
        return [(0, 0)]
    coarse = [P.PTG_COARSE_RUNS] + ([P.PTG_COARSE_TILE] if kind in TILE_KINDS else [])
    return [(sh, co) for sh in SHAPES for co in coarse]


SEED_OF = {"c1": 0, "c2": 3, "perlin_s5": 2, "perlin_s3": 1, "opensimplex": 0, "paper_gauge": 1, "zero_grad": 2}


@pytest.mark.parametrize("dtype", [P.PTG_F32, P.PTG_F16])
@pytest.mark.parametrize("kind", ALL_KINDS)
def test_sampled_8192_n12(ctx, kind, dtype):
    """The 8192^2, 12-octave field (spc 1024) in every launch configuration --
    so whichever the autotuner picks for the benchmark is covered -- sampled on
    every 64th row, 2^20 random samples and the base lattice's columns."""
    cfg = W.CONFIGS["2d_8192_n12"]
    seed = SEED_OF[kind]
    idx = W.subsample(cfg["size"], every=64, n_random=1 << 20, seed=seed, lattice_spc=cfg["spc"])
    ref = oracle_at(kind, idx, spc=cfg["spc"], octaves=cfg["octaves"], seed=seed)
    bound = tol32(cfg["octaves"]) + (half_ulp16(ref) if dtype == P.PTG_F16 else 0.0)
    a_tot = W.total_amplitude(cfg["octaves"])
    for shape, coarse in configs_of(kind):
        out = gpu_field(ctx, kind, size=cfg["size"], spc=cfg["spc"], octaves=cfg["octaves"], seed=seed, dtype=dtype,
                        shape=shape or P.PTG_SHAPE_AUTO, coarse=coarse)
        rw, nt = launch_of(ctx, kind, cfg["size"], cfg["spc"], cfg["octaves"], shape or P.PTG_SHAPE_AUTO, coarse)
        err = np.abs(gather(out, idx) - ref)
        errlog.record("2d_8192_n12", kind, dtype_name(dtype), err.max(), a_tot, err.size,
                      launch=rw_nt_name(kind, rw, nt), bound_ratio=float((err / bound).max()))
        assert np.all(err <= bound), (rw_nt_name(kind, rw, nt), err.max())
        # range bound |H| <= (1 + D w beta) A_tot holds on the whole field
        if kind == "c1":
            assert float(out.float().abs().max()) <= 1.5 * a_tot + 1e-5
        del out


@pytest.mark.parametrize("dtype", [P.PTG_F16, P.PTG_F32])
@pytest.mark.parametrize("kind", ["c1", "perlin_s5", "opensimplex"])
def test_sampled_3d_512_n8(ctx, kind, dtype):
    cfg = W.CONFIGS["3d_512_n8"]
    out = gpu_field(ctx, kind, dims=3, size=cfg["size"], spc=cfg["spc"], octaves=cfg["octaves"],
                    origin=cfg["origin"], seed=0, dtype=dtype)
    # every 64th plane, 2^20 random samples and the base lattice's lines along z
    idx = W.subsample(cfg["size"], every=64, n_random=1 << 20, seed=1, lattice_spc=cfg["spc"])
    ref = oracle_at(kind, idx, dims=3, spc=cfg["spc"], octaves=cfg["octaves"], origin=cfg["origin"], seed=0)
    err = np.abs(gather(out, idx) - ref)
    bound = tol32(cfg["octaves"]) + (half_ulp16(ref) if dtype == P.PTG_F16 else 0.0)
    errlog.record("3d_512_n8", kind, dtype_name(dtype), err.max(), W.total_amplitude(cfg["octaves"]), err.size,
                  bound_ratio=float((err / bound).max()))
    assert np.all(err <= bound), err.max()
    del out


# ---------------------------------------------------------------------------
# fields taller than one launch (65535 tiles along the slowest axis) run as
# consecutive launches; the samples on both sides of the seam match the oracle
# and every sample is written
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind,dims,lac", [("c1", 2, 2.0), ("opensimplex", 2, 2.0), ("c1", 2, 1.9),
                                           ("c1", 3, 2.0), ("perlin_s5", 3, 2.0)])
def test_field_taller_than_one_launch(ctx, kind, dims, lac):
    tile = 64 if dims == 2 else 8
    seam = 65535 * tile
    size = (16, seam + 3 * tile + 7) if dims == 2 else (8, 16, seam + 13)
    spc, octaves = (64, 5) if dims == 2 else (32, 5)
    out = gpu_field(ctx, kind, dims=dims, size=size, spc=spc, octaves=octaves, seed=5, lacunarity=lac,
                    origin=(3, -7, 2))
    assert not torch.isnan(out).any()
    rng = np.random.default_rng(11)
    slow = size[dims - 1]
    rows = np.concatenate([np.arange(seam - 6, seam + 6), np.arange(slow - 3, slow), [0, 1]])
    if dims == 2:
        near = np.stack(np.meshgrid(np.arange(size[0]), rows, indexing="ij"), -1).reshape(-1, 2)
    else:
        near = np.stack(np.meshgrid(np.arange(size[0]), np.arange(size[1]), rows, indexing="ij"), -1).reshape(-1, 3)
    rand = np.stack([rng.integers(0, n, 4096) for n in size[:dims]], -1)
    idx = np.concatenate([near, rand]).astype(np.int64)
    ref = oracle_at(kind, idx, dims=dims, spc=spc, octaves=octaves, seed=5, lacunarity=lac, origin=(3, -7, 2))
    err = np.abs(gather(out, idx) - ref)
    assert np.all(err <= tol32(octaves)), err.max()
    del out


# ---------------------------------------------------------------------------
# locality (Sec. 1): windows tile the world exactly; determinism; host path
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["c1", "c2", "perlin_s5", "paper_gauge", "zero_grad"])
def test_chunk_mosaic_bit_exact(ctx, kind):
    big = gpu_field(ctx, kind, size=(512, 384), spc=128, octaves=9, origin=(11, -4, 0), seed=8)
    for oy in (0, 192):
        for ox in (0, 256):
            part = gpu_field(ctx, kind, size=(256, 192), spc=128, octaves=9, origin=(11, -4, 0),
                             offset=(ox, oy, 0), seed=8)
            assert torch.equal(part, big[oy:oy + 192, ox:ox + 256])


@pytest.mark.parametrize("kind", ["c1", "perlin_s5"])
def test_3d_chunk_mosaic_bit_exact(ctx, kind):
    big = gpu_field(ctx, kind, dims=3, size=(64, 32, 16), spc=16, octaves=7, seed=4)
    part = gpu_field(ctx, kind, dims=3, size=(32, 16, 8), spc=16, octaves=7, offset=(32, 16, 8), seed=4)
    assert torch.equal(part, big[8:16, 16:32, 32:64])


def test_deterministic(ctx):
    a = gpu_field(ctx, "c2", size=(1024, 512), spc=256, octaves=10, seed=3)
    b = gpu_field(ctx, "c2", size=(1024, 512), spc=256, octaves=10, seed=3)
    assert torch.equal(a, b)


@pytest.mark.parametrize("method,dims,size,dtype", [
    (0, 2, (2048, 1536), P.PTG_F32), (0, 2, (1000, 777), P.PTG_F16), (1, 2, (2048, 1100), P.PTG_F32),
    (2, 2, (700, 900), P.PTG_F32), (0, 3, (128, 96, 80), P.PTG_F16),
])
def test_generate_host_matches_device(ctx, method, dims, size, dtype):
    kind = ["c1", "perlin_s5", "opensimplex"][method]
    spc = 64 if dims == 2 else 16
    dev = gpu_field(ctx, kind, dims=dims, size=size, spc=spc, octaves=9, seed=6, dtype=dtype)
    d = P.make_desc(dims=dims, size=size, spc=spc, octaves=9, seed=6, dtype=dtype)
    host = torch.empty(dev.shape, dtype=dev.dtype).pin_memory()
    P.ptg_generate_host(ctx, d, method, host)
    assert torch.equal(host, dev.cpu())


def test_short_forms(ctx):
    out = torch.empty((200, 300), dtype=torch.float32, device="cuda")
    P.ptg_heightmap2d(ctx, (300, 200), 5, P.PTG_C2, 0.5, 2.0, 9, out)
    ref = gpu_field(ctx, "c2", size=(300, 200), spc=64, octaves=5, seed=9)
    assert torch.equal(out, ref)
    vol = torch.empty((40, 30, 20), dtype=torch.float32, device="cuda")
    P.ptg_volume3d(ctx, (20, 30, 40), 4, P.PTG_C1, 0.5, 2.0, 9, vol)
    ref3 = gpu_field(ctx, "c1", dims=3, size=(20, 30, 40), spc=64, octaves=4, seed=9)
    assert torch.equal(vol, ref3)


# ---------------------------------------------------------------------------
# argument errors write nothing
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kw,code", [
    (dict(size=(0, 16)), P.PTG_ERR_INVALID), (dict(smoothness=4, dims=3, size=(16, 16, 16)), P.PTG_ERR_UNSUPPORTED),
    (dict(octaves=0), P.PTG_ERR_INVALID), (dict(lacunarity=0.5), P.PTG_ERR_INVALID),
    (dict(smoothness=9), P.PTG_ERR_INVALID), (dict(seed=1 << 24), P.PTG_ERR_INVALID),
])
def test_invalid_arguments_write_nothing(ctx, kw, code):
    args = dict(size=(64, 64), spc=16, octaves=3)
    args.update(kw)
    d = P.make_desc(**args)
    out = torch.full((64, 64), 7.0, device="cuda")
    with pytest.raises(P.PtgError) as e:
        P.ptg_field(ctx, d, out.data_ptr())
    assert e.value.code == code
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())


@pytest.mark.parametrize("dims,size", [(2, (65536, 34000)), (3, (1024, 1024, 2100))])
def test_beyond_2g_elements(ctx, dims, size):
    """Fields of more than 2^31 elements (FP16, about 4.4 GB): 64-bit output
    offsets; samples from the first and last rows / planes against the oracle."""
    n = int(np.prod(size))
    assert n > 2**31
    out = gpu_field(ctx, "c1", dims=dims, size=size, spc=1024 if dims == 2 else 128, octaves=8, seed=3,
                    dtype=P.PTG_F16)
    rng = np.random.default_rng(dims)
    k = 4096
    idx = np.stack([rng.integers(0, s, k) for s in size[:-1]] +
                   [np.concatenate([rng.integers(0, 8, k // 2), size[-1] - 1 - rng.integers(0, 8, k // 2)])], 1)
    ti = torch.from_numpy(idx.astype(np.int64)).cuda()
    sel = out[ti[:, 1], ti[:, 0]] if dims == 2 else out[ti[:, 2], ti[:, 1], ti[:, 0]]  # gathered on the device
    got = sel.float().cpu().numpy().astype(np.float64)
    ref = oracle_at("c1", idx, dims=dims, spc=1024 if dims == 2 else 128, octaves=8, seed=3)
    assert np.all(np.abs(got - ref) <= tol32(8) + half_ulp16(ref))
    del out
    torch.cuda.empty_cache()
