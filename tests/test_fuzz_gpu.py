"""Randomised parity: seeded random descriptors -- every generator, 2D and 3D,
powers of two and other spc, frequency ratios, origins on both sides of zero,
window offsets, octave counts, persistence, gradient weight, FP32/FP16,
ridged noise, thread shapes and coarse-octave modes -- against the oracle on
whole small fields, with the bars of test_parity_gpu (fractal sum of Sec. 4;
cell polynomials of Sec. 2-3)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1610_03525_gb300 as P  # noqa: E402
from paper_1610_03525_gb300 import workloads as W  # noqa: E402
import errlog  # noqa: E402
from test_parity_gpu import dtype_name, gather, gpu_field, half_ulp16, oracle_at, tol32  # noqa: E402

pytestmark = pytest.mark.gpu

KINDS_2D = ["c1", "c2", "paper_gauge", "zero_grad", "perlin_s5", "perlin_s3", "opensimplex"]
KINDS_3D = ["c1", "c2", "perlin_s5", "perlin_s3", "opensimplex"]
DEGREE_LE4 = {"c1", "paper_gauge", "zero_grad", "perlin_s3"}
N_CASES = 72


def draw(idx, wrap=False):
    """One random case: a dict of gpu_field keyword arguments plus the kind.
    wrap: fused generators only (power-of-two spc, f = 2), origins anywhere in
    the 32-bit lattice (cell indices wrap mod 2^32) and up to 24 octaves."""
    rng = np.random.default_rng(20161012 + idx + (100000 if wrap else 0))
    dims = 3 if rng.random() < 0.3 else 2
    kinds = KINDS_3D if dims == 3 else KINDS_2D
    if wrap:
        kinds = [k for k in kinds if k != "opensimplex"]
    kind = str(rng.choice(kinds))
    spc = int(2 ** rng.integers(0, 12)) if wrap or rng.random() < 0.6 else int(rng.integers(1, 301))
    f = 2.0 if wrap or rng.random() < 0.7 else float(np.float32(rng.uniform(1.2, 3.5)))
    ridged = kind != "opensimplex" and not wrap and rng.random() < 0.2
    if dims == 2:
        size = (int(rng.integers(1, 151)), int(rng.integers(1, 151)), 1)
    else:
        size = (int(rng.integers(1, 41)), int(rng.integers(1, 31)), int(rng.integers(1, 21)))
    fused = spc & (spc - 1) == 0 and f == 2.0 and not ridged and kind != "opensimplex"
    tile = (64, 64, 1) if dims == 2 else (32, 16, 8)
    offset = []
    for k in range(dims):
        if fused:
            offset.append(int(rng.integers(0, 4)) * min(spc, tile[k]))
        else:
            offset.append(int(rng.integers(0, 101)))
    offset += [0] * (3 - dims)
    lim = (1 << 31) if wrap else (1 << 12)
    origin = [int(rng.integers(-lim, lim + 1)) for _ in range(dims)] + [0] * (3 - dims)
    if wrap:
        octaves = int(rng.integers(1, 25))
    else:
        # octaves: as many as keep every lattice coordinate below 2^30 (and at most 14)
        extent = max(abs(origin[k]) + (offset[k] + size[k]) / spc for k in range(dims))
        nmax = 1
        while nmax < 14 and extent * f ** nmax < 2 ** 29:
            nmax += 1
        octaves = int(rng.integers(1, nmax + 1))
    kw = dict(dims=dims, size=size[:dims] if dims == 3 else size[:2], spc=spc, octaves=octaves,
              origin=tuple(origin), offset=tuple(offset), seed=int(rng.integers(0, 1 << 24)),
              persistence=float(np.float32(rng.uniform(0.3, 0.9))), lacunarity=f, ridged=ridged,
              dtype=P.PTG_F16 if rng.random() < 0.2 else P.PTG_F32)
    if kind in ("c1", "c2", "paper_gauge", "zero_grad"):
        kw["grad_weight"] = float(np.float32(rng.uniform(0.0, 1.0)))
    if dims == 2 and fused:
        kw["shape"] = int(rng.choice([P.PTG_SHAPE_AUTO, P.PTG_SHAPE_8X4, P.PTG_SHAPE_16X2]))
        modes = [0, P.PTG_COARSE_RUNS] + ([P.PTG_COARSE_TILE] if kind in DEGREE_LE4 else [])
        kw["coarse"] = int(rng.choice(modes))
    return kind, kw


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03525_gb300 import build
    build.build()
    c = P.ptg_create(0)
    yield c
    c.close()


@pytest.mark.parametrize("idx,wrap", [(i, False) for i in range(N_CASES)] + [(i, True) for i in range(24)])
def test_random_descriptor_vs_oracle(ctx, idx, wrap):
    kind, kw = draw(idx, wrap)
    method = 2 if kind == "opensimplex" else (1 if kind.startswith("perlin") else 0)
    variant = (P.PTG_PERLIN_S3 if kind == "perlin_s3" else 0) | kw.get("shape", 0) | kw.get("coarse", 0)
    variant |= P.PTG_RIDGED if kw["ridged"] else 0
    smooth = {"c2": P.PTG_C2, "paper_gauge": P.PTG_PAPER_D2M1N3, "zero_grad": P.PTG_ZERO_GRADIENT}.get(kind, P.PTG_C1)
    d = P.make_desc(dims=kw["dims"], size=kw["size"], spc=kw["spc"], origin=kw["origin"], offset=kw["offset"],
                    octaves=kw["octaves"], smoothness=smooth, persistence=kw["persistence"],
                    grad_weight=kw.get("grad_weight", 1.0), seed=kw["seed"], dtype=kw["dtype"], variant=variant,
                    lacunarity=kw["lacunarity"])
    rc, msg = P.ptg_validate(d, method)
    if rc != P.PTG_OK:
        pytest.skip("descriptor outside the supported range: " + msg)
    out = gpu_field(ctx, kind, **kw)
    dims = kw["dims"]
    idxs = W.grid_indices_2d(*kw["size"]) if dims == 2 else W.grid_indices_3d(*kw["size"])
    ref = oracle_at(kind, idxs, dims=dims, spc=kw["spc"], octaves=kw["octaves"], origin=kw["origin"],
                    offset=kw["offset"], seed=kw["seed"], persistence=kw["persistence"],
                    grad_weight=kw.get("grad_weight", 1.0), lacunarity=kw["lacunarity"], ridged=kw["ridged"])
    got = gather(out, idxs)
    assert np.all(np.isfinite(got))
    bar = tol32(kw["octaves"], kw["persistence"])
    bound = bar + (half_ulp16(ref) if kw["dtype"] == P.PTG_F16 else 0.0)
    err = np.abs(got - ref)
    errlog.record("fuzz" + ("_ridged" if kw["ridged"] else ""), kind, dtype_name(kw["dtype"]), err.max(),
                  W.total_amplitude(kw["octaves"], kw["persistence"]), err.size,
                  bound_ratio=float((err / bound).max()))
    assert np.all(err <= bound), (kind, kw, float(err.max()))
