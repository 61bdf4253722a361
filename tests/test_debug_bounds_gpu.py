"""Debug build (libptg_debug.so, the same sources compiled with
-DPTG_DEBUG_BOUNDS): the checked kernels test every shared-memory and global
index before use, skip and record a violation instead of faulting.  Small and
odd-sized fields (1 x 1 up to a few ragged tiles) in every launch
configuration must match the FP64 oracle with no violation recorded; the
recording path itself is exercised by a self-test kernel that evaluates an
out-of-range check without touching memory there.  The debug library runs in
a child process of its own (it is built on first use)."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

import paper_1610_03525_gb300 as P  # noqa: E402

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, sys.argv[1] + "/tests")
import numpy as np, torch
import oracle as O
import paper_1610_03525_gb300 as P
from paper_1610_03525_gb300 import workloads as W
assert P.LIB_PATH.endswith("libptg_debug.so"), P.LIB_PATH
ORC = {"c1": O.C1, "c2": O.C2, "perlin_s5": O.PERLIN_S5, "perlin_s3": O.PERLIN_S3, "paper_gauge": O.PAPER_GAUGE,
       "zero_grad": O.ZERO_GRAD, "opensimplex": O.OPENSIMPLEX}
SM = {"c2": P.PTG_C2, "paper_gauge": P.PTG_PAPER_D2M1N3, "zero_grad": P.PTG_ZERO_GRADIENT}
ctx = P.ptg_create(0)
res = {"cases": 0, "violations": [], "worst": 0.0}

def run(kind, dims, size, spc, N, variant=0, origin=(-(1 << 20) + 3, 12345, 7), p=0.6, w=0.75, ridged=False):
    smooth = SM.get(kind, P.PTG_C1)
    var = variant | (P.PTG_PERLIN_S3 if kind == "perlin_s3" else 0) | (P.PTG_RIDGED if ridged else 0)
    d = P.make_desc(dims=dims, size=size, spc=spc, origin=origin, octaves=N, smoothness=smooth, persistence=p,
                    grad_weight=w, seed=31, variant=var)
    out = torch.full(tuple(reversed(size)), float("nan"), device="cuda")
    fn = P.ptg_opensimplex if kind == "opensimplex" else (P.ptg_perlin if kind.startswith("perlin") else P.ptg_field)
    fn(ctx, d, out)
    first = P.ptg_debug_bounds(ctx)
    idx = W.grid_indices_2d(*size) if dims == 2 else W.grid_indices_3d(*size)
    ref = O.field_samples(dims, (spc,) * dims, (1,) * dims, idx, octaves=N, method=ORC[kind], persistence=p,
                          grad_weight=w, seed=31, origin=origin, ridged=ridged)
    a = out.cpu().numpy()
    got = a[idx[:, 1], idx[:, 0]] if dims == 2 else a[idx[:, 2], idx[:, 1], idx[:, 0]]
    err = float(np.abs(got.astype(np.float64) - ref).max()) / W.total_amplitude(N, p)
    res["cases"] += 1
    res["worst"] = max(res["worst"], err if np.isfinite(err) else 1e30)
    if first:
        res["violations"].append([kind, dims, list(size), spc, N, variant, first >> 48, first & ((1 << 48) - 1)])

sizes2 = [(1, 1), (3, 5), (17, 13), (64, 64), (65, 33), (130, 70)]
cfgs = [P.PTG_SHAPE_8X4 | P.PTG_COARSE_RUNS, P.PTG_SHAPE_8X4 | P.PTG_COARSE_TILE,
        P.PTG_SHAPE_16X2 | P.PTG_COARSE_RUNS, P.PTG_SHAPE_16X2 | P.PTG_COARSE_TILE]
for kind in ["c1", "c2", "perlin_s5", "perlin_s3", "paper_gauge", "zero_grad"]:
    for size in sizes2:
        for spc, N in [(1, 2), (2, 3), (8, 6), (64, 9), (1024, 13)]:
            for v in cfgs:
                if v & P.PTG_COARSE_TILE and kind in ("c2", "perlin_s5"):
                    continue
                run(kind, 2, size, spc, N, v)
for size in [(1, 1), (17, 13), (130, 70)]:
    for spc, N in [(1, 2), (16, 5), (1024, 12)]:
        run("opensimplex", 2, size, spc, N, origin=(-3, 5, 0))
for kind in ["c1", "zero_grad", "paper_gauge", "perlin_s5"]:  # the fused ridged kernel
    for size in [(1, 1), (17, 13), (130, 70)]:
        for spc, N in [(1, 2), (2, 3), (8, 6), (64, 9), (1024, 12)]:
            run(kind, 2, size, spc, N, origin=(-(1 << 10) + 3, 345, 0), ridged=True)
for kind in ["c1", "c2", "perlin_s5"]:  # the fused ridged kernel, 3D
    for size in [(1, 1, 1), (5, 3, 2), (37, 19, 11)]:
        for spc, N in [(1, 2), (4, 5), (32, 8)]:
            run(kind, 3, size, spc, N, origin=(-(1 << 10) + 3, 345, 7), ridged=True)
for kind in ["c1", "c2", "perlin_s5", "perlin_s3"]:
    for size in [(1, 1, 1), (5, 3, 2), (37, 19, 11)]:
        for spc, N in [(1, 2), (4, 5), (32, 8)]:
            run(kind, 3, size, spc, N)
# a batch of small uneven fields through the persistent kernel
descs = [P.make_desc(dims=2, size=sz, spc=64, octaves=n, seed=k, smoothness=P.PTG_C1 if k % 2 else P.PTG_C2)
         for k, (sz, n) in enumerate([((64, 64), 7), ((128, 64), 4), ((64, 192), 9), ((192, 128), 12)])]
outs = [torch.empty((d.size[1], d.size[0]), device="cuda") for d in descs]
P.ptg_batch(ctx, descs, outs)
first = P.ptg_debug_bounds(ctx)
res["cases"] += 1
if first:
    res["violations"].append(["batch", first >> 48, first & ((1 << 48) - 1)])
# the recording path: first record kept, cleared by reading
P.ptg_debug_bounds_selftest(ctx, 15, 5, 10)          # in range: nothing recorded
res["selftest_in_range"] = P.ptg_debug_bounds(ctx)
P.ptg_debug_bounds_selftest(ctx, 15, 1000, 10)
P.ptg_debug_bounds_selftest(ctx, 15, 2000, 10)
res["selftest_first"] = P.ptg_debug_bounds(ctx)
res["selftest_cleared"] = P.ptg_debug_bounds(ctx)
ctx.close()
print("RESULT " + json.dumps(res))
"""


def test_regular_library_has_no_bounds_checks():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03525_gb300 import build
    build.build()
    ctx = P.ptg_create(0)
    try:
        with pytest.raises(P.PtgError) as e:
            P.ptg_debug_bounds(ctx)
        assert e.value.code == P.PTG_ERR_UNSUPPORTED
    finally:
        ctx.close()


def test_debug_build_small_fields_record_no_violation():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03525_gb300 import build
    lib = build.build(debug_bounds=True)
    env = dict(os.environ, PTG_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True, env=env, timeout=900)
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")]
    assert r.returncode == 0 and line, r.stderr[-3000:]
    res = json.loads(line[0][7:])
    assert res["cases"] > 400
    assert res["violations"] == []
    assert res["worst"] <= 2e-6, res["worst"]
    assert res["selftest_in_range"] == 0
    assert res["selftest_first"] == (15 << 48) | 1000
    assert res["selftest_cleared"] == 0
