"""Request loop: admission under the HBM budget, overlap on worker streams,
results identical alone and in the mix, timestamps, cancel and timeouts
(the stall is made on the host; no device wait is involved)."""
import pytest

torch = pytest.importorskip("torch")

import paper_1610_03525_gb300 as P  # noqa: E402
from paper_1610_03525_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


def _ctx(budget=0):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03525_gb300 import build
    build.build()
    return P.ptg_create(0, budget)


def _requests(n, seed=12345, scale=4):
    """The serving mix, with sides divided by `scale` to keep the test short."""
    reqs = W.request_stream(rate_hz=20000.0, duration_s=1.0, seed=seed)[:n]
    out = []
    for r in reqs:
        if r["dims"] == 2:
            side = max(64, r["size"][0] // scale // 64 * 64)
            size = (side, side)
        else:
            side = max(32, r["size"][0] // scale // 32 * 32)
            size = (side, side, side)
        d = P.make_desc(dims=r["dims"], size=size, spc=r["spc"], origin=r["origin"], octaves=r["octaves"],
                        smoothness=r["smoothness"], seed=r["seed"])
        out.append(d)
    return out


def _buf(d):
    shape = tuple(reversed([d.size[k] for k in range(d.dims)]))
    return torch.full(shape, float("nan"), device="cuda")


def test_mix_equals_alone_and_timestamps():
    ctx = _ctx(budget=64 << 20)
    try:
        descs = _requests(60)
        alone = []
        for d in descs:
            o = _buf(d)
            P.ptg_field(ctx, d, o)
            alone.append(o)
        torch.cuda.synchronize()
        outs = [_buf(d) for d in descs]
        ids = [P.ptg_submit(ctx, d, o) for d, o in zip(descs, outs)]
        for i in ids:
            assert P.ptg_wait(ctx, i, 30_000_000_000) == P.PTG_OK
        spans = []
        for i, d, o, a in zip(ids, descs, outs, alone):
            st, ts = P.ptg_poll(ctx, i)
            assert st == P.PTG_OK
            assert 0 < ts[0] <= ts[1] <= ts[2] <= ts[3]
            nbytes = 4 * o.numel()
            spans.append((ts[1], ts[3], nbytes))
            assert torch.equal(o, a)
        # admitted bytes never exceed the budget: check at every admit time
        for t, _, _ in spans:
            live = sum(b for (a0, e0, b) in spans if a0 <= t < e0)
            assert live <= 64 << 20
        # the record is released after the final status was polled
        with pytest.raises(P.PtgError):
            P.ptg_poll(ctx, ids[0])
    finally:
        ctx.close()


def test_budget_rejects_oversized_request():
    ctx = _ctx(budget=1 << 20)
    try:
        d = P.make_desc(dims=2, size=(1024, 1024), spc=64, octaves=4)
        with pytest.raises(P.PtgError) as e:
            P.ptg_submit(ctx, d, _buf(d))
        assert e.value.code == P.PTG_ERR_BUDGET
    finally:
        ctx.close()


def test_cancel_and_timeout_with_host_stall():
    ctx = _ctx(budget=6 << 20)
    try:
        d = P.make_desc(dims=2, size=(1024, 1024), spc=256, octaves=6)   # 4 MB each: one fits the budget
        outs = [_buf(d) for _ in range(4)]
        P.ptg_debug_hold(ctx, 1)
        ids = [P.ptg_submit(ctx, d, o) for o in outs]
        # the first request's stream is held on the host: it cannot finish
        assert P.ptg_wait(ctx, ids[0], 50_000_000) == P.PTG_ERR_TIMEOUT
        for i in ids[1:]:
            st, ts = P.ptg_poll(ctx, i)
            assert st == P.PTG_PENDING and ts[1] == 0        # not admitted: budget full
        P.ptg_cancel(ctx, ids[3])
        P.ptg_debug_hold(ctx, 0)
        for i in ids[:3]:
            assert P.ptg_wait(ctx, i, 30_000_000_000) == P.PTG_OK
        assert P.ptg_wait(ctx, ids[3], 1_000_000) == P.PTG_ERR_CANCELLED
        st, _ = P.ptg_poll(ctx, ids[3])
        assert st == P.PTG_ERR_CANCELLED
        ref = _buf(d)
        P.ptg_field(ctx, d, ref)
        torch.cuda.synchronize()
        for o in outs[:3]:
            assert torch.equal(o, ref)
    finally:
        ctx.close()


def test_unknown_request():
    ctx = _ctx()
    try:
        with pytest.raises(P.PtgError) as e:
            P.ptg_poll(ctx, 12345)
        assert e.value.code == P.PTG_ERR_INVALID
    finally:
        ctx.close()


def test_per_sample_requests_in_the_mix():
    """Ridged fields, other frequency ratios and spc that are not powers of
    two go through the request loop too (the per-sample generators), with the
    same values as a direct call."""
    ctx = _ctx(budget=256 << 20)
    try:
        descs = [P.make_desc(dims=2, size=(300, 200), spc=100, octaves=7, seed=1),
                 P.make_desc(dims=2, size=(256, 256), spc=64, octaves=9, seed=2, variant=P.PTG_RIDGED),
                 P.make_desc(dims=2, size=(128, 96), spc=1024, octaves=12, seed=3, lacunarity=1.9),
                 P.make_desc(dims=3, size=(40, 24, 16), spc=16, octaves=6, seed=4, lacunarity=1.7),
                 P.make_desc(dims=3, size=(64, 32, 16), spc=16, octaves=6, seed=5, smoothness=P.PTG_C2,
                             variant=P.PTG_RIDGED)]
        alone = []
        for d in descs:
            o = _buf(d)
            P.ptg_field(ctx, d, o)
            alone.append(o)
        torch.cuda.synchronize()
        outs = [_buf(d) for d in descs]
        ids = [P.ptg_submit(ctx, d, o) for d, o in zip(descs, outs)]
        for i in ids:
            assert P.ptg_wait(ctx, i, 30_000_000_000) == P.PTG_OK
            assert P.ptg_poll(ctx, i)[0] == P.PTG_OK
        for o, a in zip(outs, alone):
            assert torch.equal(o, a)
    finally:
        ctx.close()


_NVTX_CHILD = r"""
import sys, torch
sys.path.insert(0, sys.argv[1])
import paper_1610_03525_gb300 as P
ctx = P.ptg_create(0, 64 << 20)
descs = [P.make_desc(dims=2, size=(256, 128), spc=1024, octaves=6, seed=k) for k in range(12)]
outs = [torch.empty((128, 256), device="cuda") for _ in descs]
ids = [P.ptg_submit(ctx, d, o) for d, o in zip(descs, outs)]
for i in ids:
    assert P.ptg_wait(ctx, i, 30_000_000_000) == P.PTG_OK
    P.ptg_poll(ctx, i)
ctx.close()
"""


def test_nvtx_ranges_of_the_request_loop(tmp_path):
    """The request loop's NVTX ranges, as an NVTX tool sees them: a minimal
    tool (tests/nvtx_probe.c, loaded by NVTX through NVTX_INJECTION64_PATH)
    counts the ranges and marks of a child process that serves 12 requests."""
    import os
    import shutil
    import subprocess
    import sys
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler for the NVTX probe")
    from paper_1610_03525_gb300 import build
    build.build()
    here = os.path.dirname(os.path.abspath(__file__))
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    probe = str(tmp_path / "nvtx_probe.so")
    subprocess.run([gcc, "-shared", "-fPIC", "-O2", "-I", cuda_inc, os.path.join(here, "nvtx_probe.c"), "-o", probe,
                    "-lpthread"], check=True)
    log = tmp_path / "nvtx.log"
    env = dict(os.environ, NVTX_INJECTION64_PATH=probe, PTG_NVTX_LOG=str(log))
    subprocess.run([sys.executable, "-c", _NVTX_CHILD, os.path.dirname(here)], check=True, env=env, timeout=300)
    seen = {}
    for line in log.read_text().splitlines():
        key, count = line.rsplit("\t", 1)
        seen[key] = int(count)
    assert seen.get("push ptg_submit") == 12
    assert seen.get("push ptg_admit") == 12
    assert seen.get("push ptg_launch") == 12
    assert seen.get("mark ptg_complete") == 12
    assert seen.get("start ptg_request") == 12
    assert seen.get("end ", 0) >= 12
    assert seen.get("pop ", 0) >= 36
