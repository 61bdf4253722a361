"""ptg_batch_noalloc: batched generation for callers that cannot allocate
device memory (an engine with its own fixed arena, or a real-time loop that
must not pay cudaMalloc's device synchronisation).  Its launch plans and
work counter live in a fixed device array inside the library; its results
must match ptg_batch's, call after call.  This file is collected last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1610_03525_gb300 as P  # noqa: E402
from paper_1610_03525_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


def _fields(n, seed):
    descs, outs = [], []
    for k, c in enumerate(W.chunk_batch(n, seed=seed)):
        dtype = P.PTG_F16 if k % 7 == 3 else P.PTG_F32
        descs.append(P.make_desc(dims=2, size=c["size"], spc=c["spc"], origin=c["origin"], octaves=c["octaves"],
                                 smoothness=c["smoothness"], seed=c["seed"], dtype=dtype))
        outs.append(torch.full((c["size"][1], c["size"][0]), float("nan"),
                               dtype=torch.float16 if dtype == P.PTG_F16 else torch.float32, device="cuda"))
    return descs, outs


def _call_noalloc(ctx, descs, outs):
    """Straight through the C ABI."""
    n = len(descs)
    arr = (P.ptg_field_desc * n)(*descs)
    ptrs = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    stream = torch.cuda.current_stream().cuda_stream
    return P.lib().ptg_batch_noalloc(ctx.handle, arr, ptrs, n, stream)


def test_noalloc_matches_ptg_batch_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03525_gb300 import build
    build.build()
    ctx = P.ptg_create(0)
    try:
        for call, (n, seed) in enumerate([(120, 11), (200, 12)]):
            descs, outs = _fields(n, seed)
            refs = [torch.empty_like(o) for o in outs]
            P.ptg_batch(ctx, descs, refs)
            assert _call_noalloc(ctx, descs, outs) == P.PTG_OK, P.ptg_last_error(ctx)
            torch.cuda.synchronize()
            for d, o, r in zip(descs, outs, refs):
                tol = 2e-6 * W.total_amplitude(d.octaves)
                err = (o.float() - r.float()).abs().max().item()
                assert np.isfinite(err) and err <= tol, (call, err)
    finally:
        ctx.close()


def test_noalloc_rejects_more_than_256_fields():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = P.ptg_create(0)
    try:
        d = P.make_desc(dims=2, size=(64, 64), spc=64, octaves=2)
        out = torch.empty((64, 64), device="cuda")
        rc = _call_noalloc(ctx, [d] * 257, [out] * 257)
        assert rc == P.PTG_ERR_INVALID
        assert "256" in P.ptg_last_error(ctx)
    finally:
        ctx.close()
