"""ptg_batch_noalloc: batched generation for callers that cannot allocate
device memory (an engine with its own fixed arena, or a real-time loop that
must not pay cudaMalloc's device synchronisation).  Its launch plans and
work counter live in a fixed device array inside the library; both calls run
the same persistent kernel on the same plans as ptg_batch, so its results
must equal ptg_batch's bit for bit, call after call.  This file is collected
last, and each test also runs alone in a fresh process."""
import ctypes

import pytest

torch = pytest.importorskip("torch")

import paper_1610_03525_gb300 as P  # noqa: E402
from paper_1610_03525_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

MAX_FIELDS = 256
TWO_MIB = 2 << 20  # the smallest device allocation cudaMalloc reserves


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


@pytest.fixture()
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03525_gb300 import build
    build.build()
    c = P.ptg_create(0)
    yield c
    c.close()


def test_noalloc_matches_ptg_batch_on_two_calls(ctx):
    for call, (n, seed) in enumerate([(120, 11), (200, 12)]):
        descs, outs = _fields(n, seed)
        refs = [torch.empty_like(o) for o in outs]
        P.ptg_batch(ctx, descs, refs)
        assert _call_noalloc(ctx, descs, outs) == P.PTG_OK, P.ptg_last_error(ctx)
        torch.cuda.synchronize()
        for k, (o, r) in enumerate(zip(outs, refs)):
            assert torch.equal(o, r), (call, k)


def test_noalloc_full_batch_allocates_nothing(ctx):
    """256 fields (the stated maximum) are accepted; once the first call has
    looked up the array's address, further calls leave the device's free
    memory unchanged (any cudaMalloc would reserve at least 2 MiB)."""
    descs, outs = _fields(MAX_FIELDS, 13)
    refs = [torch.empty_like(o) for o in outs]
    P.ptg_batch(ctx, descs, refs)
    assert _call_noalloc(ctx, descs, outs) == P.PTG_OK, P.ptg_last_error(ctx)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _call_noalloc(ctx, descs, outs) == P.PTG_OK, P.ptg_last_error(ctx)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 < TWO_MIB, (free0, free1)
    for k, (o, r) in enumerate(zip(outs, refs)):
        assert torch.equal(o, r), k


def test_noalloc_rejects_more_than_256_fields(ctx):
    d = P.make_desc(dims=2, size=(64, 64), spc=64, octaves=2)
    out = torch.empty((64, 64), device="cuda")
    rc = _call_noalloc(ctx, [d] * (MAX_FIELDS + 1), [out] * (MAX_FIELDS + 1))
    assert rc == P.PTG_ERR_INVALID
    assert "256" in P.ptg_last_error(ctx)
    # a later good call clears the message; a bad field is named by its index
    assert _call_noalloc(ctx, [d], [out]) == P.PTG_OK
    assert P.ptg_last_error(ctx) == ""
    bad = P.make_desc(dims=2, size=(64, 64), spc=64, octaves=0)
    assert _call_noalloc(ctx, [d, bad], [out, out]) == P.PTG_ERR_INVALID
    assert "batch field 1" in P.ptg_last_error(ctx)


def test_noalloc_large_fields_take_tile_groups(ctx):
    """A few large fields (32,775 tiles, 36 per resident CTA on a 152-SM
    GB300): the kernel hands out 4 tiles at a time, groups cross field
    boundaries, and the output equals one ptg_field launch per field bit for
    bit, on two calls in a row."""
    descs, outs, refs = [], [], []
    for k, (w, h, sm) in enumerate([(8192, 4096, P.PTG_C1), (4096, 8192, P.PTG_C2), (8192, 4096, P.PTG_C1),
                                    (8192, 4096, P.PTG_ZERO_GRADIENT), (64, 64, P.PTG_C1), (192, 128, P.PTG_C2)]):
        d = P.make_desc(dims=2, size=(w, h), spc=1024, origin=(k * 3, -k, 0), octaves=12, smoothness=sm, seed=k)
        descs.append(d)
        outs.append(torch.full((h, w), float("nan"), device="cuda"))
        refs.append(torch.empty((h, w), device="cuda"))
        P.ptg_field(ctx, d, refs[-1])
    torch.cuda.synchronize()
    for call in range(2):
        for o in outs:
            o.fill_(float("nan"))
        assert _call_noalloc(ctx, descs, outs) == P.PTG_OK, P.ptg_last_error(ctx)
        torch.cuda.synchronize()
        for k, (o, r) in enumerate(zip(outs, refs)):
            assert torch.equal(o, r), (call, k)
