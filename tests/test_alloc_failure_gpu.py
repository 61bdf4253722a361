"""Memory exhaustion, injected on the host (ptg_debug_fail_alloc): every call
that needs a device or pinned-host allocation returns PTG_ERR_NOMEM and writes
nothing, and the same call succeeds once the injection is spent.  No GPU
fault is involved: the failed allocations are never attempted."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1610_03525_gb300 as P  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture()
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03525_gb300 import build
    build.build()
    c = P.ptg_create(0)  # fresh: no staging or batch buffers allocated yet
    yield c
    c.close()


def _nomem(fn):
    with pytest.raises(P.PtgError) as e:
        fn()
    assert e.value.code == P.PTG_ERR_NOMEM


def test_generate_host_nomem_writes_nothing(ctx):
    d = P.make_desc(dims=2, size=(640, 300), spc=64, octaves=7, seed=3)
    host = torch.full((300, 640), 7.0).pin_memory()
    P.ptg_debug_fail_alloc(ctx, 1)
    _nomem(lambda: P.ptg_generate_host(ctx, d, P.METHOD_FIELD, host))
    assert bool((host == 7.0).all())
    P.ptg_generate_host(ctx, d, P.METHOD_FIELD, host)  # the injection is spent
    dev = torch.empty((300, 640), device="cuda")
    P.ptg_field(ctx, d, dev)
    torch.cuda.synchronize()
    assert torch.equal(host, dev.cpu())


@pytest.mark.parametrize("after", range(5))
def test_batch_nomem_at_each_allocation(ctx, after):
    """ptg_batch's allocations (plans, tile offsets, counter on the device;
    pinned plan and tile staging) succeed up to the `after`-th and the next
    fails: PTG_ERR_NOMEM, what was allocated is freed, no output is written,
    and the next call allocates afresh and succeeds."""
    descs = [P.make_desc(dims=2, size=(128, 64), spc=64, octaves=5, seed=k) for k in range(3)]
    outs = [torch.full((64, 128), 7.0, device="cuda") for _ in descs]
    P.ptg_debug_fail_alloc(ctx, 1, after=after)
    _nomem(lambda: P.ptg_batch(ctx, descs, outs))
    torch.cuda.synchronize()
    assert all(bool((o == 7.0).all()) for o in outs)
    P.ptg_batch(ctx, descs, outs)
    torch.cuda.synchronize()
    for d, o in zip(descs, outs):
        ref = torch.empty_like(o)
        P.ptg_field(ctx, d, ref)
        torch.cuda.synchronize()
        assert torch.equal(o, ref)


@pytest.mark.parametrize("after", range(3))
def test_batch_prepare_nomem(ctx, after):
    descs = [P.make_desc(dims=2, size=(128, 64), spc=64, octaves=5, seed=k) for k in range(2)]
    outs = [torch.full((64, 128), 7.0, device="cuda") for _ in descs]
    P.ptg_debug_fail_alloc(ctx, 1, after=after)
    _nomem(lambda: P.ptg_batch_prepare(ctx, descs, outs))
    plan = P.ptg_batch_prepare(ctx, descs, outs)
    P.ptg_batch_launch(plan)
    torch.cuda.synchronize()
    P.ptg_batch_free(plan)
    assert all(bool(torch.isfinite(o).all()) for o in outs)


def test_box_counts_nomem(ctx):
    m = torch.randn((256, 256), device="cuda")
    P.ptg_debug_fail_alloc(ctx, 1)
    _nomem(lambda: P.ptg_box_counts(ctx, m, 0.0, 5))
    counts = P.ptg_box_counts(ctx, m, 0.0, 5)
    assert np.all(np.asarray(counts) > 0)


def test_autotune_nomem(ctx):
    P.ptg_debug_fail_alloc(ctx, 1)
    _nomem(lambda: P.ptg_autotune(ctx, 0, None))


def test_fail_alloc_rejects_negative(ctx):
    for n, after in ((-1, 0), (1, -1)):
        with pytest.raises(P.PtgError) as e:
            P.ptg_debug_fail_alloc(ctx, n, after=after)
        assert e.value.code == P.PTG_ERR_INVALID
