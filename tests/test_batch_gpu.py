"""Batched generation (one persistent launch over many fields) and prepared
batches replayed as CUDA graphs: bit-identical to one launch per field."""
import pytest

torch = pytest.importorskip("torch")

import paper_1610_03525_gb300 as P  # noqa: E402
from paper_1610_03525_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03525_gb300 import build
    build.build()
    c = P.ptg_create(0)
    yield c
    c.close()


def _chunks(n, seed=12345):
    descs, outs = [], []
    for k, c in enumerate(W.chunk_batch(n, seed=seed)):
        dtype = P.PTG_F16 if k % 5 == 0 else P.PTG_F32
        d = P.make_desc(dims=2, size=c["size"], spc=c["spc"], origin=c["origin"], octaves=c["octaves"],
                        smoothness=c["smoothness"], seed=c["seed"], dtype=dtype)
        descs.append(d)
        outs.append(torch.full((c["size"][1], c["size"][0]), float("nan"),
                               dtype=torch.float16 if dtype == P.PTG_F16 else torch.float32, device="cuda"))
    return descs, outs


def _singles(ctx, descs, outs):
    ref = [torch.empty_like(o) for o in outs]
    for d, r in zip(descs, ref):
        P.ptg_field(ctx, d, r)
    torch.cuda.synchronize()
    return ref


def test_batch_equals_single_launches(ctx):
    descs, outs = _chunks(96)
    # mixed in: a ragged field, an offset window, a spc-1 (all-lattice) field
    extra = [P.make_desc(dims=2, size=(100, 37), spc=8, octaves=7, seed=5, smoothness=P.PTG_C2),
             P.make_desc(dims=2, size=(128, 64), spc=1024, offset=(512, 192, 0), octaves=12, seed=6),
             P.make_desc(dims=2, size=(33, 65), spc=1, octaves=5, seed=7)]
    for d in extra:
        descs.append(d)
        outs.append(torch.full((d.size[1], d.size[0]), float("nan"), device="cuda"))
    ref = _singles(ctx, descs, outs)
    P.ptg_batch(ctx, descs, outs)
    torch.cuda.synchronize()
    for k, (o, r) in enumerate(zip(outs, ref)):
        assert torch.equal(o, r), k


@pytest.mark.parametrize("n", [128, 400, 1024])
def test_batch_tile_groups(ctx, n):
    """Batches large enough that each CTA takes 2 or 4 consecutive tiles at a
    time (on a 152-SM GB300: about 6, 20 and 52 tiles per resident CTA, so
    groups of 1, 2 and 4), and groups that span several fields: every field
    equals its own single launch bit for bit, the prepared graph too."""
    descs, outs = _chunks(n, seed=77)
    ref = _singles(ctx, descs, outs)
    P.ptg_batch(ctx, descs, outs)
    torch.cuda.synchronize()
    for k, (o, r) in enumerate(zip(outs, ref)):
        assert torch.equal(o, r), k
    for o in outs:
        o.fill_(float("nan"))
    plan = P.ptg_batch_prepare(ctx, descs, outs)
    P.ptg_batch_launch(plan)
    torch.cuda.synchronize()
    P.ptg_batch_free(plan)
    for k, (o, r) in enumerate(zip(outs, ref)):
        assert torch.equal(o, r), k


def test_batch_mixed_launch_configs(ctx):
    """Fields pinned to every 2D launch configuration in one batch: each
    equals its own single launch with the same configuration."""
    descs, outs = _chunks(48, seed=11)
    for k, d in enumerate(descs):
        d.variant = (P.PTG_SHAPE_8X4 if k % 2 else P.PTG_SHAPE_16X2) | \
            (P.PTG_COARSE_TILE if (k // 2) % 2 and d.smoothness == P.PTG_C1 else P.PTG_COARSE_RUNS)
    ref = _singles(ctx, descs, outs)
    P.ptg_batch(ctx, descs, outs)
    torch.cuda.synchronize()
    for k, (o, r) in enumerate(zip(outs, ref)):
        assert torch.equal(o, r), k


def test_prepared_batch_graph_replays(ctx):
    descs, outs = _chunks(40, seed=7)
    ref = _singles(ctx, descs, outs)
    plan = P.ptg_batch_prepare(ctx, descs, outs)
    try:
        for _ in range(2):
            for o in outs:
                o.fill_(float("nan"))
            P.ptg_batch_launch(plan)
            torch.cuda.synchronize()
            for o, r in zip(outs, ref):
                assert torch.equal(o, r)
    finally:
        P.ptg_batch_free(plan)


def test_batch_rejects_bad_field_and_writes_nothing(ctx):
    descs, outs = _chunks(4, seed=3)
    descs[2].octaves = 0
    for o in outs:
        o.fill_(3.0)
    with pytest.raises(P.PtgError) as e:
        P.ptg_batch(ctx, descs, outs)
    assert e.value.code == P.PTG_ERR_INVALID
    torch.cuda.synchronize()
    assert all(bool((o == 3.0).all()) for o in outs)
