"""The 2D thread-shape autotuner: it times both shapes per octave structure,
keeps the faster, writes and reloads its cache, and the shapes it picks are
the ones the generators then use."""
import json
import os

import pytest

torch = pytest.importorskip("torch")

import paper_1610_03525_gb300 as P  # noqa: E402

pytestmark = pytest.mark.gpu

METHODS = [(1, P.PTG_C1, P.METHOD_FIELD, 0), (2, P.PTG_C2, P.METHOD_FIELD, 0),
           (3, P.PTG_PAPER_D2M1N3, P.METHOD_FIELD, 0), (4, P.PTG_ZERO_GRADIENT, P.METHOD_FIELD, 0),
           (10, P.PTG_C1, P.METHOD_PERLIN, P.PTG_PERLIN_S5), (11, P.PTG_C1, P.METHOD_PERLIN, P.PTG_PERLIN_S3)]


@pytest.fixture(scope="module")
def tuned(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03525_gb300 import build
    build.build()
    path = str(tmp_path_factory.mktemp("tune") / "shapes.json")
    ctx = P.ptg_create(0)
    P.ptg_autotune(ctx, 2, path)
    yield ctx, path
    ctx.close()


def _key_desc(smooth, variant, dtype, n16, tail, size=(320, 192)):
    return P.make_desc(dims=2, size=size, spc=1 << (n16 + 3), octaves=n16 + (3 if tail else 0),
                       smoothness=smooth, variant=variant, dtype=dtype)


def test_cache_holds_every_key(tuned):
    _, path = tuned
    table = json.load(open(path))
    assert table["version"] == 1 and table["sms"] == torch.cuda.get_device_properties(0).multi_processor_count
    keys = {(e["method"], e["dtype"], e["n16"], e["tail"]) for e in table["entries"]}
    assert len(keys) == len(table["entries"]) == 6 * 2 * (9 * 2 - 1)
    for e in table["entries"]:
        assert e["us_rw8"] > 0 and e["us_rw16"] > 0
        assert e["rw"] == (16 if e["us_rw16"] < e["us_rw8"] else 8)


def test_context_uses_the_tuned_table(tuned):
    ctx, path = tuned
    table = {(e["method"], e["dtype"], e["n16"], e["tail"]): e["rw"] for e in json.load(open(path))["entries"]}
    for code, smooth, method, variant in METHODS:
        for dtype in (P.PTG_F32, P.PTG_F16):
            for n16 in (0, 1, 4, 8):
                for tail in (0, 1):
                    if n16 == 0 and tail == 0:
                        continue
                    d = _key_desc(smooth, variant, dtype, n16, tail)
                    assert P.ptg_thread_shape(ctx, d, method) == table[(code, dtype, n16, tail)]
    # keys cap at 8 octaves of 16-wide runs; size and offset never enter
    a = P.make_desc(dims=2, size=(64, 64), spc=1 << 20, octaves=12)
    b = P.make_desc(dims=2, size=(8192, 64), spc=1 << 20, octaves=12, offset=(1 << 20, 0, 0))
    assert P.ptg_thread_shape(ctx, a) == P.ptg_thread_shape(ctx, b) == table[(1, 0, 8, 0)]


def test_reload_from_cache_and_reject_bad_files(tuned, tmp_path):
    ctx, path = tuned
    with P.ptg_create(0) as c2:
        P.ptg_autotune(c2, 1, path)  # loads, does not re-time
        for code, smooth, method, variant in METHODS:
            d = _key_desc(smooth, variant, P.PTG_F32, 3, 1)
            assert P.ptg_thread_shape(c2, d, method) == P.ptg_thread_shape(ctx, d, method)
        bad = tmp_path / "bad.json"
        bad.write_text("not a table")
        with pytest.raises(P.PtgError) as e:
            P.ptg_autotune(c2, 1, str(bad))
        assert e.value.code == P.PTG_ERR_INVALID
        # a table written for another device model is re-timed and replaced
        other = json.load(open(path))
        other["device"] = "some other GPU"
        stale = tmp_path / "stale.json"
        stale.write_text(json.dumps(other))
        P.ptg_autotune(c2, 1, str(stale))
        assert json.load(open(stale))["device"] == torch.cuda.get_device_name(0)


def test_auto_shape_is_the_forced_shape(tuned):
    ctx, _ = tuned
    for smooth, n16, tail in [(P.PTG_C1, 7, 1), (P.PTG_C2, 2, 1), (P.PTG_C1, 0, 1), (P.PTG_ZERO_GRADIENT, 5, 0)]:
        d = _key_desc(smooth, 0, P.PTG_F32, n16, tail)
        rw = P.ptg_thread_shape(ctx, d)
        auto = torch.empty((192, 320), device="cuda")
        P.ptg_field(ctx, d, auto)
        d.variant = P.PTG_SHAPE_16X2 if rw == 16 else P.PTG_SHAPE_8X4
        forced = torch.empty_like(auto)
        P.ptg_field(ctx, d, forced)
        torch.cuda.synchronize()
        assert torch.equal(auto, forced)


def test_bad_effort(tuned):
    ctx, _ = tuned
    with pytest.raises(P.PtgError):
        P.ptg_autotune(ctx, -1)
    assert os.path.exists(tuned[1])
