"""The 2D launch-configuration autotuner: it times every configuration per
octave structure, keeps the fastest, writes and reloads its cache, and the
configurations it picks are the ones the generators then use."""
import json
import os

import pytest

torch = pytest.importorskip("torch")

import paper_1610_03525_gb300 as P  # noqa: E402

pytestmark = pytest.mark.gpu

# (kernel method code, smoothness, generator, Perlin blend, tile-node capable)
METHODS = [(1, P.PTG_C1, P.METHOD_FIELD, 0, True), (2, P.PTG_C2, P.METHOD_FIELD, 0, False),
           (3, P.PTG_PAPER_D2M1N3, P.METHOD_FIELD, 0, True), (4, P.PTG_ZERO_GRADIENT, P.METHOD_FIELD, 0, True),
           (10, P.PTG_C1, P.METHOD_PERLIN, P.PTG_PERLIN_S5, False),
           (11, P.PTG_C1, P.METHOD_PERLIN, P.PTG_PERLIN_S3, True)]


@pytest.fixture(scope="module")
def tuned(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03525_gb300 import build
    build.build()
    path = str(tmp_path_factory.mktemp("tune") / "configs.json")
    ctx = P.ptg_create(0)
    P.ptg_autotune(ctx, 2, path)
    yield ctx, path
    ctx.close()


def structure(spc, octaves):
    """(tile octaves, 16..32-sample-cell octaves, finer octaves follow)."""
    s = spc.bit_length() - 1
    n16 = max(0, min(octaves, s - 3))
    n64 = max(0, min(octaves, s - 5))
    return n64, n16 - n64, int(octaves > n16)


def _entries(path):
    return {(e["method"], e["dtype"], e["nt"], e["mid"], e["tail"]): e for e in json.load(open(path))["entries"]}


def test_cache_holds_every_key(tuned):
    _, path = tuned
    table = json.load(open(path))
    assert table["version"] == 2 and table["sms"] == torch.cuda.get_device_properties(0).multi_processor_count
    ents = _entries(path)
    assert len(ents) == len(table["entries"])
    # with finer octaves: (0, 0..2) and (1..8, 2); without: (0..8) x (0..2) minus (0, 0)
    assert len(ents) == 6 * 2 * ((3 + 8) + (9 * 3 - 1))
    for (code, _, nt, _, _), e in ents.items():
        capable = [m for m in METHODS if m[0] == code][0][4]
        us = e["us"]
        timed = [u for u in us if u >= 0]
        assert len(timed) == (4 if nt > 0 and capable else 2)
        best = us.index(min(timed))
        assert (e["rw"], e["tile"]) == ((16 if best & 1 else 8), (1 if best & 2 else 0))


def test_context_uses_the_tuned_table(tuned):
    ctx, path = tuned
    ents = _entries(path)
    for code, smooth, method, blend, _ in METHODS:
        for dtype in (P.PTG_F32, P.PTG_F16):
            for spc, octaves in [(8, 4), (16, 2), (32, 9), (64, 1), (1024, 12), (1024, 6), (2048, 7), (1 << 14, 20),
                                 (1 << 20, 9)]:
                d = P.make_desc(dims=2, size=(320, 192), spc=spc, octaves=octaves, smoothness=smooth, variant=blend,
                                dtype=dtype)
                nt, mid, tail = structure(spc, octaves)
                e = ents[(code, dtype, min(nt, 8), mid, tail)]
                assert P.ptg_launch_config(ctx, d, method) == (e["rw"], nt if e["tile"] else 0)
    # size and offset never enter the choice
    a = P.make_desc(dims=2, size=(64, 64), spc=1 << 20, octaves=12)
    b = P.make_desc(dims=2, size=(8192, 64), spc=1 << 20, octaves=12, offset=(1 << 20, 0, 0))
    assert P.ptg_launch_config(ctx, a) == P.ptg_launch_config(ctx, b)


def test_reload_from_cache_and_reject_bad_files(tuned, tmp_path):
    ctx, path = tuned
    with P.ptg_create(0) as c2:
        P.ptg_autotune(c2, 1, path)  # loads, does not re-time
        for code, smooth, method, blend, _ in METHODS:
            for spc, octaves in [(1024, 12), (64, 3), (8, 5)]:
                d = P.make_desc(dims=2, size=(128, 128), spc=spc, octaves=octaves, smoothness=smooth,
                                variant=blend)
                assert P.ptg_launch_config(c2, d, method) == P.ptg_launch_config(ctx, d, method)
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


def test_auto_config_is_the_forced_config(tuned):
    ctx, _ = tuned
    for smooth, spc, octaves in [(P.PTG_C1, 1024, 12), (P.PTG_C2, 32, 8), (P.PTG_C1, 8, 4),
                                 (P.PTG_ZERO_GRADIENT, 4096, 7), (P.PTG_PAPER_D2M1N3, 1 << 16, 14)]:
        d = P.make_desc(dims=2, size=(320, 192), spc=spc, octaves=octaves, smoothness=smooth)
        rw, nt = P.ptg_launch_config(ctx, d)
        auto = torch.empty((192, 320), device="cuda")
        P.ptg_field(ctx, d, auto)
        d.variant = (P.PTG_SHAPE_16X2 if rw == 16 else P.PTG_SHAPE_8X4) | \
            (P.PTG_COARSE_TILE if nt else P.PTG_COARSE_RUNS)
        forced = torch.empty_like(auto)
        P.ptg_field(ctx, d, forced)
        torch.cuda.synchronize()
        assert torch.equal(auto, forced)


def test_bad_effort(tuned):
    ctx, path = tuned
    with pytest.raises(P.PtgError):
        P.ptg_autotune(ctx, -1)
    assert os.path.exists(path)
