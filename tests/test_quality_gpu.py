"""Map statistics on the GPU (Sec. 5): coastline box counts and height /
slope-norm histograms, bit-exact against the oracle on generated maps, plus
the paper's qualitative findings on the fractal dimension (Sec. 5.3)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
import paper_1610_03525_gb300 as P  # noqa: E402

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


def gen(ctx, size, octaves, smoothness=P.PTG_C1, persistence=0.5, seed=0, spc=256, perlin=False):
    d = P.make_desc(dims=2, size=size, spc=spc, octaves=octaves, smoothness=smoothness, persistence=persistence,
                    seed=seed)
    out = torch.empty((size[1], size[0]), dtype=torch.float32, device="cuda")
    (P.ptg_perlin if perlin else P.ptg_field)(ctx, d, out)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("size,levels,level", [((1024, 1024), 11, 0.0), ((1000, 777), 10, 0.1), ((2, 2), 1, 0.0),
                                               ((3, 517), 10, -0.2)])
def test_box_counts_bit_exact(ctx, size, levels, level):
    m = gen(ctx, size, 8, seed=3)
    got = P.ptg_box_counts(ctx, m, level, levels)
    want = O.box_counts(m.cpu().numpy(), level, levels)
    assert np.array_equal(got, want)


def test_box_counts_constant_and_repeat(ctx):
    m = torch.full((300, 200), 0.5, device="cuda")
    assert not P.ptg_box_counts(ctx, m, 0.0, 8).any()
    m2 = gen(ctx, (512, 512), 6, seed=1)
    a = P.ptg_box_counts(ctx, m2, 0.0, 9)
    b = P.ptg_box_counts(ctx, m2, 0.0, 9)  # the pyramid buffers are reused
    assert np.array_equal(a, b)


@pytest.mark.parametrize("what,lo,hi,bins", [(0, -2.0, 2.0, 64), (1, 0.0, 0.05, 100), (0, -0.5, 0.5, 7)])
def test_histograms_bit_exact(ctx, what, lo, hi, bins):
    maps = torch.stack([gen(ctx, (128, 96), 7, seed=s, spc=64) for s in range(12)])
    got = P.ptg_histogram(ctx, maps, lo, hi, bins, what)
    torch.cuda.synchronize()
    want = O.histogram(maps.cpu().numpy(), lo, hi, bins, what)
    assert np.array_equal(got.cpu().numpy().astype(np.uint64), want)


def test_dimension_grows_with_octaves_and_persistence(ctx):
    """Sec. 5.3: D rises with the number of octaves N and approaches 2 as the
    persistence p grows (low octaves dominate less); the zero-gradient model,
    Perlin and C1 give similar dimensions."""
    def D(N, p, **kw):
        vals = []
        for seed in range(3):
            m = gen(ctx, (1024, 1024), N, persistence=p, seed=seed, spc=256, **kw)
            vals.append(P.box_dimension(P.ptg_box_counts(ctx, m, 0.0, 7), 1, 6))
        return float(np.mean(vals))
    d2, d8 = D(2, 0.5), D(8, 0.5)
    assert 1.0 < d2 < d8 < 2.0
    assert D(8, 0.3) < d8 < D(8, 0.7)
    dz = D(8, 0.5, smoothness=P.PTG_ZERO_GRADIENT)
    dp = D(8, 0.5, perlin=True)
    assert abs(dz - d8) < 0.15 and abs(dp - d8) < 0.15


def test_bad_arguments(ctx):
    m = torch.zeros((4, 4), device="cuda")
    with pytest.raises(P.PtgError):
        P.ptg_box_counts(ctx, m, 0.0, 0)
    with pytest.raises(P.PtgError):
        P.ptg_histogram(ctx, m, 1.0, 1.0, 8)
    with pytest.raises(P.PtgError):
        P.ptg_histogram(ctx, m, 0.0, 1.0, 5000)
