"""Host-side logic without a GPU: the seeded workload generators (the
benchmark's synthetic inputs) and the lane-operation model behind the
roofline fractions."""
import numpy as np

from paper_1610_03525_gb300 import roofline as R
from paper_1610_03525_gb300 import workloads as W


def test_request_stream_is_seeded_and_shaped():
    a = W.request_stream(rate_hz=20000.0, duration_s=0.5, seed=12345)
    b = W.request_stream(rate_hz=20000.0, duration_s=0.5, seed=12345)
    assert a == b
    assert 8000 < len(a) < 12000  # Poisson, mean 10000
    t = np.array([r["t"] for r in a])
    assert np.all(np.diff(t) >= 0) and t[-1] <= 0.5
    dims = np.array([r["dims"] for r in a])
    assert abs((dims == 2).mean() - 0.8) < 0.03
    for r in a[:500]:
        assert 4 <= r["octaves"] <= 12
        sides = r["size"][:r["dims"]]
        assert all(s == sides[0] for s in sides)
        lo, hi = (128, 2048) if r["dims"] == 2 else (32, 256)
        assert lo <= sides[0] <= hi


def test_chunk_batch_is_seeded_and_shaped():
    a = W.chunk_batch(256)
    assert a == W.chunk_batch(256)
    for c in a:
        w, h = c["size"][:2]
        assert 64 <= w <= 1024 and 64 <= h <= 1024 and w % 64 == 0 and h % 64 == 0
        assert 4 <= c["octaves"] <= 12
        assert all(abs(o) <= 1 << 20 for o in c["origin"][:2])


def test_subsample_covers_rows_random_and_lattice_lines():
    idx = W.subsample((256, 128), every=64, n_random=100, seed=1, lattice_spc=64)
    assert idx.shape == (2 * 256 + 100 + 4 * 128, 2)
    assert np.all((idx >= 0) & (idx < np.array([256, 128])))
    idx3 = W.subsample((64, 32, 16), every=8, n_random=10, seed=1, lattice_spc=32)
    assert idx3.shape == (2 * 64 * 32 + 10 + 2 * 1 * 16, 3)


def test_lane_op_model_regimes():
    size = (8192, 8192)
    # each added on-lattice octave costs 13 per sample (its -3 amp offset starts
    # the rows' sums: no work a sample)
    n10 = R.lane_ops_2d("c1", size, 1024, 10)
    n11 = R.lane_ops_2d("c1", size, 1024, 11)
    n12 = R.lane_ops_2d("c1", size, 1024, 12)
    assert n10["lattice"] == 0
    assert abs((n11["lattice"] / (8192 * 8192)) - 13) < 1e-9
    assert abs(((n12["lattice"] - n11["lattice"]) / (8192 * 8192)) - 13) < 1e-9
    # Perlin's lattice octaves are zero: no work
    assert R.lane_ops_2d("perlin_s5", size, 1024, 12, 16)["lattice"] == 0
    # tile octaves replace per-thread evaluation of the coarse octaves
    runs = R.lane_ops_2d("c1", size, 1024, 12, 8, 0)["per_sample"]
    tile = R.lane_ops_2d("c1", size, 1024, 12, 8, 5)["per_sample"]
    assert tile < runs
    # more octaves never cost less
    per = [R.lane_ops_2d("c1", size, 1024, n)["per_sample"] for n in range(1, 13)]
    assert all(b >= a for a, b in zip(per, per[1:]))
    # 3D: C1 at spc 128 (three octaves of cells >= 32, evaluated at the node rows) and at
    # spc 1024 (six, summed at the tile nodes)
    assert R.lane_ops_3d("c1", (512, 512, 512), 128, 8)["per_sample"] < 69.1
    assert R.lane_ops_3d("c1", (512, 512, 512), 1024, 10)["per_sample"] < R.lane_ops_3d("c1", (512, 512, 512), 1024, 11)["per_sample"]


def test_simplex3_box_rule():
    # staged only below one lattice unit a sample and up to 4096 vertices
    assert R.simplex3_box(1.0) == 0 and R.simplex3_box(2.0) == 0
    boxes = [R.simplex3_box(2.0 ** i / 128) for i in range(7)]
    assert all(0 < b <= 4096 for b in boxes)
    assert boxes == sorted(boxes)


def test_alu_peak():
    assert abs(R.alu_peak(152, 2070.0) - 152 * 128 * 2070e6) < 1.0


def test_bound_counts_distinct_corners_by_brute_force():
    """The lower bound's corner term counts each distinct lattice corner of a
    staged octave once: compare with a brute-force set of the cell corners that
    the samples of a small field touch."""
    size, spc, N = (37, 21), 8, 5
    b = R.bound_ops("c1", size, spc, N)
    want = 0
    for i in range(min(N, 3)):  # spc 8: octaves 0..2 staged (cells 8, 4, 2 samples)
        cs = spc >> i
        pts = set()
        for y in range(size[1]):
            for x in range(size[0]):
                cx, cy = x // cs, y // cs
                pts.update({(cx, cy), (cx + 1, cy), (cx, cy + 1), (cx + 1, cy + 1)})
        want += len(pts) * R.BOUND_CORNER_2D["c1"]
    assert b["corners"] == want
    assert b["lattice"] == size[0] * size[1] * (N - 3) * 12
    # cells of 8 samples are wider than d + 1 = 4: one cubic (3 additions);
    # cells of 4 and 2 samples: one operation each
    assert b["combine"] == size[0] * size[1] * (3 + 2)
    assert R.bound_ops("perlin_s5", size, spc, N)["lattice"] == 0
