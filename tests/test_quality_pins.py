"""Pins of the oracle's map statistics (Thorimbert & Chopard, Sec. 5):
coastline box counts and their dimension (Sec. 5.3) against shapes whose
counts and dimension are known in closed form, and the height / slope
frequency distributions (Sec. 5.1) against maps whose values and slopes are
exact binary fractions."""
import math

import numpy as np

import oracle as O


def test_straight_coastline_has_dimension_one():
    for W, H in [(65, 65), (130, 97), (1025, 257)]:
        x = np.arange(W, dtype=np.float32)
        h = np.tile(x - (W // 2 + 0.5), (H, 1))  # sea to the left of a vertical line between two samples
        c = O.box_counts(h, 0.0, 7)
        for k in range(7):
            assert c[k] == math.ceil((H - 1) / 2**k)
        if (H - 1) % 64 == 0:
            assert abs(O.box_dimension(c, 0, 6) - 1.0) < 1e-12


def test_checkerboard_fills_the_plane():
    W, H = 129, 65
    y, x = np.mgrid[0:H, 0:W]
    h = np.where((x + y) % 2 == 0, 1.0, -1.0).astype(np.float32)
    c = O.box_counts(h, 0.0, 7)
    for k in range(7):
        assert c[k] == math.ceil((W - 1) / 2**k) * math.ceil((H - 1) / 2**k)
    assert abs(O.box_dimension(c, 0, 6) - 2.0) < 1e-12


def test_no_coastline_counts_nothing_and_level_is_inclusive_above():
    h = np.full((40, 50), 0.25, np.float32)
    assert not O.box_counts(h, 0.0, 5).any()
    assert not O.box_counts(h, 0.25, 5).any()      # every sample is at or above the level
    assert O.box_counts(h, 0.2500001, 5)[0] == 0   # every sample is below
    h[17, 23] = 1.0                                # one sample above a level of 0.5
    c = O.box_counts(h, 0.5, 6)
    assert c[0] == 4                               # the four unit squares around it
    assert c[5] in (1, 2, 4)


def test_diagonal_coastline():
    """The anti-diagonal x + y = 255.5 of a 257^2 map crosses 2 (256 / eps) - 1
    squares of side eps: a dimension that tends to 1 as eps shrinks."""
    W = H = 257
    y, x = np.mgrid[0:H, 0:W].astype(np.float32)
    h = (x + y - 255.5).astype(np.float32)
    c = O.box_counts(h, 0.0, 8)
    for k in range(8):
        assert c[k] == 2 * (256 >> k) - 1
    assert 1.0 < O.box_dimension(c, 0, 4) < 1.02


def test_height_histogram_of_exact_values():
    bins = 16
    y, x = np.mgrid[0:32, 0:64]
    v = ((x + 3 * y) % bins + 0.5).astype(np.float32)  # bin centres of [0, 16) with width 1
    hist = O.histogram(v, 0.0, float(bins), bins, 0)
    assert hist[0] == 0 and hist[-1] == 0
    assert hist[1:-1].sum() == v.size
    for b in range(bins):
        assert hist[1 + b] == np.count_nonzero((x + 3 * y) % bins == b)
    # below lo and at or above hi go to the end bins
    hist = O.histogram(np.array([[-0.5, 0.0, 15.99, 16.0, 1e9]], np.float32), 0.0, 16.0, 16, 0)
    assert hist[0] == 1 and hist[1] == 1 and hist[16] == 1 and hist[17] == 2


def test_slope_histogram_of_a_plane():
    """h = 0.75 x + y: central differences give (0.75, 1) exactly, so every
    interior sample has slope norm 1.25; border samples have none."""
    H, W, n = 33, 47, 3
    y, x = np.mgrid[0:H, 0:W]
    h = np.stack([(0.75 * x + y + 10.0 * f).astype(np.float32) for f in range(n)])
    hist = O.histogram(h, 0.0, 2.0, 8, 1)
    assert hist[1 + 5] == n * (W - 2) * (H - 2)
    assert hist.sum() == n * (W - 2) * (H - 2)
