"""The 3D OpenSimplex kernel evaluates a fixed list of candidate vertices per
sample (after reflecting the upper half of the stretched unit cube onto the
lower one).  This checks that list against an exact minimisation: with xi the
point's position in its stretched cube and u = xi - delta, the squared real
distance to the vertex at offset delta is |u|^2 + (sum u)^2 (squish 1/3), a
convex quadratic; its minimum over the half-cube sum xi <= 3/2 is found over
every set of active faces.  A vertex can be within sqrt(2) of some point iff
that minimum is below 2 (a vertex whose minimum is exactly 2, such as the
neighbour at (-1, 0, 0) seen from the cube's corner, contributes (2 - 2)^4 = 0),
and those vertices must be exactly the kernel's."""
import itertools
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_1610_03525_gb300", "csrc", "ptg_opensimplex3d.cuh")


def kernel_candidates():
    text = open(SRC).read()
    body = text[text.index("constexpr int t[kNumCand][3] = {"):]
    body = body[:body.index("};")]
    return sorted(tuple(int(v) for v in m) for m in re.findall(r"\{(-?\d+), (-?\d+), (-?\d+)\}", body))


def min_r2(d, hi):
    """Exact minimum of |x - d|^2 + (sum(x - d))^2 over 0 <= x <= 1, sum x <= hi."""
    H = 2.0 * (np.eye(3) + np.ones((3, 3)))
    A, b = [], []
    for k in range(3):
        e = np.eye(3)[k]
        A += [e, -e]
        b += [1.0, 0.0]
    A.append(np.ones(3))
    b.append(hi)
    A, b = np.array(A), np.array(b)
    best = np.inf
    for n in range(4):
        for act in itertools.combinations(range(len(b)), n):
            Aa, ba = A[list(act)], b[list(act)]
            K = np.block([[H, Aa.T], [Aa, np.zeros((n, n))]]) if n else H
            rhs = np.concatenate([H @ d, ba]) if n else H @ d
            try:
                x = np.linalg.solve(K, rhs)[:3]
            except np.linalg.LinAlgError:
                continue
            if np.all(A @ x <= b + 1e-12):
                u = x - d
                best = min(best, u @ u + u.sum() ** 2)
    return best


def test_candidate_list_is_exact():
    deltas = [np.array(d, float) for d in itertools.product(range(-3, 5), repeat=3)]
    want = sorted(tuple(int(v) for v in d) for d in deltas if min_r2(d, 1.5) < 2.0 - 1e-9)
    assert kernel_candidates() == want
    assert len(want) == 19
    # the same list holds a little past the reflection plane (rounding there is harmless)
    assert sorted(tuple(int(v) for v in d) for d in deltas if min_r2(d, 1.6) < 2.0 - 1e-9) == want


def test_reflection_covers_the_upper_half():
    """Upper half (sum xi >= 3/2): xi -> 1 - xi maps it onto the lower half and
    a vertex at offset delta onto 1 - delta, with the same distance."""
    rng = np.random.default_rng(0)
    xi = rng.random((4000, 3))
    xi = xi[xi.sum(1) > 1.5]
    cand = np.array(kernel_candidates())
    for d in itertools.product(range(-2, 4), repeat=3):
        u = xi - np.array(d)
        inr = (u * u).sum(1) + u.sum(1) ** 2 < 2.0
        if inr.any():
            assert any(np.array_equal(1 - np.array(d), c) for c in cand), d


def _min_r2_2d(d, A, b):
    """Exact minimum of |x - d|^2 + (sum(x - d))^2 over {x : A x <= b} in 2D
    (the 2D squish (sqrt(3) - 1)/2 makes 2q + 2q^2 = 1)."""
    H = 2.0 * (np.eye(2) + np.ones((2, 2)))
    best = np.inf
    for n in range(3):
        for act in itertools.combinations(range(len(b)), n):
            Aa, ba = A[list(act)], b[list(act)]
            K = np.block([[H, Aa.T], [Aa, np.zeros((n, n))]]) if n else H
            rhs = np.concatenate([H @ d, ba]) if n else H @ d
            try:
                x = np.linalg.solve(K, rhs)[:2]
            except np.linalg.LinAlgError:
                continue
            if np.all(A @ x <= b + 1e-12):
                u = x - d
                best = min(best, u @ u + u.sum() ** 2)
    return best


def test_2d_vertex_choice_is_complete():
    """The 2D kernel takes the three vertices of the point's triangle and one
    more: across the edge opposite the vertex of smallest barycentric weight.
    Over each of the six regions (two triangles x three smallest weights) every
    vertex that can come within sqrt(2) must be among those four."""
    sq = np.sqrt(3.0)
    assert abs(2 * ((sq - 1) / 2) + 2 * ((sq - 1) / 2) ** 2 - 1.0) < 1e-15
    # lower triangle xi + yi <= 1: weights (wc, wx, wy) = (1 - x - y, x, y); upper: (x + y - 1, 1 - y, 1 - x)
    tri = {
        "lower": (np.array([[-1.0, 0.0], [0.0, -1.0], [1.0, 1.0]]), np.array([0.0, 0.0, 1.0]),
                  lambda x, y: (1 - x - y, x, y), [(1, 0), (0, 1), (0, 0)],
                  {0: (1, 1), 1: (-1, 1), 2: (1, -1)}),
        "upper": (np.array([[1.0, 0.0], [0.0, 1.0], [-1.0, -1.0]]), np.array([1.0, 1.0, -1.0]),
                  lambda x, y: (x + y - 1, 1 - y, 1 - x), [(1, 0), (0, 1), (1, 1)],
                  {0: (0, 0), 1: (0, 2), 2: (2, 0)}),
    }
    # weights as affine functions w = g . (x, y) + h, to write "w_m <= w_n" as a face
    lin = {"lower": [(np.array([-1.0, -1.0]), 1.0), (np.array([1.0, 0.0]), 0.0), (np.array([0.0, 1.0]), 0.0)],
           "upper": [(np.array([1.0, 1.0]), -1.0), (np.array([0.0, -1.0]), 1.0), (np.array([-1.0, 0.0]), 1.0)]}
    for name, (A0, b0, _, verts, extra) in tri.items():
        for m in range(3):  # region where weight m is the smallest
            A, b = [*A0], [*b0]
            for n in range(3):
                if n != m:  # w_m - w_n <= 0
                    A.append(lin[name][m][0] - lin[name][n][0])
                    b.append(lin[name][n][1] - lin[name][m][1])
            A, b = np.array(A), np.array(b)
            chosen = set(verts) | {extra[m]}
            for d in itertools.product(range(-3, 5), repeat=2):
                if _min_r2_2d(np.array(d, float), A, b) < 2.0 - 1e-9:
                    assert d in chosen, (name, m, d)
