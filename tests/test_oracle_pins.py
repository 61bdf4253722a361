"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: a formula the
paper prints (Sec. 3.1 coefficients, Eq. nconstraints counts), a textbook
closed form (1D Hermite bases, smoothstep S3 / smootherstep S5), an invariant
(interpolation at corners, continuity across faces, the edge boundary
condition of Eq. independance, the range bound) or exact rational arithmetic
on tiny inputs.  Thorimbert & Chopard, arXiv:1610.03525.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(20161012)


# --------------------------------------------------------------------------
# textbook 1D Hermite bases (value/derivative at 0 and 1), monomial coeffs
# in increasing power; independent of the oracle's numeric solve.
# --------------------------------------------------------------------------
CUBIC = {
    "v0": [1, 0, -3, 2],   # 1 - 3t^2 + 2t^3
    "d0": [0, 1, -2, 1],   # t - 2t^2 + t^3
    "d1": [0, 0, -1, 1],   # -t^2 + t^3
    "v1": [0, 0, 3, -2],   # 3t^2 - 2t^3 = S3
}
QUINTIC = {
    "v0": [1, 0, 0, -10, 15, -6],
    "d0": [0, 1, 0, -6, 8, -3],
    "d1": [0, 0, 0, -4, 7, -3],
    "v1": [0, 0, 0, 10, -15, 6],   # S5
}


def _check_basis(basis, order):
    """The textbook basis itself: values/derivatives at the end points."""
    P = np.polynomial.polynomial
    want = {"v0": (1, 0), "v1": (0, 1)}
    for name, c in basis.items():
        for k in range(order + 1):
            dc = P.polyder(c, k) if k else np.array(c, float)
            at0, at1 = P.polyval(0.0, dc), P.polyval(1.0, dc)
            if k == 0:
                exp0, exp1 = want.get(name, (0, 0))
            elif k == 1:
                exp0, exp1 = (1, 0) if name == "d0" else (0, 1) if name == "d1" else (0, 0)
            else:
                exp0, exp1 = 0, 0
            assert abs(at0 - exp0) < 1e-12 and abs(at1 - exp1) < 1e-12, (name, k)


def test_textbook_bases_are_hermite():
    _check_basis(CUBIC, 1)
    _check_basis(QUINTIC, 2)


def _poly1(c, t):
    return sum(ci * t**i for i, ci in enumerate(c))


def _corner_data(dims, w=1.0):
    return RNG.uniform(-1, 1, size=(1 << dims, dims + 1))


# --------------------------------------------------------------------------
# Eq. (nconstraints): constraint counts; Sec. 3.1: n = 3 minimal for D2M1
# --------------------------------------------------------------------------
def test_constraint_counts_match_paper():
    rows = []
    with open(os.path.join(GOLDEN, "constraint_counts.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(tuple(int(x) for x in line.split()))
    for dims, m, count in rows:
        # closed form of Eq. (nconstraints)
        formula = (2**dims) * sum(math.comb(dims + i - 1, i) for i in range(m + 1))
        assert formula == count
        # the oracle's system: rows with total derivative order <= m
        A, rc, rd = O.system(dims, O.C1 if m == 1 else O.C2)
        base = m + 1
        n_paper_rows = 0
        for s, di in zip(rc, rd):
            d = [(di // base**k) % base for k in range(dims)]
            n_paper_rows += int(s >= 0 and sum(d) <= m)
        assert n_paper_rows == count
        # the count inequality holds for the degree the build uses (n = 2m+1)
        assert count <= (2 * m + 2) ** dims
    # D2M1: degree 2 has only 9 coefficients < 12 constraints (n=3 minimal)
    assert 3**2 < 12 <= 4**2


def test_lu_inverse_residual():
    for dims, meth in [(2, O.C1), (2, O.C2), (3, O.C1), (3, O.C2), (2, O.PAPER_GAUGE)]:
        A, _, _ = O.system(dims, meth)
        X = O.invert(A)
        R = A @ X - np.eye(A.shape[0])
        assert np.abs(R).max() / (np.abs(A).max() * np.abs(X).max()) < 1e-13


# --------------------------------------------------------------------------
# Sec. 3.1 printed coefficients (golden fixture) = numeric solve with gauge
# --------------------------------------------------------------------------
def _load_paper_coefficients():
    exprs = []
    with open(os.path.join(GOLDEN, "d2m1n3_paper_coefficients.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                name, rhs = [s.strip() for s in line.split("=")]
                exprs.append((name, rhs))
    return exprs


def test_paper_gauge_reproduces_printed_coefficients():
    exprs = _load_paper_coefficients()
    assert len(exprs) == 16
    for _ in range(50):
        corner = _corner_data(2)
        w = float(RNG.uniform(0.1, 2.0))
        env = {}
        for s, (i, j) in enumerate([(0, 0), (1, 0), (0, 1), (1, 1)]):
            env["h%d%d" % (i, j)] = corner[s, 0]
            env["f%d%d" % (i, j)] = w * corner[s, 1]
            env["g%d%d" % (i, j)] = w * corner[s, 2]
        for name, rhs in exprs:
            env[name] = eval(rhs, {"__builtins__": {}}, env)
        coef = O.cell_coeffs(2, O.PAPER_GAUGE, corner, w)
        for i in range(4):
            for j in range(4):
                assert abs(coef[i + 4 * j] - env["c%d%d" % (i, j)]) < 1e-12, (i, j)


def test_tensor_c1_c2_coefficients_are_hermite_products():
    for meth, basis, n in [(O.C1, CUBIC, 3), (O.C2, QUINTIC, 5)]:
        for dims in (2, 3):
            corner = _corner_data(dims)
            w = 0.7
            coef = O.cell_coeffs(dims, meth, corner, w)
            expect = np.zeros([n + 1] * dims)
            for s in range(1 << dims):
                bits = [(s >> k) & 1 for k in range(dims)]
                vals = [np.array(basis["v%d" % b], float) for b in bits]
                term = vals[0]
                for v in vals[1:]:
                    term = np.multiply.outer(term, v)
                expect += corner[s, 0] * term
                for k in range(dims):
                    fac = [np.array(basis["d%d" % bits[m]] if m == k else basis["v%d" % bits[m]], float)
                           for m in range(dims)]
                    term = fac[0]
                    for v in fac[1:]:
                        term = np.multiply.outer(term, v)
                    expect += w * corner[s, 1 + k] * term
            # oracle index sum_k a_k (n+1)^k  <->  numpy C-order [a_{D-1}..a_0]
            got = coef.reshape([n + 1] * dims).transpose(list(range(dims))[::-1])
            assert np.abs(got - expect).max() < 1e-9 * (1 if meth == O.C1 else 10)


# --------------------------------------------------------------------------
# Zero-gradient model (Eq. zg) and its sign
# --------------------------------------------------------------------------
def _s3(x):
    return 3 * x * x - 2 * x**3


def _s5(x):
    return 6 * x**5 - 15 * x**4 + 10 * x**3


def test_zero_gradient_is_paper_gauge_with_zero_gradients_and_minus_xy():
    cells = RNG.integers(0, 2**32, size=(200, 2), dtype=np.uint64).astype(np.uint32)
    t = RNG.uniform(0, 1, size=(200, 2))
    gauge = O.octave_at(2, O.PAPER_GAUGE, 3, 2, 0.0, cells, t)
    zg = O.octave_at(2, O.ZERO_GRAD, 3, 2, 0.0, cells, t)
    assert np.abs(gauge - zg).max() < 1e-13
    # the printed "+xy" fails to interpolate h11 at the corner (1, 1)
    corner = _corner_data(2)
    h00, h10, h01, h11 = corner[:, 0]
    A = h11 + h00 - h10 - h01
    plus = h00 + (h10 - h00) + (h01 - h00) + A * (1 + 1 + 1)
    minus = h00 + (h10 - h00) + (h01 - h00) + A * (1 + 1 - 1)
    assert abs(minus - h11) < 1e-14 and abs(plus - h11) > 1e-6


def test_w0_reduces_to_smoothstep_value_noise():
    """C1 / C2 with zero gradient weight: bilinear blend by S3 / S5."""
    for meth, S in [(O.C1, _s3), (O.C2, _s5)]:
        corner = _corner_data(2)
        coef = O.cell_coeffs(2, meth, corner, 0.0)
        n = 5 if meth == O.C2 else 3
        for x, y in RNG.uniform(0, 1, size=(50, 2)):
            h = sum(coef[i + (n + 1) * j] * x**i * y**j for i in range(n + 1) for j in range(n + 1))
            h00, h10, h01, h11 = corner[:, 0]
            A = h11 + h00 - h10 - h01
            ref = h00 + S(x) * (h10 - h00) + S(y) * (h01 - h00) + A * S(x) * S(y)
            assert abs(h - ref) < 1e-12


def test_edge_slice_is_1d_hermite():
    """On the y = 0 edge the C1 cell is the 1D cubic Hermite of that edge
    (D1M1N3 of Sec. 3.4); likewise the quintic for C2."""
    for meth, basis in [(O.C1, CUBIC), (O.C2, QUINTIC)]:
        corner = _corner_data(2)
        w = 1.3
        cells = np.tile(np.array([[5, 9]], np.uint32), (40, 1))
        x = np.linspace(0, 1, 40)
        t = np.stack([x, np.zeros_like(x)], 1)
        got = O.octave_at(2, meth, 11, 1, w, cells, t)
        c = [np.zeros(4)] * 0
        # corner data from the oracle's hash at the cell's corners
        cd = []
        for s in range(4):
            cc = np.array([[5 + (s & 1), 9 + (s >> 1), (11 << 8) | 1]], np.uint32)
            hsh = O.hash_batch(2, cc)[0]
            cd.append([O.unit(v) for v in hsh])
        cd = np.array(cd)
        ref = (cd[0, 0] * _poly1(basis["v0"], x) + cd[1, 0] * _poly1(basis["v1"], x)
               + w * cd[0, 1] * _poly1(basis["d0"], x) + w * cd[1, 1] * _poly1(basis["d1"], x))
        assert np.abs(got - ref).max() < 1e-12


# --------------------------------------------------------------------------
# Interpolation at corners, continuity across faces (Eq. independance)
# --------------------------------------------------------------------------
def _grid_eval(meth, dims, cell0, t_local, seed=7, octave=3, w=0.8):
    cells = np.asarray(cell0, np.uint32)[None, :].repeat(t_local.shape[0], 0)
    return O.octave_at(dims, meth, seed, octave, w, cells, t_local)


@pytest.mark.parametrize("meth", [O.C1, O.C2, O.PAPER_GAUGE])
def test_corner_values_and_slopes(meth):
    dims = 2
    w = 0.8
    eps = 1e-6
    for s in range(4):
        b = np.array([s & 1, s >> 1], float)
        h = _grid_eval(meth, 2, [100, 200], b[None, :], w=w)[0]
        cc = np.array([[100 + (s & 1), 200 + (s >> 1), (7 << 8) | 3]], np.uint32)
        hv = [O.unit(v) for v in O.hash_batch(2, cc)[0]]
        assert abs(h - hv[0]) < 1e-13
        for k in range(dims):
            d = np.zeros(2)
            d[k] = eps if b[k] == 0 else -eps
            hp = _grid_eval(meth, 2, [100, 200], (b + d)[None, :], w=w)[0]
            slope = (hp - h) / d[k]
            assert abs(slope - w * hv[1 + k]) < 1e-5


def _one_sided(meth, dims, axis, cell_left, t_face, w, seed, octave, order):
    """Derivatives of order 1..order normal to the face between cell_left and
    its +axis neighbour, from each side, at points t_face on the face."""
    eps = 1e-3
    n = t_face.shape[0]
    right = np.array(cell_left, np.uint32)
    right[axis] += 1
    left_c = np.tile(np.array(cell_left, np.uint32), (n, 1))
    right_c = np.tile(right, (n, 1))
    out = []
    for side, cells, t0 in [("L", left_c, 1.0), ("R", right_c, 0.0)]:
        sgn = -1.0 if side == "L" else 1.0
        pts = []
        for k in range(5):
            t = t_face.copy()
            t[:, axis] = t0 + sgn * k * eps
            pts.append(O.octave_at(dims, meth, seed, octave, w, cells, t))
        p = np.array(pts)
        # one-sided 4th-order differences along sgn direction
        d1 = sgn * (-25 * p[0] + 48 * p[1] - 36 * p[2] + 16 * p[3] - 3 * p[4]) / (12 * eps)
        d2 = (35 * p[0] - 104 * p[1] + 114 * p[2] - 56 * p[3] + 11 * p[4]) / (12 * eps**2)
        out.append((p[0], d1, d2))
    return out


@pytest.mark.parametrize("dims,meth", [(2, O.C1), (2, O.C2), (3, O.C1), (3, O.C2)])
def test_continuity_across_faces(dims, meth):
    w = 0.9
    for axis in range(dims):
        t_face = RNG.uniform(0, 1, size=(20, dims))
        (hL, d1L, d2L), (hR, d1R, d2R) = _one_sided(meth, dims, axis, [40] * dims, t_face, w, 5, 2, 2)
        # edge boundary condition; the 216 x 216 D3M2N5 system has condition
        # number ~4e8, so its FP64 solve carries ~1e-11 of rounding
        assert np.abs(hL - hR).max() < (1e-10 if (dims, meth) == (3, O.C2) else 1e-12)
        assert np.abs(d1L - d1R).max() < 1e-6         # C1
        if meth == O.C2:
            assert np.abs(d2L - d2R).max() < 1e-3     # C2
        else:
            assert np.abs(d2L - d2R).max() > 1e-3     # cubic: curvature jumps


def test_paper_gauge_and_zero_gradient_are_only_c0():
    """The Sec. 3.1 solution meets the edge condition (values agree on the
    face) but its normal slope depends on the far corners: it jumps."""
    for meth in (O.PAPER_GAUGE, O.ZERO_GRAD):
        jumps = []
        for axis in range(2):
            t_face = RNG.uniform(0.1, 0.9, size=(20, 2))
            (hL, d1L, _), (hR, d1R, _) = _one_sided(meth, 2, axis, [40, 40], t_face, 0.9, 5, 2, 1)
            assert np.abs(hL - hR).max() < 1e-12
            jumps.append(np.abs(d1L - d1R).max())
        assert max(jumps) > 1e-2


# --------------------------------------------------------------------------
# Range bound: |h| <= 1 + D w beta_M, beta_1 = 1/4, beta_2 = 5/16
# --------------------------------------------------------------------------
def test_range_constants():
    t = np.linspace(0, 1, 20001)
    b1 = np.abs(_poly1(CUBIC["d0"], t)) + np.abs(_poly1(CUBIC["d1"], t))
    b2 = np.abs(_poly1(QUINTIC["d0"], t)) + np.abs(_poly1(QUINTIC["d1"], t))
    assert abs(b1.max() - 0.25) < 1e-8 and abs(b2.max() - 5 / 16) < 1e-8
    # value bases are non-negative and sum to one
    for B in (CUBIC, QUINTIC):
        v0, v1 = _poly1(B["v0"], t), _poly1(B["v1"], t)
        assert v0.min() >= -1e-15 and v1.min() >= -1e-15 and np.abs(v0 + v1 - 1).max() < 1e-14


@pytest.mark.parametrize("dims,meth,beta", [(2, O.C1, 0.25), (2, O.C2, 5 / 16), (3, O.C1, 0.25)])
def test_range_bound_on_fields(dims, meth, beta):
    w = 1.0
    size = (64, 64) if dims == 2 else (24, 24, 24)
    cells = (4, 4) if dims == 2 else (3, 3, 3)
    N = 4
    f = O.field_grid(dims, size, cells, octaves=N, method=meth, grad_weight=w, seed=1)
    atot = sum(0.5**i for i in range(N))
    assert np.abs(f).max() <= (1 + dims * w * beta) * atot + 1e-12


# --------------------------------------------------------------------------
# Coordinates: exact rationals; octave sum
# --------------------------------------------------------------------------
def test_axis_coordinates_exact():
    for spc in (1, 3, 4, 64, 1000, 1024):
        for origin in (0, 5, -7, 2**20, -(2**31) + 3):
            j = RNG.integers(0, 50000, size=64)
            for octave in (0, 1, 3, 7, 12, 31):
                cell, t = O.axis(origin, spc, j, octave)
                for jj, cc, tt in zip(j, cell, t):
                    pos = (Fraction(origin) + Fraction(int(jj), spc)) * 2**octave
                    fl = math.floor(pos)
                    assert int(cc) == fl % 2**32
                    assert tt == float(pos - fl)


def test_fraction_zero_on_sub_lattice():
    spc = 1024
    for octave in range(12):
        step = max(spc >> octave, 1)
        j = np.arange(0, 8192, step)
        _, t = O.axis(3, spc, j, octave)
        assert np.all(t == 0.0)


def test_octave_sum_matches_independent_composition():
    """fBm of Sec. 4 rebuilt from single octaves placed with exact rational
    coordinates: amplitude p^i, frequency 2^i, N octaves i = 0..N-1."""
    size, cells, N, p = (48, 40), (3, 5), 5, 0.6
    origin = (-17, 2**20 + 3)
    idx = np.stack(np.meshgrid(np.arange(size[0]), np.arange(size[1]), indexing="xy"), -1).reshape(-1, 2)
    idx = idx[RNG.choice(idx.shape[0], 300, replace=False)]
    for meth in (O.C1, O.C2, O.PERLIN_S5):
        got = O.field_samples(2, size, cells, idx, octaves=N, method=meth, persistence=p, grad_weight=0.5,
                              seed=9, origin=origin)
        pf = float(np.float32(p))
        ref = np.zeros(idx.shape[0])
        for i in range(N):
            cl = np.zeros((idx.shape[0], 2), np.uint32)
            tl = np.zeros((idx.shape[0], 2))
            for m, (jx, jy) in enumerate(idx):
                for k, jj in enumerate((jx, jy)):
                    pos = (Fraction(origin[k]) + Fraction(int(jj) * cells[k], size[k])) * 2**i
                    fl = math.floor(pos)
                    cl[m, k] = fl % 2**32
                    tl[m, k] = float(pos - fl)
            ref += pf**i * O.octave_at(2, meth, 9, i, float(np.float32(0.5)), cl, tl)
        assert np.abs(got - ref).max() < 1e-12


@pytest.mark.parametrize("f", [1.0, 1.5, 2.0, 3.0, 4.0])
def test_axis_any_frequency_matches_exact_rationals(f):
    """Sec. 4, f_i proportional to f^i: sample j of an axis sits at
    (origin + j/spc) f^i lattice units; cell = floor, t = the rest."""
    for spc in (1, 64, 1024):
        for origin in (0, -7, 2**10):
            j = RNG.integers(0, 5000, size=32)
            for octave in (0, 1, 5, 9):
                cell, t = O.axis_freq(origin, spc, j, f, octave)
                for jj, cc, tt in zip(j, cell, t):
                    pos = (Fraction(origin) + Fraction(int(jj), spc)) * Fraction(f) ** octave
                    fl = math.floor(pos)
                    assert int(cc) == fl % 2**32
                    assert tt == float(pos - fl)


def test_octave_sum_any_frequency_matches_independent_composition():
    """The same fBm rebuilt from single octaves for frequency ratios 1.5 and
    3: amplitude p^i, lattice coordinate (origin + j/spc) f^i."""
    size, cells, N, p = (48, 40), (3, 5), 6, 0.6
    origin = (-17, 2**10 + 3)
    idx = np.stack(np.meshgrid(np.arange(size[0]), np.arange(size[1]), indexing="xy"), -1).reshape(-1, 2)
    idx = idx[RNG.choice(idx.shape[0], 200, replace=False)]
    for f in (1.5, 3.0):
        for meth in (O.C1, O.PERLIN_S5, O.ZERO_GRAD):
            got = O.field_samples(2, size, cells, idx, octaves=N, method=meth, persistence=p, grad_weight=0.5,
                                  seed=9, origin=origin, frequency=f)
            pf = float(np.float32(p))
            ref = np.zeros(idx.shape[0])
            for i in range(N):
                cl = np.zeros((idx.shape[0], 2), np.uint32)
                tl = np.zeros((idx.shape[0], 2))
                for m, (jx, jy) in enumerate(idx):
                    for k, jj in enumerate((jx, jy)):
                        pos = (Fraction(origin[k]) + Fraction(int(jj) * cells[k], size[k])) * Fraction(f) ** i
                        fl = math.floor(pos)
                        cl[m, k] = fl % 2**32
                        tl[m, k] = float(pos - fl)
                ref += pf**i * O.octave_at(2, meth, 9, i, float(np.float32(0.5)), cl, tl)
            assert np.abs(got - ref).max() < 1e-12


# --------------------------------------------------------------------------
# Perlin (Sec. 3.2) and OpenSimplex-style pins
# --------------------------------------------------------------------------
@pytest.mark.parametrize("meth", [O.PERLIN_S5, O.PERLIN_S3])
def test_perlin_zero_at_lattice_points_and_gradient(meth):
    eps = 1e-6
    for s in range(4):
        b = np.array([s & 1, s >> 1], float)
        h = _grid_eval(meth, 2, [3, 4], b[None, :])[0]
        assert abs(h) < 1e-15
        cc = np.array([[3 + (s & 1), 4 + (s >> 1), (7 << 8) | 3]], np.uint32)
        hv = [O.unit(v) for v in O.hash_batch(2, cc)[0]]
        for k in range(2):
            d = np.zeros(2)
            d[k] = eps if b[k] == 0 else -eps
            hp = _grid_eval(meth, 2, [3, 4], (b + d)[None, :])[0]
            assert abs((hp - h) / d[k] - hv[1 + k]) < 1e-5


def test_perlin_edge_depends_on_edge_corners_only():
    """On y = 0: h = f00 x + S(x) (f10 (x - 1) - f00 x)  (Sec. 3.2 with y = 0)."""
    x = np.linspace(0, 1, 33)
    for meth, S in [(O.PERLIN_S5, _s5), (O.PERLIN_S3, _s3)]:
        got = _grid_eval(meth, 2, [3, 4], np.stack([x, 0 * x], 1))
        f00 = O.unit(O.hash_batch(2, np.array([[3, 4, (7 << 8) | 3]], np.uint32))[0][1])
        f10 = O.unit(O.hash_batch(2, np.array([[4, 4, (7 << 8) | 3]], np.uint32))[0][1])
        ref = f00 * x + S(x) * (f10 * (x - 1) - f00 * x)
        assert np.abs(got - ref).max() < 1e-14


@pytest.mark.parametrize("dims", [2, 3])
def test_perlin_s5_is_c2_s3_is_c1(dims):
    cell0 = [7, 8, 9][:dims]
    for meth in (O.PERLIN_S5, O.PERLIN_S3):
        for axis in range(dims):
            t_face = RNG.uniform(0, 1, size=(10, dims))
            (hL, d1L, d2L), (hR, d1R, d2R) = _one_sided(meth, dims, axis, cell0, t_face, 1.0, 2, 1, 2)
            assert np.abs(hL - hR).max() < 1e-13 and np.abs(d1L - d1R).max() < 1e-6
            if meth == O.PERLIN_S5:
                assert np.abs(d2L - d2R).max() < 1e-3


@pytest.mark.parametrize("meth", [O.PERLIN_S5, O.PERLIN_S3])
def test_perlin_3d_zero_at_lattice_points_and_gradient(meth):
    """3D Perlin: zero at the 8 corners, gradient there = hash words 1..3 of
    the corner (pcg4d of (ix, iy, iz, key))."""
    eps = 1e-6
    for s in range(8):
        b = np.array([s & 1, (s >> 1) & 1, s >> 2], float)
        h = _grid_eval(meth, 3, [3, 4, 5], b[None, :])[0]
        assert abs(h) < 1e-15
        cc = np.array([[3 + (s & 1), 4 + ((s >> 1) & 1), 5 + (s >> 2), (7 << 8) | 3]], np.uint32)
        hv = [O.unit(v) for v in O.hash_batch(3, cc)[0]]
        for k in range(3):
            d = np.zeros(3)
            d[k] = eps if b[k] == 0 else -eps
            hp = _grid_eval(meth, 3, [3, 4, 5], (b + d)[None, :])[0]
            assert abs((hp - h) / d[k] - hv[1 + k]) < 1e-5


def test_perlin_3d_face_is_2d_perlin_of_face_corners():
    """On the face z = 0 the 3D cell is the 2D Perlin polynomial of the four
    face corners with their x and y gradients (S(0) = 0, and z - 0 = 0)."""
    t2 = RNG.uniform(0, 1, size=(64, 2))
    for meth in (O.PERLIN_S5, O.PERLIN_S3):
        got = _grid_eval(meth, 3, [3, 4, 5], np.concatenate([t2, np.zeros((64, 1))], 1))
        S = _s5 if meth == O.PERLIN_S5 else _s3
        g = {}
        for a in (0, 1):
            for b in (0, 1):
                w = O.hash_batch(3, np.array([[3 + a, 4 + b, 5, (7 << 8) | 3]], np.uint32))[0]
                g[a, b] = (O.unit(w[1]), O.unit(w[2]))
        x, y = t2[:, 0], t2[:, 1]
        v = {k: g[k][0] * (x - k[0]) + g[k][1] * (y - k[1]) for k in g}
        h0 = v[0, 0] + S(x) * (v[1, 0] - v[0, 0])
        h1 = v[0, 1] + S(x) * (v[1, 1] - v[0, 1])
        assert np.abs(got - (h0 + S(y) * (h1 - h0))).max() < 1e-14


SQ = (math.sqrt(3) - 1) / 2


def test_opensimplex_zero_at_vertices_and_gradient():
    eps = 1e-6
    for a, b in [(0, 0), (3, -2), (10, 7), (-5, 12)]:
        px, py = a + (a + b) * SQ, b + (a + b) * SQ
        h = O.opensimplex_points(4, 2, np.array([[px, py]]))[0]
        assert abs(h) < 1e-12
        g = O.hash_batch(2, np.array([[a % 2**32, b % 2**32, (4 << 8) | 2]], np.uint32))[0]
        gx, gy = O.unit(g[1]), O.unit(g[2])
        hx = O.opensimplex_points(4, 2, np.array([[px + eps, py]]))[0]
        hy = O.opensimplex_points(4, 2, np.array([[px, py + eps]]))[0]
        # d/dd [(2 - r^2)^4 (g.d)] at d = 0 is 16 g; scale 1/8
        assert abs(hx / eps - 2 * gx) < 1e-4 and abs(hy / eps - 2 * gy) < 1e-4


def test_opensimplex_is_smooth():
    """The (2 - r^2)^4 kernel vanishes with three derivatives at r^2 = 2: the
    field is C1 everywhere, in particular across simplex edges."""
    pts = RNG.uniform(0, 20, size=(200, 2))
    e = 1e-4
    for dx, dy in [(1, 0), (0, 1)]:
        f = lambda s: O.opensimplex_points(1, 0, pts + s * np.array([dx, dy]))
        d_c = (f(e) - f(-e)) / (2 * e)
        d_c2 = (f(2 * e) - f(-2 * e)) / (4 * e)
        assert np.abs(d_c - d_c2).max() < 1e-5


# --------------------------------------------------------------------------
# Hash sanity (Jarzynski & Olano pcg3d / pcg4d): uniform, uncorrelated words
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dims", [2, 3])
def test_hash_statistics(dims):
    # 2^22 lattice corners (a 2048 x 2048 block): the mean of a uniform draw on
    # [-1, 1) has standard error 0.58 / 2^11 = 2.8e-4 and its variance 1.5e-4
    n = 1 << 22
    keys = np.zeros((n, dims + 1), np.uint32)
    keys[:, 0] = np.arange(n) % 2048
    keys[:, 1] = np.arange(n) // 2048
    keys[:, dims] = (5 << 8) | 3
    h = O.hash_batch(dims, keys)
    v = (h >> 9).astype(np.float32) / np.float32(4194304.0) - np.float32(1.0)
    assert np.abs(v.mean(0, dtype=np.float64)).max() < 1.5e-3
    assert np.abs(v.var(0, dtype=np.float64) - 1 / 3).max() < 1.5e-3
    c = np.corrcoef(v.T)
    assert np.abs(c - np.eye(dims + 1)).max() < 1e-2
    # neighbouring corners are uncorrelated too
    assert abs(np.corrcoef(v[:-1, 0], v[1:, 0])[0, 1]) < 1e-2
    # avalanche: flipping one input bit flips about half of the output bits
    flip = keys.copy()
    flip[:, 0] ^= 1
    diff = np.unpackbits((O.hash_batch(dims, flip) ^ h).view(np.uint8)).mean()
    assert abs(diff - 0.5) < 0.02
    # unit(): exact grid of 2^-22 in [-1, 1)
    assert O.unit(0) == -1.0 and O.unit(0xFFFFFFFF) == 1.0 - 2.0**-22


# --------------------------------------------------------------------------
# 3D OpenSimplex-style noise: squish 1/3, stretch -1/6, nearest vertices
# sqrt(2) apart, kernel (2 - r^2)^4 (g . d), scale 1/8
# --------------------------------------------------------------------------
def _vertex3(a, b, c):
    s = (a + b + c) / 3.0
    return np.array([a + s, b + s, c + s])


def test_opensimplex3_zero_at_vertices_and_gradient():
    """At a vertex only that vertex is in range (its neighbours sit at r^2 = 2
    exactly, where the kernel vanishes with three derivatives): h = 0 and
    grad h = 16 g / 8 = 2 g, g = pcg4d words 1..3."""
    eps = 1e-6
    for a, b, c in [(0, 0, 0), (3, -2, 5), (10, 7, -1), (-5, 12, 4)]:
        p = _vertex3(a, b, c)
        assert abs(O.opensimplex3_points(4, 2, p[None])[0]) < 1e-12
        w = O.hash_batch(3, np.array([[a % 2**32, b % 2**32, c % 2**32, (4 << 8) | 2]], np.uint32))[0]
        g = np.array([O.unit(w[1]), O.unit(w[2]), O.unit(w[3])])
        for k in range(3):
            e = np.zeros(3)
            e[k] = eps
            hk = O.opensimplex3_points(4, 2, (p + e)[None])[0]
            assert abs(hk / eps - 2 * g[k]) < 1e-4


def test_opensimplex3_neighbours_are_sqrt2_apart():
    """The squished lattice is face-centred cubic: the twelve stretched offsets
    +-e_k and e_i - e_j are at distance sqrt(2); the next shell is at 2."""
    base = _vertex3(0, 0, 0)
    offs = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, -1, 0), (1, 0, -1), (0, 1, -1)]
    for o in offs:
        for sgn in (1, -1):
            v = _vertex3(*(sgn * np.array(o)))
            assert abs(np.sum((v - base) ** 2) - 2.0) < 1e-12
    for o in [(1, 1, 0), (1, 1, 1), (2, 0, 0), (1, 1, -1)]:
        assert np.sum((_vertex3(*o) - base) ** 2) >= 4.0 - 1e-12


def test_opensimplex3_is_smooth():
    """The kernel vanishes with three derivatives at r^2 = 2: the field is C1,
    also across the faces of the simplices."""
    pts = RNG.uniform(-10, 10, size=(200, 3))
    e = 1e-4
    for k in range(3):
        dv = np.zeros(3)
        dv[k] = 1.0
        f = lambda s: O.opensimplex3_points(1, 0, pts + s * dv)
        d_c = (f(e) - f(-e)) / (2 * e)
        d_c2 = (f(2 * e) - f(-2 * e)) / (4 * e)
        assert np.abs(d_c - d_c2).max() < 1e-5


def test_opensimplex3_field_routes_agree():
    """The field's exact integer / fraction route to the stretched lattice
    (dyadic frequencies) equals the real-position route, octave by octave,
    at origins on both sides of zero."""
    size, cells, origin = (12, 10, 9), (3, 2, 3), (5, -3, 7)
    spc = [s // c for s, c in zip(size, cells)]
    rng = np.random.default_rng(3)
    idx = np.stack([rng.integers(0, s, 300) for s in size], 1)
    for i in range(4):
        one = O.field_samples(3, size, cells, idx, origin=origin, octaves=i + 1, method=O.OPENSIMPLEX, seed=9,
                              persistence=1.0)
        prev = O.field_samples(3, size, cells, idx, origin=origin, octaves=i, method=O.OPENSIMPLEX, seed=9,
                               persistence=1.0) if i else 0.0
        pos = np.stack([(origin[k] + idx[:, k] / spc[k]) * 2.0**i for k in range(3)], 1)
        assert np.abs((one - prev) - O.opensimplex3_points(9, i, pos)).max() < 1e-12


@pytest.mark.parametrize("dims", [2, 3])
def test_opensimplex_second_moment_closed_form(dims):
    """Closed form of E[h^2] over positions and seeds.  With gradient
    components independent and uniform on [-1, 1), E[(g . d)^2] = |d|^2 / 3 and
    distinct vertices are uncorrelated, so E[h^2] = (1/64) sum_v (2 - r_v^2)^8
    r_v^2 / 3.  Averaged over the position, the sum over the lattice becomes
    the vertex density times the integral over the disc (ball) of radius
    sqrt(2).  The squished lattice has one vertex per det(I + q J): sqrt(3) in
    2D (q = (sqrt(3) - 1)/2), 2 in 3D (q = 1/3).  Radial integrals:
    2D  2 pi int_0^sqrt2 (2 - r^2)^8 r^3 dr = pi (2^10/9 - 2^10/10);
    3D  4 pi int_0^sqrt2 (2 - r^2)^8 r^4 dr = 4 pi 2^9 sqrt(2) B(5/2, 9)
        (r = sqrt(2) s, then t = s^2).
    This ties together the kernel exponent, its radius, the scale 1/8, the
    stretch / squish constants and the gradient distribution."""
    if dims == 2:
        want = math.pi * (2.0**10 / 9 - 2.0**10 / 10) / 3 / 64 / math.sqrt(3.0)
    else:
        beta = math.gamma(2.5) * math.gamma(9.0) / math.gamma(11.5)
        want = 4 * math.pi * 2.0**9 * math.sqrt(2.0) * beta / 3 / 64 / 2
    for seed in (1, 2):
        rng = np.random.default_rng(seed)
        if dims == 2:
            h = O.opensimplex_points(seed, 0, rng.uniform(-500, 500, size=(400000, 2)))
        else:
            h = O.opensimplex3_points(seed, 0, rng.uniform(-60, 60, size=(200000, 3)))
        # about 6e5 (2D) and 9e5 (3D) vertices in the region: the estimate's
        # relative standard error is near 0.3%
        assert abs(np.mean(h * h) / want - 1.0) < 0.02
        assert abs(h.mean()) < 0.005


def test_opensimplex3_range_and_mean():
    """|h| stays below the sum of the kernel maxima of the vertices in range;
    the hashed gradients are centred, so the field is too."""
    h = O.opensimplex3_points(2, 1, RNG.uniform(-40, 40, size=(100000, 3)))
    assert abs(h.mean()) < 0.01 and 0.2 < h.std() < 0.5
    assert np.abs(h).max() < 2.0


# --------------------------------------------------------------------------
# Ridged multifractal sum (the paper's ridged mountains, Sec. 5.1): octave i
# adds p^i r_i, r_i = (1 - |h_i|)^2 w_i, w_0 = 1, w_{i+1} = clamp(2 r_i, 0, 1)
# --------------------------------------------------------------------------
def _ridged_field(method, N, p=0.5, dims=2, size=(40, 24), cells=(2, 3), origin=(3, -5), seed=7):
    return O.field_grid(dims, size, cells, origin=origin, octaves=N, method=method, persistence=p, seed=seed,
                        ridged=True)


@pytest.mark.parametrize("method", [O.C1, O.C2, O.ZERO_GRAD, O.PERLIN_S5])
def test_ridged_one_octave_is_the_squared_ridge(method):
    h = O.field_grid(2, (40, 24), (2, 3), origin=(3, -5), octaves=1, method=method, seed=7)
    assert np.abs(_ridged_field(method, 1) - (1 - np.abs(h)) ** 2).max() < 1e-15


def test_ridged_at_the_lattice_origin_uses_corner_values():
    """At sample (0, 0) every octave sits on a corner, so h_i is corner value
    v_i (hash word 0) and the sum follows from the hash alone."""
    N, p, seed = 6, 0.6, 9
    got = O.field_grid(2, (8, 8), (1, 1), origin=(0, 0), octaves=N, method=O.C1, persistence=p, seed=seed,
                       ridged=True)[0, 0]
    keys = np.array([[0, 0, (seed << 8) | i] for i in range(N)], np.uint32)
    v = [O.unit(w[0]) for w in O.hash_batch(2, keys)]
    want, weight, amp = 0.0, 1.0, 1.0
    for i in range(N):
        r = (1 - abs(v[i])) ** 2 * weight
        want += amp * r
        amp *= float(np.float32(p))  # the persistence enters as the float32 the GPU path receives
        weight = min(max(2 * r, 0.0), 1.0)
    assert abs(got - want) < 1e-15


@pytest.mark.parametrize("method", [O.C1, O.ZERO_GRAD, O.PERLIN_S3])
def test_ridged_range_and_monotone_in_octaves(method):
    """|h_i| <= 1.5 for these models, so 0 <= r_i <= 1 and 0 <= H <= A_tot;
    every octave adds a non-negative term."""
    prev = np.zeros((24, 40))
    for N in range(1, 7):
        H = _ridged_field(method, N, p=0.7)
        assert H.min() >= 0.0 and H.max() <= sum(0.7 ** i for i in range(N)) + 1e-12
        assert np.all(H >= prev - 1e-15)
        prev = H


def test_ridged_3d_and_any_frequency():
    h = O.field_grid(3, (12, 10, 8), (2, 2, 2), origin=(1, 2, 3), octaves=1, method=O.C1, seed=3, frequency=1.7)
    r = O.field_grid(3, (12, 10, 8), (2, 2, 2), origin=(1, 2, 3), octaves=1, method=O.C1, seed=3, frequency=1.7,
                     ridged=True)
    assert np.abs(r - (1 - np.abs(h)) ** 2).max() < 1e-15
