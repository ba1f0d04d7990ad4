"""Pins for the oracle's changeover functions and direct long-range sum.

Everything here checks the oracle against facts the paper or mathematics fix
independently of the oracle's own formulas: the boundary values printed in
Sec. 6.1 (Eq. 19), the relations of Eq. 18 between W, K and f, force being the
negative gradient of the potential, the Newtonian limits, momentum
conservation and the closed-form Plummer potential energy.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2006_16560_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")
R_IN, R_OUT = 1.0, 10.0          # the radii of the paper's Fig. 4
LAM = (R_OUT - R_IN) / (R_OUT + R_IN)


def _poly_fit(fun, deg, lo=0.02, hi=0.98, n=41):
    """Recover the polynomial that fun equals on (0, 1) by least squares."""
    xs = np.linspace(lo, hi, n)
    ys = np.array([fun(x) for x in xs])
    return np.polynomial.Polynomial.fit(xs, ys, deg, domain=[0, 1], window=[0, 1])


def test_boundary_values_eq19():
    """Eq. 19: W(1) = 0, K(0) = 1, K(1) = 0 and K', K'', K''' vanish at 0 and 1."""
    K = _poly_fit(lambda x: oracle.changeover_K(x, LAM), 8)
    W = _poly_fit(lambda x: oracle.changeover_W(x, LAM), 8)
    funcs = {"K": K, "W": W}
    rows = [l.split() for l in open(os.path.join(GOLD, "changeover_boundary.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 9
    for name, n, x, v in rows:
        p = funcs[name].deriv(int(n)) if int(n) else funcs[name]
        assert abs(p(float(x)) - float(v)) < 1e-8, (name, n, x)
    # the piecewise values at the ends agree with the polynomial limits
    assert oracle.changeover_K(0.0, LAM) == 1.0
    assert oracle.changeover_K(1.0, LAM) == 0.0
    assert oracle.changeover_W(1.0, LAM) == 0.0


def test_W_continuous_at_zero():
    """Eq. 15: both branches give Lambda at x = 0."""
    assert oracle.changeover_W(0.0, LAM) == pytest.approx(LAM, rel=1e-15)
    assert oracle.changeover_W(1e-12, LAM) == pytest.approx(LAM, rel=1e-10)


@pytest.mark.parametrize("x", [0.05, 0.2, 0.37, 0.5, 0.71, 0.9, 0.99])
def test_eq18_relations(x):
    """Eq. 18: W = f - f(1) r/r_out and K = f - (x + r_in/(r_out - r_in)) f'.

    f' is taken by a central difference of the oracle's f, so K (Eq. 17) and
    W (Eq. 15) are checked against f (Eq. 16), three separately printed forms.
    """
    r = R_IN + x * (R_OUT - R_IN)
    f = lambda t: oracle.changeover_f(t, LAM)
    h = 1e-5
    fp = (f(x + h) - f(x - h)) / (2 * h)
    assert oracle.changeover_W(x, LAM) == pytest.approx(f(x) - f(1.0) * r / R_OUT, abs=1e-13)
    assert oracle.changeover_K(x, LAM) == pytest.approx(
        f(x) - (x + R_IN / (R_OUT - R_IN)) * fp, abs=1e-9)


def test_f_at_one():
    """f(1) = 1 + Lambda (14 - 28 + 20 - 5) = 1 + Lambda."""
    assert oracle.changeover_f(1.0, LAM) == pytest.approx(1.0 + LAM, rel=1e-15)


def _pair(r, r_in, r_out, m=0.7):
    pos = np.array([[0.0, 0.0, 0.0], [r * 0.6, r * 0.0, r * 0.8]])
    mass = np.array([0.3, m])
    acc, pot = oracle.direct_force(pos, mass, r_in, r_out, G=1.0)
    return pos, mass, acc, pot


def test_newtonian_outside_r_out():
    """r >= r_out: (1 - K) = (1 - W) = 1, the textbook Newtonian pair."""
    for r in (R_OUT, 1.5 * R_OUT, 40.0):
        pos, mass, acc, pot = _pair(r, R_IN, R_OUT)
        d = pos[1] - pos[0]
        np.testing.assert_allclose(acc[0], mass[1] * d / r ** 3, rtol=1e-14)
        assert pot[0] == pytest.approx(-mass[1] / r, rel=1e-14)


def test_inside_r_in():
    """r <= r_in: no force and the constant potential -2 m / (r_out + r_in),
    which is the x -> 0 value of -m (1 - W)/r with W = Lambda (1 - 2x)."""
    for r in (0.0, 1e-9, 0.3 * R_IN, R_IN):
        pos, mass, acc, pot = _pair(r, R_IN, R_OUT)
        assert np.all(acc[0] == 0.0)
        assert pot[0] == pytest.approx(-2 * mass[1] / (R_OUT + R_IN), rel=1e-14)
    r = 0.5 * R_IN
    x = (r - R_IN) / (R_OUT - R_IN)
    direct = -0.7 * (1 - oracle.changeover_W(x, LAM)) / r
    assert direct == pytest.approx(-2 * 0.7 / (R_OUT + R_IN), rel=1e-13)


def test_force_is_minus_gradient_of_potential():
    """a_i = -grad_i phi_i for the long-range pair (K = W - r dW/dr)."""
    rng = np.random.default_rng(5)
    r_in, r_out = 0.1, 1.0
    pos = rng.uniform(-0.7, 0.7, (12, 3))
    mass = rng.uniform(0.5, 1.5, 12)
    acc, _ = oracle.direct_force(pos, mass, r_in, r_out)
    h = 1e-6
    for i in range(12):
        g = np.zeros(3)
        for d in range(3):
            pp = pos.copy(); pp[i, d] += h
            pm = pos.copy(); pm[i, d] -= h
            _, php = oracle.direct_force(pp, mass, r_in, r_out, targets=[i])
            _, phm = oracle.direct_force(pm, mass, r_in, r_out, targets=[i])
            g[d] = (php[0] - phm[0]) / (2 * h)
        np.testing.assert_allclose(acc[i], -g, rtol=1e-6, atol=1e-7)


def test_split_identity_sums_to_newton():
    """Long-range (1 - K, 1 - W) plus short-range (K, W) parts give Newton."""
    rng = np.random.default_rng(3)
    pos = rng.normal(size=(64, 3))
    mass = rng.uniform(0.1, 1.0, 64)
    aL, pL = oracle.direct_force(pos, mass, 0.2, 1.5)
    aS, pS = oracle.direct_force(pos, mass, 0.2, 1.5, shortrange=True)
    d = pos[None, :, :] - pos[:, None, :]
    r = np.linalg.norm(d, axis=2)
    np.fill_diagonal(r, np.inf)
    aN = (mass[None, :, None] * d / r[:, :, None] ** 3).sum(1)
    pN = -(mass[None, :] / r).sum(1)
    np.testing.assert_allclose(aL + aS, aN, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(pL + pS, pN, rtol=1e-12)


def test_newton_limit_and_momentum():
    """r_in < r_out -> 0 reduces to plain Newton; sum m a = 0."""
    d = inputs.plummer(512, 11, masses="kroupa")
    acc, pot = oracle.direct_force(d["pos"], d["mass"], 1e-14, 1e-13)
    dd = d["pos"][None, :, :] - d["pos"][:, None, :]
    r = np.linalg.norm(dd, axis=2)
    np.fill_diagonal(r, np.inf)
    aN = (d["mass"][None, :, None] * dd / r[:, :, None] ** 3).sum(1)
    np.testing.assert_allclose(acc, aN, rtol=1e-10, atol=1e-10)
    mom = (d["mass"][:, None] * acc).sum(0)
    assert np.abs(mom).max() < 1e-13 * np.abs(d["mass"][:, None] * acc).sum()
    acc, pot = oracle.direct_force(d["pos"], d["mass"], 0.005, 0.05)
    mom = (d["mass"][:, None] * acc).sum(0)
    assert np.abs(mom).max() < 1e-13 * np.abs(d["mass"][:, None] * acc).sum()


def test_plummer_potential_energy():
    """Plummer W = -3 pi G M^2 / (32 a) = -1/2 in Henon units (a = 3 pi/16);
    with N = 4096 the sampled value is within a few percent."""
    d = inputs.plummer(4096, 1)
    _, pot = oracle.direct_force(d["pos"], d["mass"], 1e-14, 1e-13)
    pe = 0.5 * float((d["mass"] * pot).sum())
    assert pe == pytest.approx(-3 * math.pi / (32 * inputs.PLUMMER_A), rel=0.03)
    assert pe == pytest.approx(-0.5, rel=0.03)


def test_neighbours_match_kdtree():
    """Brute-force neighbour sets equal scipy's kd-tree pair query."""
    from scipy.spatial import cKDTree
    d = inputs.plummer(3000, 4)
    r_out = 0.05
    off, idx = oracle.neighbours(d["pos"], r_out)
    pairs = cKDTree(d["pos"]).query_pairs(r_out, output_type="ndarray")
    want = [set() for _ in range(3000)]
    for a, b in pairs:
        want[a].add(b)
        want[b].add(a)
    for i in range(3000):
        got = idx[off[i]:off[i + 1]]
        assert list(got) == sorted(want[i])
