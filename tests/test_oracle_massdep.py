"""Pins for the oracle's mass-dependent changeover radii (Sec. 6.1, Eq. 12):
r_in,i = s_i r_in, r_out,i = s_i r_out with s_i = max(1, m_i/<m>)^(1/3), and a
pair uses the larger radii (Eq. 16)."""
import numpy as np
import pytest

import oracle
from paper_2006_16560_gb300 import inputs


def test_eq12_scale_factors():
    d = inputs.plummer(5000, 31, masses="kroupa")
    s = oracle.radius_scale(d["mass"])
    q = d["mass"] / d["mass"].mean()
    light = q <= 1.0
    assert np.all(s[light] == 1.0)
    np.testing.assert_allclose(s[~light] ** 3, q[~light], rtol=1e-12)
    assert s.max() > 3.0          # a Kroupa IMF reaches well above the mean mass


def test_unit_scales_equal_scalar_radii():
    d = inputs.plummer(1500, 32, masses="kroupa")
    one = np.ones(1500)
    a0, p0 = oracle.direct_force(d["pos"], d["mass"], 0.01, 0.1)
    a1, p1 = oracle.direct_force(d["pos"], d["mass"], 0.01, 0.1, scale=one)
    assert np.array_equal(a0, a1) and np.array_equal(p0, p1)
    o0, i0 = oracle.neighbours(d["pos"], 0.1)
    o1, i1 = oracle.neighbours(d["pos"], 0.1, scale=one)
    assert np.array_equal(o0, o1) and np.array_equal(i0, i1)
    T0 = oracle.Tree(d["pos"], d["mass"], 8, 32)
    T1 = oracle.Tree(d["pos"], d["mass"], 8, 32, scale=one)
    b0, q0, _ = T0.force(0.5, 0.01, 0.1)
    b1, q1, _ = T1.force(0.5, 0.01, 0.1)
    assert np.array_equal(b0, b1) and np.array_equal(q0, q1)


def test_pair_uses_the_larger_radii():
    """Two particles with factors s1 < s2 interact as with scalar radii s2 (r_in, r_out)."""
    pos = np.array([[0.0, 0.0, 0.0], [0.13, -0.05, 0.02]])
    mass = np.array([0.4, 0.9])
    for s1, s2 in ((1.0, 1.7), (2.5, 1.2)):
        a, p = oracle.direct_force(pos, mass, 0.02, 0.2, scale=np.array([s1, s2]))
        sm = max(s1, s2)
        b, q = oracle.direct_force(pos, mass, 0.02 * sm, 0.2 * sm)
        np.testing.assert_allclose(a, b, rtol=1e-15)
        np.testing.assert_allclose(p, q, rtol=1e-15)


def test_momentum_and_gradient_with_scales():
    rng = np.random.default_rng(4)
    pos = rng.uniform(-0.6, 0.6, (14, 3))
    mass = rng.uniform(0.2, 2.0, 14)
    s = oracle.radius_scale(mass)
    acc, _ = oracle.direct_force(pos, mass, 0.1, 1.0, scale=s)
    mom = (mass[:, None] * acc).sum(0)
    assert np.abs(mom).max() < 1e-13 * np.abs(mass[:, None] * acc).sum()
    h = 1e-6
    for i in range(14):
        g = np.zeros(3)
        for dd in range(3):
            pp = pos.copy(); pp[i, dd] += h
            pm = pos.copy(); pm[i, dd] -= h
            _, php = oracle.direct_force(pp, mass, 0.1, 1.0, targets=[i], scale=s)
            _, phm = oracle.direct_force(pm, mass, 0.1, 1.0, targets=[i], scale=s)
            g[dd] = (php[0] - phm[0]) / (2 * h)
        np.testing.assert_allclose(acc[i], -g, rtol=1e-6, atol=1e-7)


def test_scaled_neighbours_symmetric_and_superset():
    d = inputs.plummer(3000, 33, masses="kroupa")
    s = oracle.radius_scale(d["mass"])
    o1, i1 = oracle.neighbours(d["pos"], 0.05, scale=s)
    o0, i0 = oracle.neighbours(d["pos"], 0.05)
    rows = np.repeat(np.arange(3000), np.diff(o1))
    fwd = set((rows * 3000 + i1).tolist())
    assert fwd == set((i1.astype(np.int64) * 3000 + rows).tolist())      # j in nb(i) <=> i in nb(j)
    rows0 = np.repeat(np.arange(3000), np.diff(o0))
    assert set((rows0 * 3000 + i0).tolist()) <= fwd                     # s >= 1 only widens
    assert len(i1) > len(i0)


@pytest.mark.parametrize("theta", [0.0, 0.4])
def test_scaled_walk_complete_and_theta0_direct(theta):
    d = inputs.plummer(2000, 34, masses="kroupa")
    s = oracle.radius_scale(d["mass"])
    T = oracle.Tree(d["pos"], d["mass"], 4, 24, scale=s)
    key, q, perm = T.keys()
    sp, ss = d["pos"][perm], s[perm]
    off, idx = oracle.neighbours(sp, 0.05, scale=ss)
    g = T.groups()
    for k in range(0, T.ngroups, 4):
        cells, pp = T.walk(k, theta, 0.05)
        inpp = np.zeros(2000, bool)
        inpp[pp] = True
        b, c = g["begin"][k], g["count"][k]
        for t in range(b, b + c):
            assert inpp[idx[off[t]:off[t + 1]]].all()
    if theta == 0.0:
        a, p, _ = T.force(0.0, 0.005, 0.05, order=2)
        ad, pd = oracle.direct_force(d["pos"], d["mass"], 0.005, 0.05, scale=s)
        np.testing.assert_allclose(a, ad, rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(p, pd, rtol=1e-12)
