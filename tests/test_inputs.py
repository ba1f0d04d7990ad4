"""Checks of the seeded input generators against the distributions they
draw from (the paper's cluster and binary models, Sec. 7.1.1)."""
import math

import numpy as np
import pytest

from paper_2006_16560_gb300 import inputs


def test_plummer_half_mass_radius_and_centre():
    d = inputs.plummer(200_000, 7)
    r = np.linalg.norm(d["pos"], axis=1)
    # Plummer half-mass radius a / sqrt(2^(2/3) - 1) = 0.7686 for a = 3 pi / 16
    assert np.median(r) == pytest.approx(inputs.PLUMMER_A / math.sqrt(2 ** (2 / 3) - 1), rel=0.01)
    assert np.abs((d["mass"][:, None] * d["pos"]).sum(0)).max() < 1e-12
    # virial equilibrium: kinetic energy 1/4 in Henon units (E = -1/4)
    ke = 0.5 * (d["mass"] * (d["vel"] ** 2).sum(1)).sum()
    assert ke == pytest.approx(0.25, rel=0.02)


def test_kroupa_imf_slopes():
    rng = inputs.rng_for(3)
    m = inputs.kroupa_masses(400_000, rng)
    assert m.min() >= 0.08 and m.max() <= 150.0
    # log-log slopes of the number density on each segment
    for lo, hi, alpha in ((0.1, 0.4, 1.3), (1.0, 20.0, 2.3)):
        edges = np.geomspace(lo, hi, 9)
        cnt, _ = np.histogram(m, edges)
        dens = cnt / np.diff(edges)
        mid = np.sqrt(edges[1:] * edges[:-1])
        slope = np.polyfit(np.log(mid), np.log(dens), 1)[0]
        assert slope == pytest.approx(-alpha, abs=0.08)


def test_kroupa95_period_distribution_eq39():
    """The sampled lg P follows Eq. 39 (Kolmogorov-Smirnov against its CDF)."""
    rng = inputs.rng_for(5)
    x = inputs.kroupa95_log_periods(200_000, rng) - 1.0
    xs = np.sort(x)
    xmax = 8.43 - 1.0
    # CDF of f(x) = 2.5 x / (45 + x^2) on [0, xmax], integrated independently by quadrature
    grid = np.linspace(0.0, xmax, 20001)
    f = 2.5 * grid / (45.0 + grid ** 2)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(grid))])
    cdf /= cdf[-1]
    emp = np.arange(1, len(xs) + 1) / len(xs)
    ks = np.abs(np.interp(xs, grid, cdf) - emp).max()
    assert ks < 5e-3
    assert xs.min() >= 0.0 and xs.max() <= xmax


def test_kroupa95_binaries_kepler_and_thermal():
    d = inputs.kroupa95_binaries(50_000, 9)
    m = d["m1_msun"] + d["m2_msun"]
    p_yr = 10.0 ** d["log_period_days"] / 365.25
    a_au = d["semi_major"] / inputs.AU_IN_NB
    np.testing.assert_allclose(a_au ** 3, m * p_yr ** 2, rtol=1e-9)      # Kepler's third law
    assert d["ecc"].mean() == pytest.approx(2.0 / 3.0, abs=0.01)          # thermal: f(e) = 2e
    sep = np.linalg.norm(d["pos"][0::2] - d["pos"][1::2], axis=1)
    assert np.all(sep <= 2.0 * d["semi_major"] * (1 + 1e-9))             # within apocentre
    assert d["mass"].sum() == pytest.approx(1.0)
    assert d["m1_msun"].max() <= 40.0


def test_binary_members_move_on_their_orbits():
    """Both binary generators give members the relative velocity of their
    Kepler orbit: the pair's pericentre is a (1 - e) and the specific energy
    is -mu / (2a)."""
    import oracle
    for gen in (inputs.kroupa95_binaries, inputs.plummer_binaries):
        d = gen(500, 4)
        i = np.arange(0, 1000, 2)
        dx = d["pos"][i + 1] - d["pos"][i]
        dv = d["vel"][i + 1] - d["vel"][i]
        mu = d["mass"][i] + d["mass"][i + 1]
        a = d["semi_major"]
        eps = 0.5 * (dv * dv).sum(1) - mu / np.linalg.norm(dx, axis=1)
        np.testing.assert_allclose(eps, -mu / (2 * a), rtol=1e-6)
        if "ecc" in d:
            rp = np.array([oracle.pericentre(dx[k], dv[k], mu[k]) for k in range(500)])
            np.testing.assert_allclose(rp, a * (1 - d["ecc"]), rtol=1e-6)
