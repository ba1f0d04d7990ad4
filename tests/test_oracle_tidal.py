"""Pins for the oracle's tidal-tensor fit (Sec. 6.4.1, Eqs. 25-28, Table 1)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import tidal
from paper_2006_16560_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "tidal_table1.txt")


def _table1(order):
    rows = {}
    for line in open(GOLD):
        if not line.strip() or line.startswith("#"):
            continue
        parts = line.split()
        if int(parts[0]) != order:
            continue
        npts = len(tidal.POINTS[order])
        row = np.zeros(3 * npts)
        for term in parts[2:]:
            c, comp, pt = term.split(":")
            neg = c.startswith("-")
            c = c.lstrip("-")
            if c.startswith("s2"):
                val = math.sqrt(2.0) / float(Fraction(c.split("/")[1]))
            else:
                val = float(Fraction(c))
            row[3 * (int(pt) - 1) + "xyz".index(comp)] = -val if neg else val
        rows[parts[1][2:]] = row
    return np.array([rows[e] for e in tidal.elements(order)])


@pytest.mark.parametrize("order", [2, 3])
def test_pinv_equals_table1(order):
    """The pseudo-inverse of M at d_c = 1 reproduces Table 1's coefficients."""
    np.testing.assert_allclose(np.linalg.pinv(tidal.matrix(order)), _table1(order), atol=1e-12)


def test_condition_numbers():
    """Sec. 6.4.1 quotes condition numbers 2 and 12.7 for the two methods;
    they are the squared ratios of the largest to the smallest singular value."""
    for order, want in ((2, 2.0), (3, 12.7)):
        s = np.linalg.svd(tidal.matrix(order), compute_uv=False)
        assert (s[0] / s[-1]) ** 2 == pytest.approx(want, abs=0.05)


@pytest.mark.parametrize("order", [2, 3])
def test_exact_for_polynomial_fields(order):
    """A field that is exactly of the method's order is recovered exactly."""
    rng = np.random.default_rng(order)
    T = rng.normal(size=len(tidal.elements(order)))
    a0 = rng.normal(size=3)
    dc = 0.37
    pts = tidal.POINTS[order] * dc
    acc = tidal.evaluate(order, T, a0, pts)
    np.testing.assert_allclose(tidal.fit(order, a0, acc, dc), T, rtol=1e-12, atol=1e-12)


def test_tree_field_truncation_order():
    """Fitted to oracle long-range accelerations of zero-mass measure points,
    the second-order expansion errs O(d^2) and the third-order one O(d^3)
    at a probe point.  The long-range field is smooth on scales below r_in
    (the changeover removes the near field), so r_in >> d_c here."""
    d = inputs.plummer(3000, 61)
    cm = np.array([0.31, -0.22, 0.15])
    probe = np.array([0.4, -0.3, 0.5])
    errs = {2: [], 3: []}
    dcs = [0.08, 0.04, 0.02]
    for order in (2, 3):
        for dc in dcs:
            pts = np.vstack([cm, tidal.measure_points(order, cm, dc), cm + dc * probe])
            pos = np.vstack([d["pos"], pts])
            mass = np.concatenate([d["mass"], np.zeros(len(pts))])
            tg = np.arange(3000, 3000 + len(pts))
            acc, _ = oracle.direct_force(pos, mass, 0.5, 1.0, targets=tg)
            T = tidal.fit(order, acc[0], acc[1:-1], dc)
            est = tidal.evaluate(order, T, acc[0], [dc * probe])[0]
            errs[order].append(np.linalg.norm(est - acc[-1]))
    for order in (2, 3):
        slope = np.polyfit(np.log(dcs), np.log(errs[order]), 1)[0]
        assert slope == pytest.approx(order, abs=0.35)
    assert errs[3][-1] < errs[2][-1]
