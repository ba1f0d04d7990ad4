"""Tidal-tensor fit of the oracle -- TEST INFRASTRUCTURE ONLY.

Sec. 6.4.1 (Eqs. 25-28, Table 1): the long-range acceleration near a binary's
centre of mass is expanded to first (second-order method) or second order
(third-order method) in r' = r - r_cm:

    A'_i(r') = A_ij r'_j                 (rank-2 part, A_ij symmetric)
             + A_ijk r'_j r'_k           (rank-3 part, fully symmetric, as in
                                          Table 1 where the 1/2! of Eq. 25 is
                                          absorbed into A_ijk)

Measuring A' at the Table 1 points gives the linear system M T = A' (Eq. 28);
T is recovered with numpy's pseudo-inverse.  Element order as Eq. 26.
"""
from __future__ import annotations

import math

import numpy as np

S2 = math.sqrt(2.0)
RANK2 = ["xx", "xy", "xz", "yy", "yz", "zz"]
RANK3 = ["xxx", "xxy", "xxz", "xyy", "xyz", "xzz", "yyy", "yyz", "yzz", "zzz"]
POINTS = {
    2: np.array([[1, 0, -S2 / 2], [-1, 0, -S2 / 2], [0, 1, S2 / 2], [0, -1, S2 / 2]], float),
    3: np.array([[1, 0, -1], [0, 1, -1], [-1, 0, -1], [0, -1, -1],
                 [1, 0, 1], [0, 1, 1], [-1, 0, 1], [0, -1, 1]], float),
}
AX = "xyz"


def elements(order: int) -> list[str]:
    return RANK2 + (RANK3 if order == 3 else [])


def measure_points(order: int, r_cm, d_c):
    """Measure points r_cm + d_c * (Table 1 coordinates), shape (npts, 3)."""
    return np.asarray(r_cm, float)[None, :] + d_c * POINTS[order]


def _coef(i: int, name: str, r) -> float:
    """Coefficient of element `name` in A'_i(r) for the expansion above."""
    idx = [AX.index(c) for c in name]
    if len(idx) == 2:                               # A_ab contributes to A'_a (r_b) and A'_b (r_a)
        a, b = idx
        c = 0.0
        if i == a:
            c += r[b]
        if i == b and a != b:
            c += r[a]
        return c
    # fully symmetric A_abc: term A_ijk r_j r_k summed over all (j, k) with {i, j, k} = {a, b, c}
    c = 0.0
    for j in range(3):
        for k in range(3):
            if sorted([i, j, k]) == sorted(idx):
                c += r[j] * r[k]
    return c


def matrix(order: int, d_c: float = 1.0) -> np.ndarray:
    """M of Eq. 28: rows (point, component), columns the elements of T."""
    pts = d_c * POINTS[order]
    names = elements(order)
    M = np.zeros((3 * len(pts), len(names)))
    for p, r in enumerate(pts):
        for i in range(3):
            for e, nm in enumerate(names):
                M[3 * p + i, e] = _coef(i, nm, r)
    return M


def fit(order: int, acc_cm, acc_pts, d_c: float) -> np.ndarray:
    """T from the accelerations at the centre of mass and at the points.

    As Table 1 writes it: the generalized inverse of M at unit distance,
    applied to A', then divided by d_c for the rank-2 and by d_c^2 for the
    rank-3 elements.  (The same T as pinv(M(d_c)) A' in exact arithmetic;
    inverting M at scale d_c in floating point loses about log10(1/d_c)
    digits, because its columns then differ in size by a factor 1/d_c.)"""
    Ap = (np.asarray(acc_pts, float) - np.asarray(acc_cm, float)[None, :]).reshape(-1)
    k = np.array([len(e) - 1 for e in elements(order)], float)
    return (np.linalg.pinv(matrix(order, 1.0)) @ Ap) / d_c ** k


def evaluate(order: int, T, acc_cm, rel) -> np.ndarray:
    """A(r) = A(r_cm) + expansion at offsets rel (n, 3)."""
    rel = np.atleast_2d(np.asarray(rel, float))
    names = elements(order)
    out = np.repeat(np.asarray(acc_cm, float)[None, :], len(rel), axis=0)
    for n, r in enumerate(rel):
        for i in range(3):
            out[n, i] += sum(T[e] * _coef(i, nm, r) for e, nm in enumerate(names))
    return out
