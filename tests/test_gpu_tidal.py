"""Tidal tensor of a binary's perturbation (Sec. 6.4.1, Eqs. 25-28, Table 1)
on the GPU, against the oracle's fit and Table 1."""
import numpy as np
import pytest

import oracle
from oracle import tidal
from paper_2006_16560_gb300 import binding as B
from paper_2006_16560_gb300 import inputs
from gpu_helpers import run_gpu
from test_oracle_tidal import _table1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return B.Context(0)


def _cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("order", [2, 3])
def test_operator_equals_table1(ctx, order):
    """Unit accelerations at one point component at a time (centre of mass
    at rest, d_c = 1) read the device's least-squares operator column by
    column; it must equal Table 1."""
    P = B.TIDAL_POINTS[order]
    nr = 3 * P
    acc = np.zeros((nr, 1 + P, 3))
    for r in range(nr):
        acc[r, 1 + r // 3, r % 3] = 1.0
    T = B.tidal_tensor(ctx, order, _cuda(acc), _cuda(np.ones(nr))).cpu().numpy()
    np.testing.assert_allclose(T.T, _table1(order), atol=1e-13)


@pytest.mark.parametrize("order", [2, 3])
def test_points_bit_exact(ctx, order):
    rng = np.random.default_rng(order)
    n = 1000
    cm = rng.normal(size=(n, 3))
    dc = rng.uniform(1e-5, 1e-2, n)
    g = B.tidal_points(ctx, order, _cuda(cm), _cuda(dc)).cpu().numpy()
    want = np.stack([tidal.measure_points(order, cm[b], dc[b]) for b in range(n)])
    assert np.array_equal(g, want)
    # host arrays take the staging path and give the same bytes
    assert np.array_equal(B.tidal_points(ctx, order, cm, dc), want)


@pytest.mark.parametrize("order", [2, 3])
def test_fit_matches_oracle_same_inputs(ctx, order):
    rng = np.random.default_rng(10 + order)
    n, P = 777, B.TIDAL_POINTS[order]
    acc = rng.normal(size=(n, 1 + P, 3))
    dc = rng.uniform(1e-4, 1e-1, n)
    g = B.tidal_tensor(ctx, order, _cuda(acc), _cuda(dc)).cpu().numpy()
    absL = np.abs(_table1(order))
    rank = np.array([1.0 if len(e) == 2 else 2.0 for e in tidal.elements(order)])
    eps = np.finfo(float).eps
    for b in range(n):
        want = tidal.fit(order, acc[b, 0], acc[b, 1:], dc[b])
        # rounding bound of the differences A(point) - A(cm) and of a
        # length-3P dot product (both sides), plus the last-bit differences
        # of the two least-squares operators (an SVD-based pseudo-inverse
        # errs by a few eps of its largest entry, zeros included)
        Ap = (np.abs(acc[b, 1:]) + np.abs(acc[b, 0])).reshape(-1)
        tol = eps * ((3 * P + 8) * (absL @ Ap) + 4 * absL.max() * Ap.sum()) / dc[b] ** rank
        assert (np.abs(g[b] - want) <= tol).all()
    assert np.array_equal(B.tidal_tensor(ctx, order, acc, dc), g)


@pytest.mark.parametrize("order", [2, 3])
def test_eval_matches_oracle(ctx, order):
    rng = np.random.default_rng(20 + order)
    nb, nq, E = 50, 600, B.TIDAL_ELEMENTS[order]
    T = rng.normal(size=(nb, E))
    acm = rng.normal(size=(nb, 3))
    owner = rng.integers(0, nb, nq).astype(np.int64)
    rel = rng.normal(size=(nq, 3)) * 1e-2
    g = B.tidal_eval(ctx, order, _cuda(owner), _cuda(T), _cuda(acm), _cuda(rel)).cpu().numpy()
    want = np.stack([tidal.evaluate(order, T[owner[q]], acm[owner[q]], rel[q:q + 1])[0]
                     for q in range(nq)])
    np.testing.assert_allclose(g, want, rtol=1e-14, atol=1e-15)
    # an owner outside [0, n_binaries) gives NaN for that query only
    owner[7] = nb
    owner[9] = -1
    g2 = B.tidal_eval(ctx, order, owner, T, acm, rel)
    assert np.isnan(g2[[7, 9]]).all()
    keep = np.ones(nq, bool)
    keep[[7, 9]] = False
    np.testing.assert_allclose(g2[keep], want[keep], rtol=1e-14, atol=1e-15)


def test_bad_arguments(ctx):
    acc = np.zeros((1, 5, 3))
    for order in (0, 1, 4):
        assert B.pt_tidal_tensor(ctx.h, order, 1, B._ptr(acc), B._ptr(np.ones(1)),
                                 B._ptr(np.zeros(16))) == B.PT_ERR_ARG
    assert B.pt_tidal_tensor(ctx.h, 2, 1, None, None, None) == B.PT_ERR_ARG
    assert "pt_tidal_tensor" in B.pt_last_error(ctx.h)
    assert B.pt_tidal_tensor(ctx.h, 2, 0, None, None, None) == B.PT_OK


def _binaries(d, nbin, seed):
    rng = np.random.default_rng(seed)
    cm = d["pos"][rng.choice(len(d["mass"]), nbin, replace=False)] + 1e-3 * rng.normal(size=(nbin, 3))
    dc = rng.uniform(2e-4, 1e-3, nbin)
    return cm, dc


@pytest.mark.parametrize("order", [2, 3])
def test_tree_pipeline_matches_oracle(ctx, order):
    """Measure points as zero-mass particles in the long-range force (FP64),
    fitted on the device, against the oracle tree's forces fitted by the
    oracle."""
    n, nbin, P = 8000, 40, B.TIDAL_POINTS[order]
    d = inputs.plummer(n, 71 + order)
    cm, dc = _binaries(d, nbin, order)
    pts = B.tidal_points(ctx, order, _cuda(cm), _cuda(dc)).cpu().numpy()
    meas = np.concatenate([cm[:, None, :], pts], axis=1).reshape(-1, 3)
    pos = np.vstack([d["pos"], meas])
    mass = np.concatenate([d["mass"], np.zeros(len(meas))])
    p = B.Params(theta=0.4, r_in=0.01, r_out=0.05, n_leaf=8, n_group=64, order=2, precision=B.PT_FP64)
    g = run_gpu(ctx, pos, mass, p, neighbours=False)
    acc_g = g["acc"][n:].reshape(nbin, 1 + P, 3)
    T_g = B.tidal_tensor(ctx, order, _cuda(acc_g), _cuda(dc)).cpu().numpy()
    a_o, _, _ = oracle.Tree(pos, mass, 8, 64).force(p.theta, p.r_in, p.r_out, order=2)
    acc_o = a_o[n:].reshape(nbin, 1 + P, 3)
    # the FP64 force parity bound (1e-10 relative, both A(point) and A(cm))
    # carried through the fit: |dT_e| <= sum_r |L_er| 2e-10 |A| / d_c^k
    rowsum = np.abs(_table1(order)).sum(axis=1)
    rank = np.array([1.0 if len(e) == 2 else 2.0 for e in tidal.elements(order)])
    for b in range(nbin):
        want = tidal.fit(order, acc_o[b, 0], acc_o[b, 1:], dc[b])
        tol = 2e-10 * np.abs(acc_o[b]).max() * rowsum / dc[b] ** rank
        assert (np.abs(T_g[b] - want) <= tol).all()


def test_tidal_force_converges_at_members(ctx):
    """At the members of a binary, the centre-of-mass force plus the fitted
    expansion approaches the long-range force measured there directly, the
    third-order fit closer than the second, both closer than the bare
    centre-of-mass force (Sec. 6.4.1)."""
    n, nbin = 6000, 30
    d = inputs.plummer(n, 81)
    cm, dc = _binaries(d, nbin, 5)
    rng = np.random.default_rng(9)
    u = rng.normal(size=(nbin, 3))
    rel = 0.8 * dc[:, None] * u / np.linalg.norm(u, axis=1)[:, None]
    members = np.concatenate([cm + rel, cm - rel])
    owner = np.concatenate([np.arange(nbin), np.arange(nbin)]).astype(np.int64)
    rel_q = np.concatenate([rel, -rel])
    p = B.Params(theta=0.3, r_in=0.02, r_out=0.1, n_leaf=8, n_group=64, order=2, precision=B.PT_FP64)
    err = {}
    for order in (2, 3):
        P = B.TIDAL_POINTS[order]
        pts = B.tidal_points(ctx, order, cm, dc)
        meas = np.concatenate([cm[:, None, :], pts], axis=1).reshape(-1, 3)
        pos = np.vstack([d["pos"], meas, members])
        mass = np.concatenate([d["mass"], np.zeros(len(meas) + len(members))])
        a = run_gpu(ctx, pos, mass, p, neighbours=False)["acc"]
        acc = a[n:n + len(meas)].reshape(nbin, 1 + P, 3)
        truth = a[n + len(meas):]
        T = B.tidal_tensor(ctx, order, acc, dc)
        est = B.tidal_eval(ctx, order, owner, T, np.ascontiguousarray(acc[:, 0]), rel_q)
        err[order] = np.linalg.norm(est - truth, axis=1)
        err[0] = np.linalg.norm(acc[owner, 0] - truth, axis=1)
    assert np.median(err[3]) < np.median(err[2]) < np.median(err[0])
