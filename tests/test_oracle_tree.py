"""Pins for the oracle's keys, sort, octree, moments, groups, walk and tree force.

Checks are against hand-derived values, brute force on tiny inputs, library
routines (numpy stable argsort, scipy kd-tree), invariants of the walk, the
paper's printed quadrupole of a binary (Sec. 6.4.2, Eqs. 36-38) and the
expected truncation order of monopole and quadrupole expansions.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2006_16560_gb300 import inputs

BITS = 21


def _bits_interleave(qx, qy, qz):
    """Brute-force Morton interleave through binary strings."""
    sx, sy, sz = (format(int(v), "021b") for v in (qx, qy, qz))
    return int("".join(a + b + c for a, b, c in zip(sx, sy, sz)), 2)


def test_keys_cube_corners():
    """The 8 unit-cube corners: q is 0 or 2^21-1 per dimension, so the key of
    corner (a, b, c) is (4a + 2b + c) * (8^21 - 1) / 7."""
    pos = np.array([[a, b, c] for a in (0, 1) for b in (0, 1) for c in (0, 1)], float)
    T = oracle.Tree(pos, np.ones(8), 1, 1)
    key, q, perm = T.keys()
    rep = (8 ** 21 - 1) // 7
    for i, (a, b, c) in enumerate(pos.astype(int)):
        assert int(key[i]) == (4 * a + 2 * b + c) * rep
    assert list(perm) == list(range(8))
    assert T.S == 1.0 and T.scale == 2.0 ** 21


def test_keys_brute_force_small():
    rng = np.random.default_rng(9)
    for n in (1, 2, 7, 64):
        pos = rng.normal(size=(n, 3)) * rng.uniform(0.1, 10)
        T = oracle.Tree(pos, np.ones(n), 4, 8)
        key, q, perm = T.keys()
        lo = pos.min(0)
        S = float((pos.max(0) - lo).max()) or 1.0
        scale = 2.0 ** 21 / S
        for i in range(n):
            qq = [min(max(math.floor((float(pos[i, d]) - float(lo[d])) * scale), 0), 2 ** 21 - 1)
                  for d in range(3)]
            assert list(q[i]) == qq
            assert int(key[i]) == _bits_interleave(*qq)


def test_sort_is_stable_argsort():
    rng = np.random.default_rng(2)
    pos = rng.integers(0, 4, size=(500, 3)).astype(float)   # many equal keys
    T = oracle.Tree(pos, np.ones(500), 8, 16)
    key, q, perm = T.keys()
    assert np.array_equal(perm, np.argsort(key, kind="stable"))


def _brute_nodes(skeys, n_leaf):
    """All (level, begin, count) nodes from the run definition, by brute force."""
    n = len(skeys)
    out = set()
    stack = [(0, 0, n)]
    while stack:
        lev, b, c = stack.pop()
        out.add((lev, b, c))
        if c <= n_leaf or lev == BITS:
            continue
        sh = 3 * (BITS - lev - 1)
        pref = [int(k) >> sh for k in skeys[b:b + c]]
        s = 0
        for i in range(1, c + 1):
            if i == c or pref[i] != pref[s]:
                stack.append((lev + 1, b + s, i - s))
                s = i
    return out


@pytest.mark.parametrize("n,n_leaf", [(1, 1), (2, 1), (64, 1), (64, 4), (200, 8), (150, 3)])
def test_topology_brute_force(n, n_leaf):
    rng = np.random.default_rng(n + n_leaf)
    pos = rng.normal(size=(n, 3)) ** 3            # clustered, uneven
    T = oracle.Tree(pos, np.ones(n), n_leaf, 4 * n_leaf)
    key, q, perm = T.keys()
    nd = T.nodes()
    got = set(zip(nd["level"].tolist(), nd["begin"].tolist(), nd["count"].tolist()))
    assert got == _brute_nodes(key[perm], n_leaf)
    # children tile their parent in key order
    for v in range(T.nnodes):
        if nd["leaf"][v]:
            assert nd["count"][v] <= n_leaf or nd["level"][v] == BITS
            continue
        fc, nc = nd["first_child"][v], nd["nchild"][v]
        b = nd["begin"][v]
        for c in range(fc, fc + nc):
            assert nd["begin"][c] == b and nd["level"][c] == nd["level"][v] + 1
            b += nd["count"][c]
        assert b == nd["begin"][v] + nd["count"][v]


def test_depth_cap_with_coincident_points():
    pos = np.zeros((40, 3))
    pos[20:] = 1.0
    T = oracle.Tree(pos, np.ones(40), 4, 8)
    nd = T.nodes()
    leaves = nd["leaf"] == 1
    assert set(nd["count"][leaves].tolist()) == {20}
    assert set(nd["level"][leaves].tolist()) == {BITS}


def test_moments_mass_com_and_traceless():
    d = inputs.plummer(2000, 3, masses="kroupa")
    T = oracle.Tree(d["pos"], d["mass"], 8, 32)
    key, q, perm = T.keys()
    nd = T.nodes()
    sp, sm = d["pos"][perm], d["mass"][perm]
    for v in range(0, T.nnodes, 7):
        b, c = nd["begin"][v], nd["count"][v]
        m, x = sm[b:b + c], sp[b:b + c]
        assert nd["mass"][v] == pytest.approx(m.sum(), rel=1e-13)
        np.testing.assert_allclose(nd["com"][v], (m[:, None] * x).sum(0) / m.sum(), rtol=1e-12, atol=1e-14)
        Q = nd["quad"][v]
        assert abs(Q[0] + Q[1] + Q[2]) <= 1e-12 * max(1e-300, np.abs(Q).max())
        assert np.all(nd["qmin"][v] == q[perm[b:b + c]].min(0))
        assert np.all(nd["qmax"][v] == q[perm[b:b + c]].max(0))


def _quad_matrix(Q):
    xx, yy, zz, xy, xz, yz = Q
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])


@pytest.mark.parametrize("e", [0.0, 0.3, 0.6, 0.95])
def test_pseudoparticle_quadrupole_eq37_38(e):
    """Sec. 6.4.2: three pseudoparticles of mass (m1+m2)/3 at Eq. 38 reproduce
    the orbit-averaged traceless moment Eq. 37, <A'> = mu a^2/4 diag(9e^2+1,
    1-6e^2, -3e^2-2).  The oracle's Q is 2 A' (Eq. 31)."""
    m1, m2, a = 0.7, 0.4, 1.3
    mu = m1 * m2 / (m1 + m2)
    s = a * math.sqrt(mu / (m1 + m2))
    pts = s * np.array([[0, math.sqrt(1 - e * e), 0],
                        [math.sqrt(3 * e * e + 0.75), -math.sqrt((1 - e * e) / 4), 0],
                        [-math.sqrt(3 * e * e + 0.75), -math.sqrt((1 - e * e) / 4), 0]])
    T = oracle.Tree(pts, np.full(3, (m1 + m2) / 3), 8, 8)
    Q = _quad_matrix(T.nodes()["quad"][0])
    want = 0.25 * mu * a * a * np.diag([9 * e * e + 1, 1 - 6 * e * e, -3 * e * e - 2])
    np.testing.assert_allclose(Q, 2 * want, atol=1e-14)


@pytest.mark.parametrize("e", [0.0, 0.5, 0.9])
def test_orbit_average_quadrupole_eq36(e):
    """Sec. 6.4.2, Eq. 36: a binary sampled uniformly in time (mean anomaly)
    has <A> = mu a^2 diag(2e^2 + 1/2, 1/2 - e^2/2, 0) about its centre of
    mass; the oracle's moment of the sampled orbit is 3<A> - tr<A> I."""
    m1, m2, a, K = 0.6, 0.25, 2.0, 4000
    M = (np.arange(K) + 0.5) * 2 * math.pi / K
    E = M.copy()
    for _ in range(60):
        E -= (E - e * np.sin(E) - M) / (1 - e * np.cos(E))
    dr = np.stack([a * (np.cos(E) - e), a * math.sqrt(1 - e * e) * np.sin(E), 0 * E], 1)
    pos = np.concatenate([-m2 / (m1 + m2) * dr, m1 / (m1 + m2) * dr])
    mass = np.concatenate([np.full(K, m1 / K), np.full(K, m2 / K)])
    T = oracle.Tree(pos, mass, 2 * K, 2 * K)
    nd = T.nodes()
    mu = m1 * m2 / (m1 + m2)
    A = mu * a * a * np.diag([2 * e * e + 0.5, 0.5 - e * e / 2, 0.0])
    # each sample pair has its centre of mass at the origin; the shift below
    # (parallel axis) only guards against rounding in the computed COM
    c = nd["com"][0]
    A_c = A - (m1 + m2) * np.outer(c, c)
    want = 3 * A_c - np.trace(A_c) * np.eye(3)
    np.testing.assert_allclose(_quad_matrix(nd["quad"][0]), want, atol=2e-6 * np.abs(want).max())


def test_groups_partition():
    d = inputs.plummer(5000, 8)
    for n_group in (1, 16, 64, 300):
        T = oracle.Tree(d["pos"], d["mass"], 8, n_group)
        g = T.groups()
        nd = T.nodes()
        assert g["begin"][0] == 0
        assert np.all(g["begin"][1:] == g["begin"][:-1] + g["count"][:-1])
        assert g["begin"][-1] + g["count"][-1] == 5000
        big = g["count"] > n_group
        # an oversized group is always a single leaf
        leaves = {(b, c) for b, c, l in zip(nd["begin"], nd["count"], nd["leaf"]) if l}
        for b, c in zip(g["begin"][big], g["count"][big]):
            assert (b, c) in leaves


@pytest.mark.parametrize("n_group,n_leaf", [(64, 16), (24, 8), (7, 4)])
def test_groups_follow_the_rule(n_group, n_leaf):
    """The group partition restated in Python from the node list: top-down, a
    node with at most n_group particles (or a leaf) is a group; a larger node's
    children in key order, each larger child recursively; the smaller
    children of a node with at most 8 n_group particles in runs of
    consecutive children cut into pieces of exactly n_group (the last piece of
    a run smaller), those of a larger node packed whole and greedily into
    groups of at most n_group; boxes are the tight boxes of the particles'
    grid cells."""
    d = inputs.plummer(6000, 9, masses="kroupa")
    T = oracle.Tree(d["pos"], d["mass"], n_leaf, n_group)
    nd = T.nodes()
    key, q, perm = T.keys()
    sq = q[perm]
    want = []

    def visit(v):
        if nd["count"][v] <= n_group or nd["leaf"][v]:
            want.append((nd["begin"][v], nd["count"][v]))
            return
        cut = nd["count"][v] <= 8 * n_group

        def close(b, c):
            if cut:
                for o in range(0, c, n_group):
                    want.append((b + o, min(n_group, c - o)))
            elif c:
                want.append((b, c))

        run_b, run_c = 0, 0
        for c in range(nd["first_child"][v], nd["first_child"][v] + nd["nchild"][v]):
            if nd["count"][c] > n_group:
                close(run_b, run_c)
                run_c = 0
                visit(c)
                continue
            if not cut and run_c and run_c + nd["count"][c] > n_group:
                close(run_b, run_c)
                run_c = 0
            if run_c == 0:
                run_b = nd["begin"][c]
            run_c += nd["count"][c]
        close(run_b, run_c)

    root = int(np.argmin(nd["level"]))
    visit(root)
    g = T.groups()
    assert sorted(want) == list(zip(g["begin"].tolist(), g["count"].tolist()))
    for b, c, mn, mx in zip(g["begin"], g["count"], g["qmin"], g["qmax"]):
        assert np.array_equal(mn, sq[b:b + c].min(0)) and np.array_equal(mx, sq[b:b + c].max(0))
    if n_group == 64:
        assert np.mean(g["count"] == 64) > 0.3


def _brute_min_dist2(A, B):
    return float(((A[:, None, :] - B[None, :, :]) ** 2).sum(2).min())


@pytest.mark.parametrize("theta", [0.0, 0.3, 0.5, 0.9])
def test_walk_coverage_and_completeness(theta):
    """Each particle is counted exactly once per group (cells + PP), every
    pair closer than r_out is in PP, and accepted cells lie >= r_out away."""
    d = inputs.plummer(1500, 6)
    r_out = 0.08
    T = oracle.Tree(d["pos"], d["mass"], 4, 24)
    key, q, perm = T.keys()
    sp = d["pos"][perm]
    nd = T.nodes()
    g = T.groups()
    nb_off, nb_idx = oracle.neighbours(sp, r_out)
    for k in range(0, T.ngroups, 3):
        cells, pp = T.walk(k, theta, r_out)
        if theta == 0.0:
            assert len(cells) == 0
        cover = np.zeros(1500, int)
        np.add.at(cover, pp, 1)
        for v in cells:
            cover[nd["begin"][v]:nd["begin"][v] + nd["count"][v]] += 1
        assert np.all(cover == 1)
        b, c = g["begin"][k], g["count"][k]
        inpp = np.zeros(1500, bool)
        inpp[pp] = True
        for s in range(b, b + c):
            assert inpp[nb_idx[nb_off[s]:nb_off[s + 1]]].all()
        for v in cells:
            assert _brute_min_dist2(sp[b:b + c], sp[nd["begin"][v]:nd["begin"][v] + nd["count"][v]]) >= r_out ** 2


@pytest.mark.parametrize("theta", [0.3, 0.6])
def test_leaves_passing_the_gap_test_hold_no_changeover_pair(theta):
    """A leaf opened although its grid box passes the r_out gap test
    (squared gap between whole-cell boxes >= floor((r_out 2^21/S)^2) + 2) was
    opened for the opening angle alone: brute force finds no pair of it and
    the group closer than r_out, so its pairs are plain Newtonian (the far PP
    segment).  Leaves failing the test are where the changeover pairs are."""
    d = inputs.plummer(3000, 8)
    r_out = 0.04
    T = oracle.Tree(d["pos"], d["mass"], 4, 24)
    key, q, perm = T.keys()
    sp = d["pos"][perm]
    nd = T.nodes()
    g = T.groups()
    thr = np.floor((r_out * T.scale) ** 2) + 2
    leaf_ids = np.flatnonzero(nd["leaf"] == 1)
    n_far = n_near_close = 0
    for k in range(0, T.ngroups, 2):
        _, pp = T.walk(k, theta, r_out)
        inpp = np.zeros(len(sp), bool)
        inpp[pp] = True
        b, c = g["begin"][k], g["count"][k]
        gmin = g["qmin"][k].astype(np.int64)
        gmax = g["qmax"][k].astype(np.int64)
        for v in leaf_ids:
            lb, lc = nd["begin"][v], nd["count"][v]
            if not inpp[lb:lb + lc].all():
                continue
            cmin = nd["qmin"][v].astype(np.int64)
            cmax = nd["qmax"][v].astype(np.int64)
            gap = np.maximum(np.maximum(cmin - (gmax + 1), gmin - (cmax + 1)), 0)
            d2 = _brute_min_dist2(sp[b:b + c], sp[lb:lb + lc])
            if float((gap * gap).sum()) >= thr:
                n_far += 1
                assert d2 >= r_out ** 2
            elif d2 < r_out ** 2:
                n_near_close += 1
    assert n_far > 0 and n_near_close > 0


def test_tree_theta0_equals_direct():
    d = inputs.plummer(2048, 1)
    acc, pot = oracle.direct_force(d["pos"], d["mass"], 0.005, 0.05)
    T = oracle.Tree(d["pos"], d["mass"], 8, 64)
    a, p, st = T.force(0.0, 0.005, 0.05, order=2)
    assert st[0] == 0
    rel = np.linalg.norm(a - acc, axis=1) / np.linalg.norm(acc, axis=1)
    assert rel.max() < 1e-12
    np.testing.assert_allclose(p, pot, rtol=1e-13)


def test_tree_error_decreases_with_theta_and_order():
    """Tree against direct summation: the p99 error of the acceleration and of
    the potential falls with the opening angle and with the expansion order."""
    d = inputs.plummer(4096, 1)
    acc, pot = oracle.direct_force(d["pos"], d["mass"], 0.005, 0.05)
    T = oracle.Tree(d["pos"], d["mass"], 8, 64)
    err, perr = {}, {}
    for th in (0.3, 0.6):
        for order in (0, 2):
            a, p, _ = T.force(th, 0.005, 0.05, order=order)
            err[th, order] = np.percentile(np.linalg.norm(a - acc, axis=1) / np.linalg.norm(acc, axis=1), 99)
            perr[th, order] = np.percentile(np.abs(p - pot) / np.abs(pot), 99)
    for e in (err, perr):
        assert e[0.3, 2] < e[0.3, 0] and e[0.6, 2] < e[0.6, 0]
        assert e[0.3, 0] < e[0.6, 0] and e[0.3, 2] < e[0.6, 2]
    assert err[0.6, 0] < 0.05
    # the potential converges faster than the force (one power of s/d more
    # relative to its own size), so its errors sit well below the force's
    assert perr[0.6, 0] < 0.01 and perr[0.3, 2] < err[0.3, 2]


def test_cell_truncation_order():
    """A far cell's monopole error falls as (s/d)^2 and the quadrupole's as
    (s/d)^3 against the exact Newtonian sum over its particles, for the
    acceleration and for the potential (the centre of mass removes the dipole
    term from both)."""
    rng = np.random.default_rng(1)
    pts = rng.uniform(-0.5, 0.5, (50, 3))
    m = rng.uniform(0.5, 1.5, 50)
    T = oracle.Tree(pts, m, 64, 64)
    direction = np.array([0.48, 0.6, 0.64])
    slopes, pslopes = {}, {}
    for order in (0, 2):
        e, ep = [], []
        ds = np.array([8.0, 16.0, 32.0, 64.0])
        for dist in ds:
            x = direction * dist
            a, phi = T.cell_pull(0, x, order)
            dd = pts - x
            r = np.linalg.norm(dd, axis=1)
            exact = (m[:, None] * dd / r[:, None] ** 3).sum(0)
            exact_phi = -(m / r).sum()
            e.append(np.linalg.norm(a - exact) / np.linalg.norm(exact))
            ep.append(abs(phi - exact_phi) / abs(exact_phi))
        slopes[order] = np.polyfit(np.log(ds), np.log(e), 1)[0]
        pslopes[order] = np.polyfit(np.log(ds), np.log(ep), 1)[0]
    assert slopes[0] == pytest.approx(-2.0, abs=0.25)
    assert slopes[2] == pytest.approx(-3.0, abs=0.25)
    assert pslopes[0] == pytest.approx(-2.0, abs=0.25)
    assert pslopes[2] == pytest.approx(-3.0, abs=0.25)


@pytest.mark.parametrize("gamma", [0.0, 0.4, math.pi / 2, 2.2])
def test_cell_potential_legendre_closed_form(gamma):
    """Two equal masses m at (0, 0, +-a) seen from distance d at polar angle
    gamma: the exact potential is -m/d sum_l (a/d)^l P_l(cos gamma) (1 + (-1)^l),
    so the monopole is -2m/d and the quadrupole adds -2 m a^2 P_2(cos gamma)/d^3
    (Legendre expansion of 1/|x - x'|).  The oracle's cell potential and
    acceleration must equal those truncations to rounding, and differ from the
    exact sum by the next (l = 4) term."""
    m, a, d = 0.7, 0.3, 5.0
    pts = np.array([[0.0, 0.0, a], [0.0, 0.0, -a]])
    T = oracle.Tree(pts, np.array([m, m]), 8, 8)
    u = np.array([math.sin(gamma), 0.0, math.cos(gamma)])
    x = d * u
    c = math.cos(gamma)
    p2 = 0.5 * (3 * c * c - 1)
    p4 = (35 * c ** 4 - 30 * c * c + 3) / 8
    _, phi0 = T.cell_pull(0, x, 0)
    a2, phi2 = T.cell_pull(0, x, 2)
    assert phi0 == pytest.approx(-2 * m / d, rel=1e-14)
    assert phi2 == pytest.approx(-2 * m / d - 2 * m * a * a * p2 / d ** 3, rel=1e-14)
    exact = -(m / np.linalg.norm(pts - x, axis=1)).sum()
    assert exact - phi2 == pytest.approx(-2 * m * a ** 4 * p4 / d ** 5, rel=0.05, abs=1e-3 * m * a ** 4 / d ** 5)
    # acceleration of the same truncation, -grad phi with phi(x) =
    # -2m/|x| - m a^2 (3 z^2 - |x|^2)/|x|^5 (written out by hand)
    r = d
    z = x[2]
    grad = 2 * m * x / r ** 3 - m * a * a * (np.array([0.0, 0.0, 6 * z]) - 2 * x) / r ** 5 \
        + 5 * m * a * a * (3 * z * z - r * r) * x / r ** 7
    np.testing.assert_allclose(a2, -grad, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("order", [0, 2])
def test_cell_acceleration_is_minus_grad_potential(order):
    """The cell's acceleration is minus the gradient of its potential
    (central differences of the oracle's own cell potential), at points from
    twice to ten times the cell's size away."""
    rng = np.random.default_rng(3)
    pts = rng.uniform(-0.5, 0.5, (40, 3))
    m = rng.uniform(0.2, 1.8, 40)
    T = oracle.Tree(pts, m, 64, 64)
    for dist in (2.0, 4.0, 10.0):
        for _ in range(3):
            u = rng.normal(size=3)
            x = dist * u / np.linalg.norm(u)
            a, _ = T.cell_pull(0, x, order)
            h = 1e-5 * dist
            g = np.zeros(3)
            for k in range(3):
                e = np.zeros(3)
                e[k] = h
                g[k] = (T.cell_pull(0, x + e, order)[1] - T.cell_pull(0, x - e, order)[1]) / (2 * h)
            np.testing.assert_allclose(a, -g, rtol=2e-8, atol=1e-9 * np.linalg.norm(a))
