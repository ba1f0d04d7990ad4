"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bars (the hot path's contract):
  * keys, sort order, tree topology, grid boxes, groups, interaction lists
    and neighbour lists: bit-exact;
  * float64 GPU forces vs the oracle's tree with the same lists: <= 1e-10
    relative per particle (acc) and per particle (pot);
  * mixed precision vs the float64 GPU path: p99 relative force error
    <= 1e-6 (and max <= 1e-4, a loose guard on the tail).
"""
import numpy as np
import pytest

import oracle
from paper_2006_16560_gb300 import binding as B
from paper_2006_16560_gb300 import inputs
from gpu_helpers import node_ids, rel_err, run_gpu

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_P99 = 1e-6
MIXED_MAX = 1e-4


@pytest.fixture(scope="module")
def ctx():
    return B.Context(0)


def c1_params(**kw):
    """Plummer N = 4096 workload: monopole, theta 0.5, leaf 8, r_out 0.05, r_in 0.1 r_out."""
    p = B.Params(theta=0.5, r_in=0.005, r_out=0.05, n_leaf=8, n_group=64, order=0,
                 precision=B.PT_FP64)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def check_structure(g, T, p):
    """Keys, order, topology, moments, groups and lists against the oracle tree."""
    tree = g["tree"]
    key, q, perm = T.keys()
    gk, gperm = tree.keys()
    assert np.array_equal(gperm.astype(np.int64), perm)
    assert np.array_equal(gk, key[perm])
    gn, on = tree.nodes(), T.nodes()
    gid = list(zip(gn["level"].tolist(), gn["begin"].tolist(), gn["count"].tolist()))
    oid = list(zip(on["level"].tolist(), on["begin"].tolist(), on["count"].tolist()))
    assert sorted(gid) == sorted(oid)
    omap = {(l, b): k for k, (l, b, c) in enumerate(oid)}
    order = np.array([omap[(l, b)] for (l, b, c) in gid])
    assert np.array_equal(gn["leaf"], on["leaf"][order])
    assert np.array_equal(gn["qmin"], on["qmin"][order])
    assert np.array_equal(gn["qmax"], on["qmax"][order])
    np.testing.assert_allclose(gn["mass"], on["mass"][order], rtol=1e-12, atol=0)
    scale = np.abs(on["com"]).max()
    np.testing.assert_allclose(gn["com"], on["com"][order], rtol=0, atol=1e-13 * scale)
    # Q = 3T - tr(T) I, with T of size M * extent^2: float64 rounding of that
    # size is more than 1e-9 |Q| for a nearly isotropic node (|Q| << |T|)
    qscale = np.abs(on["quad"][order]).max(axis=1, keepdims=True) + 1e-300
    cell = tree.info()[1][3] / 2.0**21
    ext2 = (((on["qmax"] - on["qmin"] + 1) * cell) ** 2).sum(axis=1)
    tscale = (on["mass"] * ext2)[order][:, None]
    assert np.all(np.abs(gn["quad"] - on["quad"][order]) <= 1e-9 * qscale + 1e-13 * tscale)
    gg, og = tree.groups(), T.groups()
    for k in ("begin", "count", "qmin", "qmax"):
        assert np.array_equal(gg[k], og[k]), k
    st = g["stats"]
    co, cells, po, pp = tree.lists(st["cell_list_total"], st["pp_list_total"])
    for k in range(len(og["begin"])):
        ocells, opp = T.walk(k, p.theta, p.r_out)
        assert node_ids(gn, cells[co[k]:co[k + 1]]) == node_ids(on, ocells)
        assert np.array_equal(np.sort(pp[po[k]:po[k + 1]]), np.sort(opp))


def check_neighbours(g, pos, r_out, targets=None):
    off, idx = oracle.neighbours(pos, r_out, targets)
    if targets is None:
        assert np.array_equal(g["nb_off"], off)
        assert np.array_equal(g["nb_idx"], idx)
    else:
        for t, i in enumerate(targets):
            got = g["nb_idx"][g["nb_off"][i]:g["nb_off"][i + 1]]
            assert np.array_equal(got, idx[off[t]:off[t + 1]])


@pytest.mark.parametrize("order", [0, 2])
def test_plummer4096_fp64_vs_oracle(ctx, order):
    d = inputs.plummer(4096, 1)
    p = c1_params(order=order)
    g = run_gpu(ctx, d["pos"], d["mass"], p)
    T = oracle.Tree(d["pos"], d["mass"], p.n_leaf, p.n_group)
    check_structure(g, T, p)
    a, phi, st = T.force(p.theta, p.r_in, p.r_out, order=order)
    assert rel_err(g["acc"], a).max() <= FP64_TOL
    assert (np.abs(g["pot"] - phi) / np.abs(phi)).max() <= FP64_TOL
    assert g["stats"]["cell_interactions"] == st[0]
    assert g["stats"]["pp_interactions"] == st[1]
    check_neighbours(g, d["pos"], p.r_out)
    # energy and momentum sums are float64 sums of the returned arrays
    e = 0.5 * (d["mass"] * g["pot"]).sum()
    assert g["stats"]["energy"] == pytest.approx(e, rel=1e-12)
    np.testing.assert_allclose(g["stats"]["momentum"], (d["mass"][:, None] * g["acc"]).sum(0),
                               atol=1e-12 * np.abs(d["mass"][:, None] * g["acc"]).sum())
    # and the tree is close to the direct sum (report-level bound only)
    ad, _ = oracle.direct_force(d["pos"], d["mass"], p.r_in, p.r_out)
    assert np.percentile(rel_err(g["acc"], ad), 99) < 0.05


@pytest.mark.parametrize("n_group", [8, 16, 24, 40, 96, 200])
def test_mixed_every_pass_configuration(ctx, n_group):
    """Group sizes that select each pass configuration of the mixed kernel
    (24 to 96 slots, and several passes for groups above 96 targets), taken in
    the kernel's class order: every target is evaluated once, within the
    mixed bound of the FP64 path, and the energy sums agree."""
    d = inputs.plummer(6000, 300 + n_group, masses="kroupa")
    kw = dict(order=2, n_leaf=8, n_group=n_group)
    g64 = run_gpu(ctx, d["pos"], d["mass"], c1_params(**kw))
    gmx = run_gpu(ctx, d["pos"], d["mass"], c1_params(precision=B.PT_MIXED, **kw))
    sizes = gmx["tree"].groups()["count"]
    assert sizes.sum() == len(d["mass"]) and sizes.max() > min(n_group, 96) // 2
    if n_group > 96:
        assert (sizes > 96).any()          # several passes per group
    e = rel_err(gmx["acc"], g64["acc"])
    assert np.percentile(e, 99) <= MIXED_P99
    assert e.max() <= MIXED_MAX
    ep = np.abs(gmx["pot"] - g64["pot"]) / np.abs(g64["pot"])
    assert np.percentile(ep, 99) <= MIXED_P99
    for k in ("cell_interactions", "pp_interactions"):
        assert gmx["stats"][k] == g64["stats"][k]
    assert gmx["stats"]["energy"] == pytest.approx(g64["stats"]["energy"], rel=1e-6)
    assert np.array_equal(gmx["nb_idx"], g64["nb_idx"])


@pytest.mark.parametrize("order", [0, 2])
def test_plummer4096_mixed(ctx, order):
    d = inputs.plummer(4096, 1)
    g64 = run_gpu(ctx, d["pos"], d["mass"], c1_params(order=order))
    gmx = run_gpu(ctx, d["pos"], d["mass"], c1_params(order=order, precision=B.PT_MIXED))
    e = rel_err(gmx["acc"], g64["acc"])
    assert np.percentile(e, 99) <= MIXED_P99
    assert e.max() <= MIXED_MAX
    ep = np.abs(gmx["pot"] - g64["pot"]) / np.abs(g64["pot"])
    assert np.percentile(ep, 99) <= MIXED_P99
    # the neighbour lists do not depend on the pair precision
    assert np.array_equal(gmx["nb_off"], g64["nb_off"])
    assert np.array_equal(gmx["nb_idx"], g64["nb_idx"])


def test_mixed_companions_across_the_changeover(ctx):
    """Heavy companions at separations spread over r_in..r_out (x from 0 to
    1, many just above r_in where K -> 1): the pull m (1 - K)/r^2 must keep
    its relative accuracy on the mixed path, where subtracting K from 1
    would not."""
    n_pairs = 3000
    d = inputs.plummer(n_pairs, 17)
    rng = np.random.default_rng(17)
    p = c1_params(order=2, precision=B.PT_FP64)
    x = np.concatenate([rng.uniform(0.0, 0.05, n_pairs // 2), rng.uniform(0.0, 1.0, n_pairs - n_pairs // 2)])
    r = p.r_in + x * (p.r_out - p.r_in)
    u = rng.normal(size=(n_pairs, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    pos = np.empty((2 * n_pairs, 3))
    pos[0::2] = d["pos"]
    pos[1::2] = d["pos"] + r[:, None] * u
    mass = np.repeat(d["mass"], 2) * 0.5
    mass[1::2] *= 50.0                              # companions 50x heavier than their partners
    mass /= mass.sum()
    g64 = run_gpu(ctx, pos, mass, p)
    gmx = run_gpu(ctx, pos, mass, c1_params(order=2, precision=B.PT_MIXED))
    e = rel_err(gmx["acc"], g64["acc"])
    assert np.percentile(e, 99) <= MIXED_P99
    assert e.max() <= MIXED_MAX


@pytest.mark.parametrize("spacing", [0.9999, 1.0001, 1.5])
def test_lattice_at_the_r_out_boundary(ctx, spacing):
    """A jittered cubic lattice whose spacing is just inside, just outside or
    well outside r_out: the walk puts every leaf that may hold a pair within
    r_out in a group's near PP segment and evaluates the rest without the
    changeover test, so the neighbour sets must equal brute force and both
    precisions must agree with the oracle tree."""
    r_out = 0.05
    k = 14
    g1 = (np.arange(k) - k / 2) * spacing * r_out
    pos = np.stack(np.meshgrid(g1, g1, g1, indexing="ij"), -1).reshape(-1, 3)
    pos = pos + np.random.default_rng(3).normal(scale=1e-7, size=pos.shape)
    mass = np.full(len(pos), 1.0 / len(pos))
    T = oracle.Tree(pos, mass, 8, 64)
    a, phi, _ = T.force(0.5, 0.1 * r_out, r_out, order=2)
    for prec in (B.PT_FP64, B.PT_MIXED):
        g = run_gpu(ctx, pos, mass, c1_params(order=2, precision=prec, r_out=r_out, r_in=0.1 * r_out))
        check_neighbours(g, pos, r_out)
        # the lattice's pulls cancel near its centre: errors relative to the
        # median force
        e = np.linalg.norm(g["acc"] - a, axis=1) / np.median(np.linalg.norm(a, axis=1))
        if prec == B.PT_FP64:
            assert e.max() <= FP64_TOL
        else:
            assert np.percentile(e, 99) <= MIXED_P99 and e.max() <= MIXED_MAX


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
@pytest.mark.parametrize("n_group,n_leaf,k_sites", [(64, 4, 15), (96, 4, 23), (24, 8, 2)])
def test_wide_sparse_groups_neighbours_exact(ctx, seed, n_group, n_leaf, k_sites):
    """Two walk groups each ~2e4 r_out wide (r_out = 0.0016, the serving
    radii's scale) whose members pair up across the face between them at
    r_out (1 -+ 1e-4).  The mixed kernel votes near / far on float32 offsets
    from the group's first particle, whose rounding here reaches ~1e-3 of
    r_out: a fixed 2^-10 margin calls about one true neighbour in ten far.
    The per-group bound must send every such pair to the exact float64 test,
    so the neighbour sets equal brute force in both precisions; the float64
    forces match the oracle tree."""
    r_out = 0.0016
    pos = inputs.wide_sparse_groups(r_out, k_sites, n_leaf - 1, seed)
    mass = np.full(len(pos), 1.0 / len(pos))
    p = c1_params(order=2, n_leaf=n_leaf, n_group=n_group, r_out=r_out, r_in=0.1 * r_out, theta=0.5)
    T = oracle.Tree(pos, mass, n_leaf, n_group)
    assert T.ngroups == 2
    a, phi, _ = T.force(p.theta, p.r_in, p.r_out, order=2)
    off, _ = oracle.neighbours(pos, r_out)
    assert off[-1] == 2 * (k_sites - k_sites // 4)
    for prec in (B.PT_FP64, B.PT_MIXED):
        p.precision = prec
        g = run_gpu(ctx, pos, mass, p)
        check_neighbours(g, pos, r_out)
        if prec == B.PT_FP64:
            assert rel_err(g["acc"], a).max() <= FP64_TOL
            np.testing.assert_allclose(g["pot"], phi, rtol=FP64_TOL)


def test_theta0_equals_direct(ctx):
    d = inputs.plummer(1500, 5, masses="kroupa")
    p = c1_params(theta=0.0, order=2)
    g = run_gpu(ctx, d["pos"], d["mass"], p)
    ad, pd = oracle.direct_force(d["pos"], d["mass"], p.r_in, p.r_out)
    assert g["stats"]["cell_list_total"] == 0
    assert rel_err(g["acc"], ad).max() <= 1e-12
    np.testing.assert_allclose(g["pot"], pd, rtol=1e-12)


@pytest.mark.parametrize("n", [1, 2, 3, 31, 33, 64, 65, 100, 257, 1000])
@pytest.mark.parametrize("precision", [B.PT_FP64, B.PT_MIXED])
def test_small_and_ragged(ctx, n, precision):
    d = inputs.plummer(n, 100 + n, masses="kroupa")
    p = c1_params(order=2, n_leaf=4, n_group=16, precision=precision, r_out=0.3, r_in=0.03)
    g = run_gpu(ctx, d["pos"], d["mass"], p)
    T = oracle.Tree(d["pos"], d["mass"], p.n_leaf, p.n_group)
    a, phi, _ = T.force(p.theta, p.r_in, p.r_out, order=2)
    tol = FP64_TOL if precision == B.PT_FP64 else 1e-5
    if n > 1:
        assert rel_err(g["acc"], a).max() <= tol
    np.testing.assert_allclose(g["pot"], phi, rtol=tol, atol=tol * (np.abs(phi).max() + 1.0))
    check_neighbours(g, d["pos"], p.r_out)


@pytest.mark.parametrize("ncoinc", [64, 130])
def test_depth_capped_leaf_larger_than_a_warp_scan_field(ctx, ncoinc):
    """More than 63 coincident particles make a depth-capped leaf whose count
    does not fit the walk's packed 11-bit scan fields (the walk then scans
    the counts one by one); the lists and neighbour sets must still be exact
    and the forces match the oracle tree."""
    d = inputs.plummer(3000, 21, masses="kroupa")
    pos = d["pos"].copy()
    pos[:ncoinc] = pos[0]
    p = c1_params(order=2)
    T = oracle.Tree(pos, d["mass"], p.n_leaf, p.n_group)
    a, phi, _ = T.force(p.theta, p.r_in, p.r_out, order=2)
    for prec in (B.PT_FP64, B.PT_MIXED):
        g = run_gpu(ctx, pos, d["mass"], c1_params(order=2, precision=prec))
        check_neighbours(g, pos, p.r_out)
        e = np.linalg.norm(g["acc"] - a, axis=1) / np.median(np.linalg.norm(a, axis=1))
        if prec == B.PT_FP64:
            assert e.max() <= FP64_TOL
        else:
            assert np.percentile(e, 99) <= MIXED_P99 and e.max() <= MIXED_MAX
    st = g["stats"]
    co, cells, po, pp = g["tree"].lists(st["cell_list_total"], st["pp_list_total"])
    gn, on = g["tree"].nodes(), T.nodes()
    for k in range(T.ngroups):
        ocells, opp = T.walk(k, p.theta, p.r_out)
        assert node_ids(gn, cells[co[k]:co[k + 1]]) == node_ids(on, ocells)
        assert np.array_equal(np.sort(pp[po[k]:po[k + 1]]), np.sort(opp))


def test_degenerate_inputs(ctx):
    # all particles at one point: box side 0 -> 1, one depth-capped leaf
    pos = np.zeros((50, 3))
    mass = np.full(50, 0.02)
    p = c1_params(order=2)
    g = run_gpu(ctx, pos, mass, p)
    assert np.all(g["acc"] == 0.0)
    np.testing.assert_allclose(g["pot"], -49 * 0.02 * 2 / (p.r_out + p.r_in), rtol=1e-12)
    assert np.all(np.diff(g["nb_off"]) == 49)
    # pairs of coincident points and zero masses in a Plummer set
    d = inputs.plummer(2000, 9)
    pos = d["pos"].copy()
    pos[1::2] = pos[0::2]
    mass = d["mass"].copy()
    mass[::7] = 0.0
    for prec in (B.PT_FP64, B.PT_MIXED):
        g = run_gpu(ctx, pos, mass, c1_params(order=2, precision=prec))
        T = oracle.Tree(pos, mass, 8, 64)
        a, phi, _ = T.force(0.5, 0.005, 0.05, order=2)
        tol = FP64_TOL if prec == B.PT_FP64 else 1e-4
        assert np.all(np.isfinite(g["acc"])) and np.all(np.isfinite(g["pot"]))
        assert np.percentile(rel_err(g["acc"], a), 99) <= tol
        check_neighbours(g, pos, 0.05)


def test_host_buffers_match_device_buffers(ctx):
    d = inputs.plummer(3000, 2, masses="kroupa")
    p = c1_params(order=2, precision=B.PT_MIXED)
    gd = run_gpu(ctx, d["pos"], d["mass"], p, device_buffers=True)
    gh = run_gpu(ctx, d["pos"], d["mass"], p, device_buffers=False)
    assert np.array_equal(gd["acc"], gh["acc"])
    assert np.array_equal(gd["pot"], gh["pot"])
    assert np.array_equal(gd["nb_idx"], gh["nb_idx"])


def test_errors(ctx):
    d = inputs.plummer(100, 3)
    pos, mass = d["pos"], d["mass"]
    bad = c1_params(r_in=0.05, r_out=0.05)
    rc, _ = B.pt_tree_build(ctx.h, 100, pos.ctypes.data, mass.ctypes.data, bad.c())
    assert rc == B.PT_ERR_ARG
    rc, _ = B.pt_tree_build(ctx.h, 0, pos.ctypes.data, mass.ctypes.data, c1_params().c())
    assert rc == B.PT_ERR_ARG
    p2 = pos.copy()
    p2[7, 1] = np.nan
    rc, h = B.pt_tree_build(ctx.h, 100, p2.ctypes.data, mass.ctypes.data, c1_params().c())
    assert rc == B.PT_ERR_ARG and "non-finite" in B.pt_last_error(ctx.h)
    B.pt_tree_free(h)
    m2 = mass.copy()
    m2[3] = -1.0
    rc, h = B.pt_tree_build(ctx.h, 100, pos.ctypes.data, m2.ctypes.data, c1_params().c())
    assert rc == B.PT_ERR_ARG
    B.pt_tree_free(h)
    # neighbour capacity too small: acc/pot still valid, total reported
    d = inputs.plummer(2000, 4)
    t = B.Tree(ctx, d["pos"], d["mass"], c1_params(r_out=0.2, r_in=0.02))
    acc, pot = np.zeros((2000, 3)), np.zeros(2000)
    off, idx = np.zeros(2001, dtype=np.int64), np.zeros(10, dtype=np.int32)
    total, st, rc = t.force(acc, pot, off, idx, 10, allow_capacity_error=True)
    assert rc == B.PT_ERR_CAPACITY
    want_off, _ = oracle.neighbours(d["pos"], 0.2)
    assert total == want_off[-1]
    T = oracle.Tree(d["pos"], d["mass"], 8, 64)
    a, _, _ = T.force(0.5, 0.02, 0.2, order=0)
    assert rel_err(acc, a).max() <= FP64_TOL


def test_tree_outlives_its_context():
    """A tree still alive when its context is destroyed keeps an empty handle:
    using it is an argument error, freeing it touches nothing of the destroyed
    context, and rebuilding it in a new context works."""
    d = inputs.plummer(500, 6)
    c1 = B.Context(0)
    rc, h = B.pt_tree_build(c1.h, 500, d["pos"].ctypes.data, d["mass"].ctypes.data, c1_params().c())
    assert rc == B.PT_OK
    c1.close()                                   # destroys the context first
    c2 = B.Context(0)
    acc, pot = np.zeros((500, 3)), np.zeros(500)
    rc, _, _ = B.pt_longrange_force(c2.h, h, acc.ctypes.data, pot.ctypes.data, None, None, 0)
    assert rc == B.PT_ERR_ARG
    rc, h2 = B.pt_tree_build(c2.h, 500, d["pos"].ctypes.data, d["mass"].ctypes.data, c1_params().c(), h)
    assert rc == B.PT_OK and h2.value == h.value
    rc, _, _ = B.pt_longrange_force(c2.h, h, acc.ctypes.data, pot.ctypes.data, None, None, 0)
    assert rc == B.PT_OK
    T = oracle.Tree(d["pos"], d["mass"], 8, 64)
    a, _, _ = T.force(0.5, 0.005, 0.05, order=0)
    assert rel_err(acc, a).max() <= FP64_TOL
    c2.close()
    assert B.pt_tree_free(h) == B.PT_OK            # after its second context is gone too


def test_rebuild_with_a_much_larger_set(ctx):
    """A tree first built over 1,000 particles and then rebuilt in place over
    600,000 needs 600 times its node capacity: the rebuild sizes it for the
    new set, and the result equals a fresh tree's (keys, forces, neighbours)."""
    small = inputs.plummer(1000, 8, masses="kroupa")
    big = inputs.plummer(600_000, 9, masses="kroupa")
    p = B.Params(theta=0.4, r_in=0.0004, r_out=0.004, n_leaf=16, n_group=64, order=2,
                 precision=B.PT_MIXED)
    t = B.Tree(ctx, small["pos"], small["mass"], p)
    n = len(big["mass"])
    t.rebuild(big["pos"], big["mass"], p)
    a1, p1 = np.zeros((n, 3)), np.zeros(n)
    off1, idx1 = np.zeros(n + 1, dtype=np.int64), np.zeros(8 * n, dtype=np.int32)
    tot1, _, _ = t.force(a1, p1, off1, idx1, 8 * n)
    k1, _ = t.keys()
    t.free()
    g = run_gpu(ctx, big["pos"], big["mass"], p, device_buffers=False)
    k2, _ = g["tree"].keys()
    assert np.array_equal(k1, k2)
    assert np.array_equal(a1, g["acc"]) and np.array_equal(p1, g["pot"])
    assert np.array_equal(off1, g["nb_off"]) and np.array_equal(idx1[:tot1], g["nb_idx"])


@pytest.mark.parametrize("precision", [B.PT_FP64, B.PT_MIXED])
def test_one_pass_walk_matches_two_pass(ctx, precision):
    """A tree's first force call walks in two passes (count, scan, fill); later
    calls walk once into arrays sized from the previous walk.  Same lists in
    the same order, so bit-identical forces, potentials and neighbours; a
    rebuild over many more particles exhausts the arrays and falls back."""
    import torch
    d = inputs.plummer(20000, 23, masses="kroupa")
    p = c1_params(order=2, precision=precision)
    p.r_out, p.r_in = 0.01, 0.001
    pos, mass = torch.from_numpy(d["pos"]).cuda(), torch.from_numpy(d["mass"]).cuda()
    t = B.Tree(ctx, pos, mass, p)
    outs, lists = [], []
    for _ in range(3):
        acc = torch.empty((20000, 3), dtype=torch.float64, device="cuda")
        pot = torch.empty(20000, dtype=torch.float64, device="cuda")
        off = torch.empty(20001, dtype=torch.int64, device="cuda")
        idx = torch.empty(400000, dtype=torch.int32, device="cuda")
        total, st, _ = t.force(acc, pot, off, idx, 400000)
        outs.append((acc.cpu().numpy(), pot.cpu().numpy(), off.cpu().numpy(), idx[:total].cpu().numpy(),
                     st.as_dict()))
        lists.append(t.lists(st.cell_list_total, st.pp_list_total))
        t.rebuild(pos, mass, p)
    for o, l in zip(outs[1:], lists[1:]):
        for a, b in zip(o[:4], outs[0][:4]):
            assert np.array_equal(a, b)
        for a, b in zip(l, lists[0]):
            assert np.array_equal(a, b)
        for k in ("cell_interactions", "pp_interactions", "cell_list_total", "pp_list_total", "neighbours"):
            assert o[4][k] == outs[0][4][k]
        assert o[4]["launches_force"] < outs[0][4]["launches_force"]   # one pass, no count/scan
    # stale size estimate: theta = 0 puts every particle in every group's PP
    # list (8e6 entries against arrays sized for theta = 0.5) -> fall back
    p0 = c1_params(order=2, precision=precision, theta=0.0)
    p0.r_out, p0.r_in = 0.01, 0.001
    t.rebuild(pos, mass, p0)
    acc = torch.empty((20000, 3), dtype=torch.float64, device="cuda")
    pot = torch.empty(20000, dtype=torch.float64, device="cuda")
    _, st, _ = t.force(acc, pot)
    ref = run_gpu(ctx, d["pos"], d["mass"], p0, neighbours=False)
    assert st.pp_list_total == ref["stats"]["pp_list_total"]
    assert st.launches_force == ref["stats"]["launches_force"]      # the two-pass sequence ran
    assert np.array_equal(acc.cpu().numpy(), ref["acc"])
    assert np.array_equal(pot.cpu().numpy(), ref["pot"])


def test_fp32_probe(ctx):
    """The measured float32 FMA rate is in the GB300's range (about 80 TFLOP/s
    at the 2.07 GHz maximum clock: 152 SMs x 128 lanes x 2 flops)."""
    rc, tf = B.pt_probe_fp32_peak(ctx.h)
    assert rc == B.PT_OK
    assert 30.0 < tf < 90.0
    assert B.pt_probe_fp32_peak(None)[0] == B.PT_ERR_ARG


def test_build_graph_replay_sees_new_data(ctx):
    """Rebuilding a tree from the same device buffers replays a captured build
    graph from the third build on; it must read the buffers' current contents
    (the positions drift between steps, as in a simulation)."""
    import torch
    n = 30000
    d = inputs.plummer(n, 29, masses="kroupa")
    p = c1_params(order=2, precision=B.PT_MIXED)
    p.r_out, p.r_in = 0.01, 0.001
    pos, mass = torch.from_numpy(d["pos"]).cuda(), torch.from_numpy(d["mass"]).cuda()
    t = B.Tree(ctx, pos, mass, p)
    rng = np.random.default_rng(29)
    for step in range(4):
        pos += torch.from_numpy(rng.normal(scale=1e-3, size=(n, 3))).cuda()    # drift in place
        t.rebuild(pos, mass, p)
        acc = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        pot = torch.empty(n, dtype=torch.float64, device="cuda")
        t.force(acc, pot)
        ref = run_gpu(ctx, pos.cpu().numpy(), d["mass"], p, neighbours=False)
        assert np.array_equal(acc.cpu().numpy(), ref["acc"]), step
        assert np.array_equal(pot.cpu().numpy(), ref["pot"]), step
    t.free()


@pytest.mark.parametrize("n_leaf", [1, 2, 16, 17, 32, 64])
def test_topology_every_leaf_size(ctx, n_leaf):
    """Leaf sizes on both sides of the topology kernel's thread / warp split
    (nodes above 16 particles take a warp): the node set, boxes, moments,
    groups and lists equal the oracle's, and the numbering is breadth-first
    in key order with every internal node's children contiguous on the next
    level, tiling its particle range in order.  Binaries from n_leaf 2 on (a
    tight pair is then a leaf, summed from its particles); at n_leaf 1 a pair
    that a cell face splits is combined from two child records whose COMs
    carry the rounding of absolute float64 positions (~1e-16 against a
    separation down to ~1e-9), which the quadrupole tolerance of the node
    comparison does not cover, so n_leaf 1 takes a Plummer set."""
    d = inputs.plummer_binaries(2048, 40 + n_leaf) if n_leaf > 1 else inputs.plummer(4096, 41)
    p = c1_params(order=2, n_leaf=n_leaf, n_group=64)
    g = run_gpu(ctx, d["pos"], d["mass"], p)
    T = oracle.Tree(d["pos"], d["mass"], p.n_leaf, p.n_group)
    check_structure(g, T, p)
    nd = g["tree"].nodes()
    lv, b, c = nd["level"], nd["begin"], nd["count"]
    assert np.all(np.diff(lv) >= 0)
    same = np.diff(lv) == 0
    assert np.all(np.diff(b)[same] > 0)
    for v in np.nonzero(nd["leaf"] == 0)[0]:
        f, k = nd["first_child"][v], nd["nchild"][v]
        assert 1 <= k <= 8
        ch = np.arange(f, f + k)
        assert np.all(lv[ch] == lv[v] + 1)
        assert b[ch[0]] == b[v] and b[ch[-1]] + c[ch[-1]] == b[v] + c[v]
        assert np.all(b[ch[1:]] == b[ch[:-1]] + c[ch[:-1]])


def _later_walk_case(kind):
    if kind == "plummer":
        d = inputs.plummer(4096, 1)
        return d["pos"], d["mass"], c1_params(order=2)
    if kind == "mono":
        d = inputs.plummer(4096, 5)
        return d["pos"], d["mass"], c1_params(order=0, n_leaf=4, n_group=16)
    if kind == "binaries":
        d = inputs.plummer_binaries(2048, 44)
        return d["pos"], d["mass"], c1_params(order=2, n_leaf=16, n_group=64)
    if kind == "groups24":
        d = inputs.plummer(6000, 324, masses="kroupa")
        return d["pos"], d["mass"], c1_params(order=2, n_leaf=8, n_group=24)
    r_out = 0.0016                                    # wide sparse groups
    pos = inputs.wide_sparse_groups(r_out, 15, 3, 2)
    mass = np.full(len(pos), 1.0 / len(pos))
    return pos, mass, c1_params(order=2, n_leaf=4, n_group=64, r_out=r_out, r_in=0.1 * r_out, theta=0.5)


@pytest.mark.parametrize("kind", ["plummer", "mono", "binaries", "groups24", "wide"])
def test_later_walks_equal_the_oracle(ctx, kind):
    """A tree's later walks run in one pass into arrays sized from the last
    walk: on Plummer, monopole, binary, 24-target-group and wide sparse-group
    sets every group's cell and PP lists equal the oracle's as sets, the
    float64 forces match the oracle tree, the neighbour lists brute force, and
    the lists equal those of the tree's first (two-pass) walk."""
    pos, mass, p = _later_walk_case(kind)
    T = oracle.Tree(pos, mass, p.n_leaf, p.n_group)
    g1 = run_gpu(ctx, pos, mass, p)                  # first walk: two passes
    st1 = g1["stats"]
    co1, cells1, po1, pp1 = g1["tree"].lists(st1["cell_list_total"], st1["pp_list_total"])
    g = run_gpu(ctx, pos, mass, p, repeat=3)         # later walks: one pass
    check_structure(g, T, p)
    st = g["stats"]
    co, cells, po, pp = g["tree"].lists(st["cell_list_total"], st["pp_list_total"])
    for k in range(len(co) - 1):
        assert np.array_equal(np.sort(cells[co[k]:co[k + 1]]), np.sort(cells1[co1[k]:co1[k + 1]]))
        assert np.array_equal(np.sort(pp[po[k]:po[k + 1]]), np.sort(pp1[po1[k]:po1[k + 1]]))
    a, phi, _ = T.force(p.theta, p.r_in, p.r_out, order=p.order)
    assert rel_err(g["acc"], a).max() <= FP64_TOL
    assert (np.abs(g["pot"] - phi) / np.abs(phi)).max() <= FP64_TOL
    check_neighbours(g, pos, p.r_out)
    for k in ("cell_interactions", "pp_interactions"):
        assert st[k] == st1[k]
