"""Orbit-dependent neighbour lists (Sec. 6.3.1, Eq. 24) on the GPU against
the oracle's brute-force two-stage search: bit-exact CSR lists, candidate
counts and r_nb."""
import numpy as np
import pytest

import oracle
from paper_2006_16560_gb300 import binding as B
from paper_2006_16560_gb300 import inputs

pytestmark = pytest.mark.gpu

MODES = [B.PT_ORBIT_ROUT, B.PT_ORBIT_RNB, B.PT_ORBIT_CANDIDATES]


@pytest.fixture(scope="module")
def ctx():
    return B.Context(0)


def _cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _tree(ctx, d, r_out, massdep, n_leaf=16, n_group=64):
    """Mass-dependent trees get the oracle's Eq. 12 factors explicitly (the
    device's own factors are compared with them elsewhere)."""
    p = B.Params(theta=0.4, r_in=0.1 * r_out, r_out=r_out, n_leaf=n_leaf, n_group=n_group, order=2,
                 precision=B.PT_MIXED, mass_dependent=massdep)
    sc = _cuda(oracle.radius_scale(d["mass"])) if massdep else None
    return B.Tree(ctx, _cuda(d["pos"]), _cuda(d["mass"]), p, scale=sc)


def _check(ctx, d, r_out, dt, massdep, mode, C_v=1.5, **kw):
    t = _tree(ctx, d, r_out, massdep, **kw)
    rnb = _cuda(np.zeros(len(d["mass"])))
    off, idx, cand = t.orbit_neighbours(_cuda(d["vel"]), dt, 3.0, C_v, mode, r_nb=rnb)
    sc = oracle.radius_scale(d["mass"]) if massdep else None
    o_off, o_idx, o_cand = oracle.orbit_neighbours(d["pos"], d["vel"], d["mass"], r_out, dt, 3.0, C_v,
                                                   mode=mode, scale=sc)
    assert np.array_equal(rnb.cpu().numpy(), oracle.neighbour_radius(d["vel"], r_out, dt, 3.0, sc))
    assert np.array_equal(off.cpu().numpy(), o_off)
    assert np.array_equal(idx.cpu().numpy(), o_idx)
    assert cand == int(o_cand.sum())
    return t, o_off, o_cand


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("massdep", [0, 1])
def test_plummer_vs_oracle(ctx, mode, massdep):
    n = 12000
    d = inputs.plummer(n, 31 + massdep, masses="kroupa")
    r_out = 0.03
    _, off, cand = _check(ctx, d, r_out, 0.5 * r_out / 0.41, massdep, mode)
    assert off[-1] > n
    if mode == B.PT_ORBIT_ROUT:
        assert off[-1] < cand.sum()          # stage 2 drops some candidates


def test_fast_particles_and_ragged_tree(ctx):
    """A few particles 50x faster (search radii across much of the system),
    n not a multiple of any tile, small leaves and groups."""
    n = 7777
    d = inputs.plummer(n, 33, masses="kroupa")
    d["vel"] = d["vel"].copy()
    d["vel"][::331] *= 50
    r_out = inputs.r_out_first_guess(n)
    for mode in MODES:
        _check(ctx, d, r_out, 0.3 * r_out / 0.41, 1, mode, n_leaf=4, n_group=16)


def test_binaries_workload(ctx):
    """Kroupa (1995) binaries: members share a position to a few AU and move
    fast relative to each other."""
    d = inputs.kroupa95_binaries(4000, 35)
    r_out = inputs.r_out_first_guess(len(d["mass"]))
    _check(ctx, d, r_out, 0.3 * r_out / 0.41, 1, B.PT_ORBIT_ROUT)


def test_zero_velocity_equals_force_neighbours(ctx):
    import torch
    n = 9000
    d = inputs.plummer(n, 37, masses="kroupa")
    d["vel"] = np.zeros_like(d["vel"])
    r_out = inputs.r_out_first_guess(n)
    t = _tree(ctx, d, r_out, 1)
    acc = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    pot = torch.empty(n, dtype=torch.float64, device="cuda")
    off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    idx = torch.empty(16 * n, dtype=torch.int32, device="cuda")
    total, _, _ = t.force(acc, pot, off, idx, 16 * n)
    o2, i2, _ = t.orbit_neighbours(_cuda(d["vel"]), 0.1)
    assert torch.equal(o2, off) and torch.equal(i2, idx[:total])


def test_host_arrays_and_capacity(ctx):
    n = 3000
    d = inputs.plummer(n, 39)
    r_out = inputs.r_out_first_guess(n)
    t = _tree(ctx, d, r_out, 0)
    op = B.pt_orbit_params(0.05, 3.0, 1.5, B.PT_ORBIT_ROUT)
    off = np.zeros(n + 1, dtype=np.int64)
    idx = np.zeros(10, dtype=np.int32)
    rc, total, cand = B.pt_orbit_neighbours(t.h, B._ptr(d["vel"]), op, B._ptr(off), B._ptr(idx), 10)
    assert rc == B.PT_ERR_CAPACITY and total > 10
    idx = np.zeros(total, dtype=np.int32)
    rc, total2, cand2 = B.pt_orbit_neighbours(t.h, B._ptr(d["vel"]), op, B._ptr(off), B._ptr(idx), total)
    assert rc == B.PT_OK and (total2, cand2) == (total, cand)
    o_off, o_idx, _ = oracle.orbit_neighbours(d["pos"], d["vel"], d["mass"], r_out, 0.05)
    assert np.array_equal(off, o_off) and np.array_equal(idx, o_idx)
    bad = B.pt_orbit_params(-1.0, 3.0, 1.5, 0)
    assert B.pt_orbit_neighbours(t.h, B._ptr(d["vel"]), bad, None, None, 0)[0] == B.PT_ERR_ARG
    bad = B.pt_orbit_params(0.1, 3.0, 1.5, 7)
    assert B.pt_orbit_neighbours(t.h, B._ptr(d["vel"]), bad, None, None, 0)[0] == B.PT_ERR_ARG


def test_full_size_sampled_rows(ctx):
    """10^6 Plummer particles with velocities: sampled rows against the
    oracle's brute force for those targets, symmetry on every row."""
    n = 1 << 20
    d = inputs.plummer(n, 2, masses="kroupa")
    r_out = 0.003
    t = _tree(ctx, d, r_out, 0)
    off, idx, cand = t.orbit_neighbours(_cuda(d["vel"]), 0.3 * r_out / 0.41)
    off, idx = off.cpu().numpy(), idx.cpu().numpy()
    rng = np.random.default_rng(5)
    tg = np.sort(rng.choice(n, 300, replace=False))
    o_off, o_idx, _ = oracle.orbit_neighbours(d["pos"], d["vel"], d["mass"], r_out, 0.3 * r_out / 0.41,
                                              targets=tg)
    for k, i in enumerate(tg):
        assert np.array_equal(idx[off[i]:off[i + 1]], o_idx[o_off[k]:o_off[k + 1]])
    # symmetric relation: the multiset of (i, j) equals that of (j, i)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(off))
    a = rows * n + idx
    b = idx.astype(np.int64) * n + rows
    assert np.array_equal(np.sort(a), np.sort(b))
    assert off[-1] <= cand
