"""Parity at the full benchmark sizes, in the benchmark's launch configuration.

The oracle computes sampled targets one by one (its own walk of the target's
group and the tree force), brute-force neighbour sets for sampled targets, and
the whole key order / topology, which it builds in seconds even at 10^7.
"""
import numpy as np
import pytest

import oracle
from paper_2006_16560_gb300 import binding as B
from paper_2006_16560_gb300 import inputs
from gpu_helpers import rel_err, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return B.Context(0)


def c2_params(precision=B.PT_FP64):
    """Kroupa Plummer workload: quadrupole, theta 0.3, leaf 16, r_out 0.003, r_in 0.1 r_out."""
    return B.Params(theta=0.3, r_in=0.0003, r_out=0.003, n_leaf=16, n_group=64, order=2,
                    precision=precision)


def sampled_parity(ctx, d, p, nsample, seed, check_mixed=True):
    n = len(d["mass"])
    g = run_gpu(ctx, d["pos"], d["mass"], p)
    T = oracle.Tree(d["pos"], d["mass"], p.n_leaf, p.n_group)
    key, q, perm = T.keys()
    gk, gperm = g["tree"].keys()
    assert np.array_equal(gperm.astype(np.int64), perm)
    assert np.array_equal(gk, key[perm])
    info, _ = g["tree"].info()
    assert info[1] == T.nnodes and info[2] == T.ngroups
    rng = np.random.default_rng(seed)
    tg = np.unique(np.concatenate([rng.choice(n, nsample, replace=False), [0, n - 1]]))
    a, phi, _ = T.force(p.theta, p.r_in, p.r_out, order=p.order, targets=tg)
    assert rel_err(g["acc"][tg], a).max() <= 1e-10
    assert (np.abs(g["pot"][tg] - phi) / np.abs(phi)).max() <= 1e-10
    off, idx = oracle.neighbours(d["pos"], p.r_out, tg)
    for t, i in enumerate(tg):
        assert np.array_equal(g["nb_idx"][g["nb_off"][i]:g["nb_off"][i + 1]], idx[off[t]:off[t + 1]])
    # CSR well formed: ascending rows, symmetric relation, no self entries
    nb_off, nb_idx = g["nb_off"], g["nb_idx"]
    assert nb_off[0] == 0 and nb_off[-1] == len(nb_idx) and np.all(np.diff(nb_off) >= 0)
    rows = np.repeat(np.arange(n), np.diff(nb_off))
    assert np.all(nb_idx != rows)
    fwd = rows.astype(np.int64) * n + nb_idx
    bwd = nb_idx.astype(np.int64) * n + rows
    assert np.array_equal(np.sort(fwd), np.sort(bwd))
    out = {"g64": g}
    if check_mixed:
        pm = B.Params(**{**p.__dict__, "precision": B.PT_MIXED})
        gm = run_gpu(ctx, d["pos"], d["mass"], pm)
        e = rel_err(gm["acc"], g["acc"])
        out["mixed_p50"], out["mixed_p99"] = np.percentile(e, [50, 99])
        assert out["mixed_p99"] <= 1e-6
        assert np.array_equal(gm["nb_off"], nb_off) and np.array_equal(gm["nb_idx"], nb_idx)
    return out


def test_kroupa_plummer_1m(ctx):
    d = inputs.plummer(1_048_576, 2, masses="kroupa")
    sampled_parity(ctx, d, c2_params(), 300, 7)


def test_binaries_1m(ctx):
    """N = 10^6 with every star in a binary (a = 0.005-50 AU): every companion is
    a neighbour (a < r_in) and the mixed path stays within the bar."""
    d = inputs.plummer_binaries(500_000, 4)
    o = sampled_parity(ctx, d, c2_params(), 200, 8)
    g = o["g64"]
    n = len(d["mass"])
    comp = np.arange(n) ^ 1
    rows = np.repeat(np.arange(n), np.diff(g["nb_off"]))
    have = set((rows.astype(np.int64) * n + g["nb_idx"]).tolist())
    assert all((i * n + comp[i]) in have for i in range(0, n, 97))


def test_kroupa_plummer_10m(ctx):
    d = inputs.plummer(10_000_000, 2, masses="kroupa")
    sampled_parity(ctx, d, c2_params(), 100, 9)


def test_kroupa95_binaries_200k(ctx):
    """The paper's own binary population (Eq. 39 periods, N100kb-like r_out of
    Table 2): every companion closer than r_out is a neighbour."""
    d = inputs.kroupa95_binaries(100_000, 12)
    p = B.Params(theta=0.3, r_in=0.0004, r_out=0.004, n_leaf=16, n_group=64, order=2,
                 precision=B.PT_FP64)
    o = sampled_parity(ctx, d, p, 200, 13)
    g = o["g64"]
    n = len(d["mass"])
    sep = np.linalg.norm(d["pos"][0::2] - d["pos"][1::2], axis=1)
    close = np.nonzero(sep < p.r_out * 0.999)[0]
    assert len(close) > 1000
    rows = np.repeat(np.arange(n), np.diff(g["nb_off"]))
    have = set((rows.astype(np.int64) * n + g["nb_idx"]).tolist())
    assert all((2 * k) * n + 2 * k + 1 in have for k in close[::13])


def test_kroupa_plummer_36m_lists_past_2_32(ctx):
    """N = 3.6*10^7: the cell list holds more than 2^32 entries (the near and
    far PP lists more than 2^31), so every list offset of the walk, the force
    kernel and the CSR must be 64-bit.  The mixed path only (the FP64 path
    would add half a minute): key order, node and group counts, sampled forces
    against the oracle tree, exact neighbour rows of the sampled targets and a
    symmetric CSR."""
    d = inputs.plummer(36_000_000, 2, masses="kroupa")
    n = len(d["mass"])
    p = c2_params(B.PT_MIXED)
    g = run_gpu(ctx, d["pos"], d["mass"], p)
    st = g["stats"]
    assert st["cell_list_total"] > 2**32 and st["pp_list_total"] > 2**31
    T = oracle.Tree(d["pos"], d["mass"], p.n_leaf, p.n_group)
    key, _, perm = T.keys()
    gk, gperm = g["tree"].keys()
    assert np.array_equal(gperm.astype(np.int64), perm) and np.array_equal(gk, key[perm])
    info, _ = g["tree"].info()
    assert info[1] == T.nnodes and info[2] == T.ngroups
    del key, perm, gk, gperm
    rng = np.random.default_rng(10)
    tg = np.unique(np.concatenate([rng.choice(n, 60, replace=False), [0, n - 1]]))
    a, phi, _ = T.force(p.theta, p.r_in, p.r_out, order=p.order, targets=tg)
    e = rel_err(g["acc"][tg], a)
    ep = np.abs(g["pot"][tg] - phi) / np.abs(phi)
    assert np.percentile(e, 99) <= 1e-6 and np.percentile(ep, 99) <= 1e-6
    off, idx = oracle.neighbours(d["pos"], p.r_out, tg)
    nb_off, nb_idx = g["nb_off"], g["nb_idx"]
    for t, i in enumerate(tg):
        assert np.array_equal(nb_idx[nb_off[i]:nb_off[i + 1]], idx[off[t]:off[t + 1]])
    assert nb_off[0] == 0 and nb_off[-1] == len(nb_idx) and np.all(np.diff(nb_off) >= 0)
    rows = np.repeat(np.arange(n), np.diff(nb_off))
    assert np.all(nb_idx != rows)
    fwd = rows.astype(np.int64) * n + nb_idx
    bwd = nb_idx.astype(np.int64) * n + rows
    assert np.array_equal(np.sort(fwd), np.sort(bwd))
