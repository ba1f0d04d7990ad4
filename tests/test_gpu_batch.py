"""pt_batch_longrange_force: many independent sets in one pass of the pipeline.

Every set gets its own root box, keys, tree, groups and lists, and its
groups accumulate in the same order as when the set is evaluated alone, so a
batch result must equal the single-set result bit for bit.  The captured
graph must give the same results as the uncaptured launch sequence, also
after the positions move (the graph is replayed with new inputs).
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


def _clusters(seed, sizes):
    out = []
    for k, n in enumerate(sizes):
        c = inputs.plummer(n, seed + k, masses="kroupa")
        c["r_out"] = inputs.r_out_first_guess(n)
        c["r_in"] = 0.1 * c["r_out"]
        out.append(c)
    return out


def _params(precision=B.PT_FP64):
    return B.Params(theta=0.4, n_leaf=8, n_group=64, order=2, precision=precision)


def _run_batch(ctx, cl, prm, flags=0, device=True, nb=True, cap_scale=8):
    import torch
    keep, descs = [], []
    for c in cl:
        n = len(c["mass"])
        if device:
            pos = torch.from_numpy(c["pos"]).cuda()
            mass = torch.from_numpy(c["mass"]).cuda()
            acc = torch.empty((n, 3), dtype=torch.float64, device="cuda")
            pot = torch.empty((n,), dtype=torch.float64, device="cuda")
            off = torch.empty((n + 1,), dtype=torch.int64, device="cuda") if nb else None
            idx = torch.empty((cap_scale * n + 16,), dtype=torch.int32, device="cuda") if nb else None
        else:
            pos, mass = c["pos"], c["mass"]
            acc, pot = np.zeros((n, 3)), np.zeros(n)
            off = np.zeros(n + 1, dtype=np.int64) if nb else None
            idx = np.zeros(cap_scale * n + 16, dtype=np.int32) if nb else None
        keep.append((pos, mass, acc, pot, off, idx))
        d = B.pt_cluster_desc()
        d.n = n
        d.pos, d.mass, d.acc, d.pot = (B._ptr(pos), B._ptr(mass), B._ptr(acc), B._ptr(pot))
        d.r_in, d.r_out = c["r_in"], c["r_out"]
        d.nb_offsets = B._ptr(off)
        d.nb_idx = B._ptr(idx)
        d.nb_capacity = (cap_scale * n + 16) if nb else 0
        descs.append(d)
    rc, arr, st = B.pt_batch_longrange_force(ctx.h, descs, prm.c(), flags)
    res = []
    for (pos, mass, acc, pot, off, idx), d in zip(keep, arr):
        to_np = (lambda x: x.cpu().numpy()) if device else (lambda x: x)
        r = {"acc": to_np(acc), "pot": to_np(pot), "nb_total": d.nb_total}
        if nb and rc == B.PT_OK:
            r["nb_off"] = to_np(off)
            r["nb_idx"] = to_np(idx)[: d.nb_total]
        res.append(r)
    return rc, res, st.as_dict()


@pytest.mark.parametrize("precision", [B.PT_FP64, B.PT_MIXED])
def test_batch_equals_single_sets(ctx, precision):
    cl = _clusters(300, [1, 17, 257, 1024, 3000, 6000])
    prm = _params(precision)
    rc, res, st = _run_batch(ctx, cl, prm)
    assert rc == B.PT_OK, B.pt_last_error(ctx.h)
    for c, r in zip(cl, res):
        p1 = B.Params(**{**prm.__dict__, "r_in": c["r_in"], "r_out": c["r_out"]})
        g = run_gpu(ctx, c["pos"], c["mass"], p1)
        assert np.array_equal(r["acc"], g["acc"])
        assert np.array_equal(r["pot"], g["pot"])
        assert np.array_equal(r["nb_off"], g["nb_off"])
        assert np.array_equal(r["nb_idx"], g["nb_idx"])
        g["tree"].free()


def test_batch_vs_oracle_fp64(ctx):
    cl = _clusters(400, [500, 2000, 4000])
    rc, res, _ = _run_batch(ctx, cl, _params())
    assert rc == B.PT_OK
    for c, r in zip(cl, res):
        T = oracle.Tree(c["pos"], c["mass"], 8, 64)
        a, phi, _ = T.force(0.4, c["r_in"], c["r_out"], order=2)
        assert rel_err(r["acc"], a).max() <= 1e-10
        np.testing.assert_allclose(r["pot"], phi, rtol=1e-10)
        off, idx = oracle.neighbours(c["pos"], c["r_out"])
        assert np.array_equal(r["nb_off"], off) and np.array_equal(r["nb_idx"], idx)


def test_batch_host_buffers(ctx):
    cl = _clusters(500, [700, 1500, 2500])
    prm = _params(B.PT_MIXED)
    rc1, r_dev, _ = _run_batch(ctx, cl, prm, device=True)
    rc2, r_host, _ = _run_batch(ctx, cl, prm, device=False)
    assert rc1 == rc2 == B.PT_OK
    for a, b in zip(r_dev, r_host):
        for k in ("acc", "pot", "nb_off", "nb_idx"):
            assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("device", [True, False])
def test_graph_replay_matches_uncaptured(ctx, device):
    cl = _clusters(600, [900, 1800, 3600, 5000])
    prm = _params(B.PT_MIXED)
    rc, ref, _ = _run_batch(ctx, cl, prm, device=device)                      # uncaptured
    rc1, first, _ = _run_batch(ctx, cl, prm, flags=B.PT_BATCH_GRAPH, device=device)   # captures
    rc2, replay, _ = _run_batch(ctx, cl, prm, flags=B.PT_BATCH_GRAPH, device=device)  # replays
    assert rc == rc1 == rc2 == B.PT_OK, B.pt_last_error(ctx.h)
    for a, b, c in zip(ref, first, replay):
        for k in ("acc", "pot", "nb_off", "nb_idx"):
            assert np.array_equal(a[k], b[k]) and np.array_equal(a[k], c[k]), k
    # the same shape with moved particles: the replayed graph sees the new inputs
    rng = np.random.default_rng(1)
    for c in cl:
        c["pos"] = c["pos"] + 1e-3 * rng.normal(size=c["pos"].shape)
    rc3, moved_graph, _ = _run_batch(ctx, cl, prm, flags=B.PT_BATCH_GRAPH, device=device)
    rc4, moved_ref, _ = _run_batch(ctx, cl, prm, device=device)
    assert rc3 == rc4 == B.PT_OK
    for a, b in zip(moved_graph, moved_ref):
        for k in ("acc", "pot", "nb_off", "nb_idx"):
            assert np.array_equal(a[k], b[k]), k


def test_batch_capacity_error_is_per_cluster(ctx):
    cl = _clusters(700, [800, 800])
    for c in cl:
        c["r_out"] = 0.4
        c["r_in"] = 0.04
    rc, res, _ = _run_batch(ctx, cl, _params(), cap_scale=0)
    assert rc == B.PT_ERR_CAPACITY
    for c, r in zip(cl, res):
        off, _ = oracle.neighbours(c["pos"], c["r_out"])
        assert r["nb_total"] == off[-1]
        T = oracle.Tree(c["pos"], c["mass"], 8, 64)
        a, _, _ = T.force(0.4, c["r_in"], c["r_out"], order=2)
        assert rel_err(r["acc"], a).max() <= 1e-10


def test_batch_argument_errors(ctx):
    cl = _clusters(800, [100, 200])
    cl[1]["r_in"] = cl[1]["r_out"]
    rc, _, _ = _run_batch(ctx, cl, _params())
    assert rc == B.PT_ERR_ARG


def test_autotune_picks_a_candidate_and_caches(ctx):
    import torch
    cl = _clusters(900, [2000, 5000, 9000])
    sets = [{"pos": torch.from_numpy(c["pos"]).cuda(), "mass": torch.from_numpy(c["mass"]).cuda(),
             "r_in": c["r_in"], "r_out": c["r_out"]} for c in cl]
    bt = B.Batch(sets)
    base = _params(B.PT_MIXED)
    best, ms = bt.autotune(ctx, base, leafs=[4, 16], groups=[32, 64], reps=1)
    assert best.n_leaf in (4, 16) and best.n_group in (32, 64) and ms > 0
    again, ms2 = bt.autotune(ctx, base, leafs=[4, 16], groups=[32, 64], reps=1)
    assert (again.n_leaf, again.n_group, ms2) == (best.n_leaf, best.n_group, ms)   # from the cache
    bt.run(ctx, best)
    for k, c in enumerate(cl):
        T = oracle.Tree(c["pos"], c["mass"], best.n_leaf, best.n_group)
        a, _, _ = T.force(0.4, c["r_in"], c["r_out"], order=2)
        e = rel_err(bt.acc[k].cpu().numpy(), a)
        assert np.percentile(e, 99) <= 1e-6


def test_group_count_beyond_the_hint(ctx):
    """A batch step sizes its force grid from the previous step's group count
    (with head room); when a step has many more groups than that, the groups
    beyond the grid are taken from a counter.  Here the previous step has
    every cluster's particles coincident (one depth-capped leaf and one group
    per cluster), the next one Plummer clusters: the results equal single-set
    runs bit for bit, uncaptured and replayed from a graph captured on the
    coincident step."""
    cl = _clusters(700, [600, 1500, 3000])
    prm = _params(B.PT_MIXED)
    same = [dict(c, pos=np.zeros_like(c["pos"]) + 0.25) for c in cl]
    singles = []
    for c in cl:
        p1 = B.Params(**{**prm.__dict__, "r_in": c["r_in"], "r_out": c["r_out"]})
        g = run_gpu(ctx, c["pos"], c["mass"], p1, neighbours=False)
        singles.append((g["acc"], g["pot"]))
        g["tree"].free()
    for flags in (0, B.PT_BATCH_GRAPH):
        rc0, _, st0 = _run_batch(ctx, same, prm, flags=flags, nb=False)
        assert rc0 == B.PT_OK, B.pt_last_error(ctx.h)
        assert st0["groups"] == len(cl)
        rc, res, st = _run_batch(ctx, cl, prm, flags=flags, nb=False)
        assert rc == B.PT_OK, B.pt_last_error(ctx.h)
        assert st["groups"] > len(cl) + len(cl) // 8 + 64    # more than the grid of the hint
        for (a, p), r in zip(singles, res):
            assert np.array_equal(r["acc"], a) and np.array_equal(r["pot"], p)
