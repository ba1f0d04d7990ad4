"""Mass-dependent changeover radii (Sec. 6.1, Eqs. 12 and 16) on the GPU,
against the oracle with the same per-particle factors."""
import numpy as np
import pytest

import oracle
from paper_2006_16560_gb300 import binding as B
from paper_2006_16560_gb300 import inputs
from gpu_helpers import node_ids, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return B.Context(0)


def _run(ctx, d, p, scale):
    import torch
    n = len(d["mass"])
    t = B.Tree(ctx, torch.from_numpy(d["pos"]).cuda(), torch.from_numpy(d["mass"]).cuda(), p,
               scale=None if scale is None else torch.from_numpy(scale).cuda())
    acc = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    pot = torch.empty(n, dtype=torch.float64, device="cuda")
    off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    idx = torch.empty(32 * n + 64, dtype=torch.int32, device="cuda")
    total, st, _ = t.force(acc, pot, off, idx, 32 * n + 64)
    return {"acc": acc.cpu().numpy(), "pot": pot.cpu().numpy(), "nb_off": off.cpu().numpy(),
            "nb_idx": idx[:total].cpu().numpy(), "stats": st.as_dict(), "tree": t}


def _params(precision=B.PT_FP64, order=2):
    return B.Params(theta=0.5, r_in=0.004, r_out=0.04, n_leaf=8, n_group=64, order=order,
                    precision=precision, mass_dependent=1)


@pytest.mark.parametrize("order", [0, 2])
def test_scaled_fp64_vs_oracle(ctx, order):
    d = inputs.plummer(4096, 41, masses="kroupa")
    s = oracle.radius_scale(d["mass"])
    assert s.max() > 3
    p = _params(order=order)
    g = _run(ctx, d, p, s)
    T = oracle.Tree(d["pos"], d["mass"], 8, 64, scale=s)
    a, phi, st = T.force(p.theta, p.r_in, p.r_out, order=order)
    assert rel_err(g["acc"], a).max() <= 1e-10
    assert (np.abs(g["pot"] - phi) / np.abs(phi)).max() <= 1e-10
    assert (g["stats"]["cell_interactions"], g["stats"]["pp_interactions"]) == st
    off, idx = oracle.neighbours(d["pos"], p.r_out, scale=s)
    assert np.array_equal(g["nb_off"], off) and np.array_equal(g["nb_idx"], idx)
    # every group's lists equal the oracle's walk with the larger-factor gap rule
    info, _ = g["tree"].info()
    co, cells, po, pp = g["tree"].lists(g["stats"]["cell_list_total"], g["stats"]["pp_list_total"])
    gn, on = g["tree"].nodes(), T.nodes()
    for k in range(0, int(info[2]), 3):
        oc, op = T.walk(k, p.theta, p.r_out)
        assert node_ids(gn, cells[co[k]:co[k + 1]]) == node_ids(on, oc)
        assert np.array_equal(np.sort(pp[po[k]:po[k + 1]]), np.sort(op))


def test_scaled_mixed_vs_fp64(ctx):
    d = inputs.plummer(20000, 42, masses="kroupa")
    s = oracle.radius_scale(d["mass"])
    g64 = _run(ctx, d, _params(), s)
    gmx = _run(ctx, d, _params(B.PT_MIXED), s)
    e = rel_err(gmx["acc"], g64["acc"])
    assert np.percentile(e, 99) <= 1e-6 and e.max() <= 1e-4
    assert np.array_equal(gmx["nb_idx"], g64["nb_idx"])


def test_device_eq12_factors(ctx):
    """NULL factors with mass_dependent = 1: Eq. 12 is computed on the device."""
    d = inputs.plummer(8000, 43, masses="kroupa")
    s = oracle.radius_scale(d["mass"])
    ref = _run(ctx, d, _params(B.PT_MIXED), s)
    dev = _run(ctx, d, _params(B.PT_MIXED), None)
    assert rel_err(dev["acc"], ref["acc"]).max() <= 1e-12
    assert np.array_equal(dev["nb_idx"], ref["nb_idx"])


@pytest.mark.parametrize("precision", [B.PT_FP64, B.PT_MIXED])
def test_unit_factors_match_scalar_radii(ctx, precision):
    d = inputs.plummer(6000, 44, masses="kroupa")
    p0 = B.Params(**{**_params(precision).__dict__, "mass_dependent": 0})
    g0 = _run(ctx, d, p0, None)
    g1 = _run(ctx, d, _params(precision), np.ones(6000))
    np.testing.assert_allclose(g1["acc"], g0["acc"], rtol=1e-13, atol=1e-13 * np.abs(g0["acc"]).max())
    assert np.array_equal(g1["nb_idx"], g0["nb_idx"])


def test_scaled_batch_equals_single(ctx):
    import torch
    sets, singles = [], []
    for k, n in enumerate([700, 3000, 9000]):
        c = inputs.plummer(n, 50 + k, masses="kroupa")
        sc = oracle.radius_scale(c["mass"])
        r_out = inputs.r_out_first_guess(n)
        sets.append({"pos": torch.from_numpy(c["pos"]).cuda(), "mass": torch.from_numpy(c["mass"]).cuda(),
                     "r_in": 0.1 * r_out, "r_out": r_out, "scale": torch.from_numpy(sc).cuda()})
        p = B.Params(**{**_params(B.PT_MIXED).__dict__, "r_in": 0.1 * r_out, "r_out": r_out, "theta": 0.4})
        singles.append(_run(ctx, c, p, sc))
    bt = B.Batch(sets)
    for dsc, st in zip(bt.descs, sets):
        dsc.radius_scale = B._ptr(st["scale"])
    bt.arr = (B.pt_cluster_desc * len(bt.descs))(*bt.descs)
    bt.run(ctx, B.Params(**{**_params(B.PT_MIXED).__dict__, "theta": 0.4}))
    for k, g in enumerate(singles):
        assert np.array_equal(bt.acc[k].cpu().numpy(), g["acc"])
        assert np.array_equal(bt.pot[k].cpu().numpy(), g["pot"])


@pytest.mark.parametrize("bad", [0.0, -1.5, float("nan"), float("inf")])
def test_bad_radius_factor_is_an_argument_error(ctx, bad):
    """A radius factor that is not finite and positive is rejected by the build
    (PT_ERR_ARG), and the context stays usable."""
    import torch
    d = inputs.plummer(2000, 61, masses="kroupa")
    sc = oracle.radius_scale(d["mass"])
    sc[1234] = bad
    pos, mass = torch.from_numpy(d["pos"]).cuda(), torch.from_numpy(d["mass"]).cuda()
    with pytest.raises(B.PTError) as e:
        B.Tree(ctx, pos, mass, _params(), scale=torch.from_numpy(sc).cuda())
    assert e.value.code == B.PT_ERR_ARG and "radius factor" in str(e.value)
    sc[1234] = 1.0
    g = _run(ctx, d, _params(), sc)
    assert np.all(np.isfinite(g["acc"]))
