"""The serving loop: resident state, admission by HBM budget, continuous
batching, and results that do not depend on what a request was batched with."""
import numpy as np
import pytest

import oracle
from paper_2006_16560_gb300 import binding as B
from paper_2006_16560_gb300 import inputs
from paper_2006_16560_gb300.serve import Server, poisson_load
from gpu_helpers import rel_err

pytestmark = pytest.mark.gpu

DT_DRIFT, DT_KICK = 2e-4, 1e-4
WAIT_S = 60.0     # a request not served within this fails the test instead of hanging it


@pytest.fixture(scope="module")
def ctx():
    return B.Context(0)


def _sims(seed, sizes):
    out = []
    for k, n in enumerate(sizes):
        c = inputs.plummer(n, seed + k, masses="kroupa")
        c["r_out"] = inputs.r_out_first_guess(n)
        c["r_in"] = 0.1 * c["r_out"]
        out.append(c)
    return out


def _params():
    return B.Params(theta=0.4, n_leaf=16, n_group=64, order=2, precision=B.PT_MIXED)


def _server(ctx, sims, **kw):
    s = Server(ctx, _params(), **kw)
    ids = [s.add_sim(c["pos"], c["vel"], c["mass"], c["r_in"], c["r_out"]) for c in sims]
    return s, ids


def test_result_is_the_same_alone_and_in_the_mix(ctx):
    sims = _sims(50, [3000, 12000, 800, 25000, 5000, 40000])
    alone = []
    for c in sims:                      # one request, nothing else queued
        s, (sid,) = _server(ctx, [c])
        info = s.wait(s.submit(sid, DT_DRIFT, DT_KICK), timeout=WAIT_S)
        assert info["batch_size"] == 1
        alone.append(s.read(sid))
        s.close()
    # all requests queued together: one worker batches them; three workers
    # run them in overlapping batches on separate streams
    for workers in (1, 3):
        s = Server(ctx, _params(), workers=workers, max_batch_particles=1 << 20)
        ids = [s.add_sim(c["pos"], c["vel"], c["mass"], c["r_in"], c["r_out"]) for c in sims]
        tickets = [s.submit(i, DT_DRIFT, DT_KICK) for i in ids]
        infos = [s.wait(t, timeout=WAIT_S) for t in tickets]
        if workers == 1:
            assert max(i["batch_size"] for i in infos) > 1
        for sid, a in zip(ids, alone):
            mixed = s.read(sid)
            for x, y in zip(a, mixed):
                assert np.array_equal(x, y)
        s.close()


def test_concurrent_workers_keep_each_simulations_order(ctx):
    """Several requests per simulation submitted at once: with three workers
    a simulation's requests still run one after the other, in order, so the
    state after k requests equals that of one worker serving them."""
    sims = _sims(60, [4000, 9000, 2500])
    out = {}
    for workers in (1, 3):
        s = Server(ctx, _params(), workers=workers)
        ids = [s.add_sim(c["pos"], c["vel"], c["mass"], c["r_in"], c["r_out"]) for c in sims]
        tickets = [s.submit(i, DT_DRIFT * (1 + k), DT_KICK) for k in range(3) for i in ids]
        for t in tickets:
            s.wait(t, timeout=WAIT_S)
        out[workers] = [s.read(i) for i in ids]
        s.close()
    for a, b in zip(out[1], out[3]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_request_is_drift_force_kick(ctx):
    """Two requests in a row equal drift, force (library call), kick twice."""
    (c,) = _sims(70, [6000])
    s, (sid,) = _server(ctx, [c])
    for _ in range(2):
        s.wait(s.submit(sid, DT_DRIFT, DT_KICK), timeout=WAIT_S)
    pos, vel, acc, pot = s.read(sid)
    s.close()
    x, v = c["pos"].copy(), c["vel"].copy()
    p = B.Params(**{**_params().__dict__, "r_in": c["r_in"], "r_out": c["r_out"]})
    for _ in range(2):
        x = x + v * DT_DRIFT
        t = B.Tree(ctx, x, c["mass"], p)
        a, ph = np.zeros_like(x), np.zeros(len(x))
        cap = 16 * len(x) + 64
        t.force(a, ph, np.zeros(len(x) + 1, dtype=np.int64), np.zeros(cap, dtype=np.int32), cap)
        t.free()
        v = v + a * DT_KICK
    assert np.array_equal(pos, x) and np.array_equal(vel, v) and np.array_equal(acc, a)
    # and the force is the P3T long-range force of the drifted set
    T = oracle.Tree(pos, c["mass"], 16, 64)
    ao, _, _ = T.force(0.4, c["r_in"], c["r_out"], order=2)
    assert np.percentile(rel_err(acc, ao), 99) <= 1e-6


def test_admission_by_budget(ctx):
    (c,) = _sims(90, [20000])
    s = Server(ctx, _params(), hbm_budget_bytes=40e6, max_batch_particles=10000, workers=1)
    rc, _ = s.try_add_sim(c["pos"], c["vel"], c["mass"], c["r_in"], c["r_out"])
    assert rc == B.PT_ERR_CAPACITY          # larger than a batch may hold
    small = _sims(91, [5000])[0]
    rc, sid = s.try_add_sim(small["pos"], small["vel"], small["mass"], small["r_in"], small["r_out"])
    assert rc == B.PT_OK
    # the budget fills up: 40 MB minus a 15 MB workspace reserve
    ok = 0
    for k in range(40):
        rc, _ = s.try_add_sim(small["pos"], small["vel"], small["mass"], small["r_in"], small["r_out"])
        if rc != B.PT_OK:
            assert rc == B.PT_ERR_CAPACITY
            break
        ok += 1
    assert 0 < ok < 40
    assert s.stats()["resident_bytes"] <= 40e6
    s.close()


def test_poisson_load_smoke(ctx):
    sims = _sims(120, [2000, 4000, 8000, 16000])
    s, ids = _server(ctx, sims)
    r = poisson_load(s, ids, rate=200.0, duration_s=0.5, seed=3, timeout=WAIT_S)
    assert r["requests"] > 0 and r["errors"] == 0
    assert r["latency_ms"]["p99"] >= r["latency_ms"]["p50"] > 0
    s.close()
