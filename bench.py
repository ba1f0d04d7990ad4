#!/usr/bin/env python
"""Benchmark of the P3T long-range force on one GB300 (or N replicas).

One step = one pass of the whole hot path on a resident particle set:
root box + Morton keys -> radix sort -> octree -> multipoles -> groups ->
group-wise walk (cell and PP lists) -> force kernel with neighbour
extraction -> neighbour CSR -> energy / momentum sums, i.e. pt_tree_build
followed by pt_longrange_force.

Workload: Plummer sphere, N = 1,048,576, Kroupa IMF 0.08-150 Msun rescaled
to M = 1, Henon units, seed 2; quadrupole tree, theta = 0.3, n_leaf = 16,
n_group = 64, r_out = 0.003, r_in = 0.0003; neighbour lists on.

value   = (cell + PP interactions per step) / device time per step of the
          FP32-mixed path (interactions counted from the emitted lists:
          sum over groups of n_G x list length)
e2e     = the same metric through the C ABI with pinned HOST buffers, the
          host<->device copies inside the timed region
fp64    = the plain float64 GPU path on the same workload
roofline: the mixed force kernel against the FP32 CUDA-core peak
          (SMs x 128 lanes x 2 flop x maximum SM clock; 152 x 128 x 2 x
          2.07 GHz = 80.55 TFLOP/s on a GB300), flops per interaction
          counted from the kernel source
c2_10m  = the same workload at N = 10^7 (mixed throughput, stage times,
          mixed vs FP64 error)
binaries_1m = N = 10^6 with every star in a primordial binary (500k pairs):
          mixed and FP64 step times, mixed vs FP64 error, companions found
cpu_baseline / --impl reference: the CPU oracle as it stands, on the host
          cores, on a bounded sample of the same workload
tree_vs_direct: the GPU tree (FP64 and mixed) against the oracle's direct
          O(N^2) sum on sampled targets, p50 / p99 relative error of the
          acceleration and the potential (N = 2^20 and 10^7)
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "P³T long-range interactions/s at N=1M, FP32-mixed vs FP64 plain; p50/p99 latency"
N_DEFAULT = 1_048_576
SEED = 2

# Flops per interaction, counted from the kernel source (FFMA = 2, other
# arithmetic = 1, reciprocal square root = 4 by convention; min / max,
# compares and selects are not counted).  Mixed PP pairs take either the
# changeover path ("pp") or, when no pair of the warp's iteration is within
# r_out, the plain Newtonian pair ("pp_newton"), which is exact there.
FLOPS = {
    ("mixed", "cell", 2): 55, ("mixed", "cell", 0): 22, ("mixed", "pp", None): 77,
    ("mixed", "pp_newton", None): 22,
    ("fp64", "cell", 2): 56, ("fp64", "cell", 0): 22, ("fp64", "pp", None): 53,
}
FP32_LANES = 128                 # FP32 lanes per SM (4 SM sub-partitions x 32)
GB300_SMS, GB300_MAX_MHZ = 152, 2070.0


def fp32_peak(sm_count: int, max_mhz: float) -> float:
    """FP32 CUDA-core peak in flop/s: SMs x 128 lanes x 2 flop (FFMA) x clock."""
    return sm_count * FP32_LANES * 2 * max_mhz * 1e6


def device_sm_count(local: int) -> int:
    import torch
    return int(torch.cuda.get_device_properties(local).multi_processor_count)

# DRAM bytes per launch of the mixed force kernel from one ncu capture of the
# same kernel build on this workload (dram__bytes_read.sum + dram__bytes_write.sum,
# 1.339 GB + 0.081 GB); None when the kernel changed after the capture.
FORCE_MIXED_DRAM_BYTES = 1.420e9


def rank_env():
    """(rank, world size, local rank) from the torchrun environment (1 process: 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, device="cpu") -> float:
    """The largest x over all ranks of the initialised process group (x itself without one)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank: float, ms_max: float, world: int) -> float:
    """Whole-job throughput of `world` independent replicas (weak scaling): every
    rank processes the same workload, the job takes as long as its slowest rank."""
    return world * units_per_rank / (ms_max * 1e-3)


def workload_config(n):
    return {
        "workload": f"Plummer N={n}, Kroupa IMF 0.08-150 Msun (total mass 1), Henon units, seed {SEED}; "
                    "quadrupole tree theta=0.3, n_leaf=16, n_group=64, r_out=0.003, r_in=0.0003; "
                    "neighbour lists on",
        "n": n, "theta": 0.3, "n_leaf": 16, "n_group": 64, "order": 2, "r_out": 0.003, "r_in": 0.0003,
        "l2": "flushed between timed steps (256 MiB write); working set > L2",
        "parallelism": "replicas (one independent set per GPU, no collective)",
    }


def params(precision):
    from paper_2006_16560_gb300 import binding as B
    return B.Params(theta=0.3, r_in=0.0003, r_out=0.003, n_leaf=16, n_group=64, order=2,
                    precision=precision)


def flops_of(stats, kind):
    cells = stats["cell_interactions"] * FLOPS[(kind, "cell", 2)]
    if kind == "mixed":
        full = stats["pp_changeover_interactions"]
        fast = stats["pp_interactions"] - full
        return cells + full * FLOPS[(kind, "pp", None)] + fast * FLOPS[(kind, "pp_newton", None)]
    return cells + stats["pp_interactions"] * FLOPS[(kind, "pp", None)]


class ClockSampler:
    """nvidia-smi clock / throttle samples during a timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(5)
            except Exception:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        try:
            with open(self.f.name) as fh:
                for line in fh:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        finally:
            os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = max((num(r[2]) for r in rows if num(r[2]) is not None), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        load = [s for s in sm if smax and s > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": smax,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def run_steps(ctx, tree_holder, pos, mass, prm, out, k, flush=None, timed=True):
    """k steps of build + force on device buffers; per-step device times (ms)."""
    import torch
    from paper_2006_16560_gb300 import binding as B
    acc, pot, nb_off, nb_idx = out
    times, stats = [], None
    stream = torch.cuda.current_stream()
    for _ in range(k):
        if flush is not None:
            flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if tree_holder[0] is None:
            tree_holder[0] = B.Tree(ctx, pos, mass, prm)
        else:
            tree_holder[0].rebuild(pos, mass, prm)
        _, st, _ = tree_holder[0].force(acc, pot, nb_off, nb_idx, nb_idx.shape[0])
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        stats = st.as_dict()
    return times, stats


def batch_leg(ctx, steps):
    """Ensemble workload: 256 Kroupa Plummer clusters, N log-uniform in
    1,024-65,536 (seed 4), theta 0.4, r_out from Eq. 42, r_in = r_out / 10,
    FP32-mixed, neighbour lists on; n_leaf / n_group from the autotuner.
    Times one batched pass (uncaptured and as a replayed CUDA graph) against
    per-cluster calls of the same work."""
    import torch
    from paper_2006_16560_gb300 import binding as B
    from paper_2006_16560_gb300 import inputs
    ens = inputs.cluster_ensemble(256, 1024, 65536, seed=4)
    sets = [{"pos": torch.from_numpy(c["pos"]).cuda(), "mass": torch.from_numpy(c["mass"]).cuda(),
             "r_in": c["r_in"], "r_out": c["r_out"]} for c in ens]
    ntot = sum(int(c["mass"].shape[0]) for c in ens)
    bt = B.Batch(sets)
    base = B.Params(theta=0.4, n_leaf=8, n_group=64, order=2, precision=B.PT_MIXED)
    t0 = time.perf_counter()
    tuned, tuned_ms = bt.autotune(ctx, base)
    tune_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()

    def timed(fn, k):
        out, st = [], None
        for _ in range(k):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = fn()
            e1.record(stream)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        return out, st

    bt.run(ctx, tuned)
    t_unc, st = timed(lambda: bt.run(ctx, tuned), steps)
    bt.run(ctx, tuned, graph=True)          # sizes and captures
    bt.run(ctx, tuned, graph=True)          # first replay
    t_graph, stg = timed(lambda: bt.run(ctx, tuned, graph=True), steps)
    # per-cluster calls, each set alone through pt_tree_build + pt_longrange_force
    trees = [None] * len(sets)
    prm = [B.Params(**{**tuned.__dict__, "r_in": s_["r_in"], "r_out": s_["r_out"]}) for s_ in sets]

    def per_cluster():
        tot = 0
        for k, s_ in enumerate(sets):
            if trees[k] is None:
                trees[k] = B.Tree(ctx, s_["pos"], s_["mass"], prm[k])
            else:
                trees[k].rebuild(s_["pos"], s_["mass"], prm[k])
            _, st1, _ = trees[k].force(bt.acc[k], bt.pot[k], bt.nb_off[k], bt.nb_idx[k], bt.descs[k].nb_capacity)
            tot += st1.cell_interactions + st1.pp_interactions
        return {"interactions": tot}
    per_cluster()
    t_per, stp = timed(per_cluster, max(2, steps // 2))
    for tr in trees:
        tr.free()
    inter = st["cell_interactions"] + st["pp_interactions"]
    return {
        "workload": "256 Kroupa Plummer clusters, N log-uniform 1024-65536 (seed 4), theta 0.4, "
                    "r_out = 0.2 N^-1/3, r_in = r_out/10, quadrupole, FP32-mixed, neighbour lists on",
        "particles": ntot, "interactions_per_step": inter,
        "autotuned": {"n_leaf": tuned.n_leaf, "n_group": tuned.n_group, "ms": tuned_ms,
                      "tuning_s": tune_s},
        "graph_ms_per_step": statistics.mean(t_graph),
        "uncaptured_ms_per_step": statistics.mean(t_unc),
        "per_cluster_ms_per_step": statistics.mean(t_per),
        "graph_interactions_per_s": inter / (statistics.mean(t_graph) * 1e-3),
        "per_cluster_interactions_per_s": stp["interactions"] / (statistics.mean(t_per) * 1e-3),
        "speedup_graph_vs_per_cluster": statistics.mean(t_per) / statistics.mean(t_graph),
        "launches_per_step": int(stg["launches_force"]),
    }


def serve_leg(ctx, duration_s):
    """Serving workload: 64 resident Kroupa Plummer simulations, N log-uniform
    in 2,000-2,000,000 (seed 5), theta 0.4, leaf 16, FP32-mixed, neighbour lists
    on, HBM budget 150 GB; Poisson arrivals at 200 requests/s, each request a
    drift + long-range force + kick of one simulation.  The server's defaults:
    4 workers, simulations of 2^20 particles or more on two low-priority
    workers, the rest on two high-priority ones, batches of up to 2^22
    particles."""
    import torch
    from paper_2006_16560_gb300 import binding as B
    from paper_2006_16560_gb300 import inputs
    from paper_2006_16560_gb300.serve import Server, poisson_load
    rng = inputs.rng_for(5)
    sizes = np.exp(rng.uniform(math.log(2000), math.log(2_000_000), 64)).astype(np.int64)
    seeds = rng.integers(1, 2 ** 31 - 1, 64)
    prm = B.Params(theta=0.4, n_leaf=16, n_group=64, order=2, precision=B.PT_MIXED)
    srv = Server(ctx, prm, hbm_budget_bytes=150e9, max_sims=64)
    ids = []
    t0 = time.perf_counter()
    for n, sd in zip(sizes, seeds):
        c = inputs.plummer(int(n), int(sd), masses="kroupa")
        r_out = inputs.r_out_first_guess(int(n))
        ids.append(srv.add_sim(c["pos"], c["vel"], c["mass"], 0.1 * r_out, r_out))
    setup_s = time.perf_counter() - t0
    # warm the pipeline's buffers with one request per simulation
    for t in [srv.submit(i, 0.0, 0.0) for i in ids]:
        srv.wait(t)
    r = poisson_load(srv, ids, rate=200.0, duration_s=duration_s, seed=6, dt_drift=1e-5, dt_kick=1e-5,
                     timeout=120.0)
    st = srv.stats()
    srv.close()
    r.update({"workload": "64 resident Kroupa Plummer simulations, N log-uniform 2e3-2e6 (seed 5), "
                          "theta 0.4, leaf 16, FP32-mixed, neighbour lists on, budget 150 GB, "
                          "Poisson arrivals 200/s (seed 6); 4 workers (2 for sims >= 2^20 particles)",
              "resident_particles": int(sizes.sum()), "resident_bytes": st["resident_bytes"],
              "max_batch_particles": st["max_batch_particles"], "setup_s": setup_s})
    return r


def _device_ms(fn, k):
    """Mean device time (ms) of fn() over k calls on the current stream."""
    import torch
    stream = torch.cuda.current_stream()
    out, res = [], None
    for _ in range(k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return statistics.mean(out), res


def orbit_leg(ctx, d, steps):
    """Orbit-dependent neighbour lists (Sec. 6.3.1, Eq. 24) on the headline
    workload: the mixed tree of the same 2^20 particles with their Plummer
    velocities, dt_L = 0.3 r_out / sigma (sigma = 0.41), C_r = 3, C_v = 1.5."""
    import torch
    from paper_2006_16560_gb300 import binding as B
    n = len(d["mass"])
    r_out, sigma = 0.003, 0.41
    dt = 0.3 * r_out / sigma
    pos, mass = torch.from_numpy(d["pos"]).cuda(), torch.from_numpy(d["mass"]).cuda()
    vel = torch.from_numpy(d["vel"]).cuda()
    t = B.Tree(ctx, pos, mass, params(B.PT_MIXED))
    rnb = torch.empty(n, dtype=torch.float64, device="cuda")
    cap = 16 * n
    off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    idx = torch.empty(cap, dtype=torch.int32, device="cuda")
    op = B.pt_orbit_params(dt, 3.0, 1.5, B.PT_ORBIT_ROUT)

    def call():
        rc, tot, cand = B.pt_orbit_neighbours(t.h, B._ptr(vel), op, B._ptr(off), B._ptr(idx), cap,
                                              B._ptr(rnb))
        ctx.check(rc, "pt_orbit_neighbours")
        return tot, cand
    for _ in range(3):
        call()
    ms, (tot, cand) = _device_ms(call, max(3, steps))
    r = (rnb / r_out).cpu().numpy()
    t.free()
    return {"workload": f"Plummer N={n} (seed {SEED}) with its velocities; dt_L = 0.3 r_out/0.41, "
                        "C_r = 3, C_v = 1.5, reference radius r_out,ij",
            "ms": ms, "candidate_pairs": int(cand), "neighbour_pairs": int(tot),
            "r_nb_over_r_out": {"p50": float(np.percentile(r, 50)), "p99": float(np.percentile(r, 99))},
            "particles_per_s": n / (ms * 1e-3)}


def tidal_leg(ctx, d, steps, n_bin=65536, order=3):
    """Tidal tensors (Sec. 6.4.1) of n_bin binaries on the headline workload:
    measure points (order 3: 8 per binary, plus the centre of mass) appended
    as zero-mass particles, one long-range step over the augmented set, then
    the fit.  d_c = 1e-4; binaries at randomly chosen particles."""
    import torch
    from paper_2006_16560_gb300 import binding as B
    n = len(d["mass"])
    n_bin = min(n_bin, n)
    rng = np.random.default_rng(12)
    cm = torch.from_numpy(d["pos"][rng.choice(n, n_bin, replace=False)]).cuda()
    dc = torch.full((n_bin,), 1e-4, dtype=torch.float64, device="cuda")
    P = B.TIDAL_POINTS[order]
    pts = torch.empty((n_bin, P, 3), dtype=torch.float64, device="cuda")
    T = torch.empty((n_bin, B.TIDAL_ELEMENTS[order]), dtype=torch.float64, device="cuda")
    pos0, mass0 = torch.from_numpy(d["pos"]).cuda(), torch.from_numpy(d["mass"]).cuda()
    m_aug = torch.cat([mass0, torch.zeros(n_bin * (1 + P), dtype=torch.float64, device="cuda")])
    na = n + n_bin * (1 + P)
    acc = torch.empty((na, 3), dtype=torch.float64, device="cuda")
    pot = torch.empty(na, dtype=torch.float64, device="cuda")
    # the augmented set in one preallocated array (nothing is allocated inside
    # the timed steps): the particles, then per binary its centre and points
    p_aug = torch.empty((na, 3), dtype=torch.float64, device="cuda")
    p_aug[:n] = pos0
    meas = p_aug[n:].view(n_bin, 1 + P, 3)
    meas[:, 0] = cm
    holder = [None]

    def step():
        ctx.check(B.pt_tidal_points(ctx.h, order, n_bin, B._ptr(cm), B._ptr(dc), B._ptr(pts)), "points")
        meas[:, 1:] = pts
        if holder[0] is None:
            holder[0] = B.Tree(ctx, p_aug, m_aug, params(B.PT_MIXED))
        else:
            holder[0].rebuild(p_aug, m_aug, params(B.PT_MIXED))
        _, st, _ = holder[0].force(acc, pot)
        a_meas = acc[n:].reshape(n_bin, 1 + P, 3)
        ctx.check(B.pt_tidal_tensor(ctx.h, order, n_bin, B._ptr(a_meas), B._ptr(dc), B._ptr(T)), "fit")
        return st.as_dict()
    for _ in range(3):                     # the tree's build graph is captured on its second build
        step()
    times = []
    for _ in range(max(3, steps)):
        t1, st = _device_ms(step, 1)
        times.append(t1)
    ms = statistics.mean(times)
    fit_ms, _ = _device_ms(lambda: B.pt_tidal_tensor(ctx.h, order, n_bin, B._ptr(acc[n:].reshape(n_bin, 1 + P, 3)),
                                                     B._ptr(dc), B._ptr(T)), 5)
    holder[0].free()
    return {"workload": f"{n_bin} binaries at random particles of the headline set, order {order} "
                        f"({P} points + centre each, d_c = 1e-4), FP32-mixed step over {na} particles",
            "ms_per_step": ms, "ms_p50": float(np.percentile(times, 50)), "ms_max": max(times),
            "fit_ms": fit_ms,
            "interactions_per_step": st["cell_interactions"] + st["pp_interactions"],
            "tensors_per_s": n_bin / (ms * 1e-3)}


def _errors(acc, pot, acc_ref, pot_ref):
    """p50 / p99 / max of the per-particle relative errors |da|/|a| and |dphi|/|phi|."""
    e = np.linalg.norm(acc - acc_ref, axis=1) / np.linalg.norm(acc_ref, axis=1)
    ep = np.abs(pot - pot_ref) / np.abs(pot_ref)
    return {"acc_p50": float(np.percentile(e, 50)), "acc_p99": float(np.percentile(e, 99)),
            "acc_max": float(e.max()), "pot_p50": float(np.percentile(ep, 50)),
            "pot_p99": float(np.percentile(ep, 99)), "pot_max": float(ep.max())}


def _device_set(d, n):
    import torch
    pos = torch.from_numpy(d["pos"]).cuda()
    mass = torch.from_numpy(d["mass"]).cuda()
    cap = 8 * n
    out = (torch.empty((n, 3), dtype=torch.float64, device="cuda"),
           torch.empty((n,), dtype=torch.float64, device="cuda"),
           torch.empty((n + 1,), dtype=torch.int64, device="cuda"),
           torch.empty((cap,), dtype=torch.int32, device="cuda"))
    return pos, mass, out


def c2_10m_leg(ctx, steps, flush):
    """The headline workload at N = 10^7 (Kroupa Plummer, seed 2, same tree
    parameters): mixed steps (build + force) timed like the headline, one
    FP64 step for the mixed-vs-FP64 error.  Returns the record and the mixed
    and FP64 results for the sampled tree-vs-direct comparison."""
    from paper_2006_16560_gb300 import binding as B
    from paper_2006_16560_gb300 import inputs
    n = 10_000_000
    d = inputs.plummer(n, SEED, masses="kroupa")
    pos, mass, out = _device_set(d, n)
    holder = [None]
    run_steps(ctx, holder, pos, mass, params(B.PT_MIXED), out, 2, flush)
    times, st = run_steps(ctx, holder, pos, mass, params(B.PT_MIXED), out, steps, flush)
    mx = (out[0].cpu().numpy().copy(), out[1].cpu().numpy().copy())
    nb_mx = int(st["neighbours"])
    t64, st64 = run_steps(ctx, holder, pos, mass, params(B.PT_FP64), out, 1, flush)
    f64 = (out[0].cpu().numpy().copy(), out[1].cpu().numpy().copy())
    holder[0].free()
    ms = statistics.mean(times)
    inter = st["cell_interactions"] + st["pp_interactions"]
    rec = {"workload": f"Plummer N={n}, Kroupa IMF, seed {SEED}; quadrupole tree theta=0.3, n_leaf=16, "
                       "n_group=64, r_out=0.003, r_in=0.0003; neighbour lists on",
           "value": inter / (ms * 1e-3), "unit": "interactions/s", "particles_per_s": n / (ms * 1e-3),
           "ms_per_step": ms, "latency_ms": {"p50": float(np.percentile(times, 50)),
                                             "p99": float(np.percentile(times, 99))},
           "interactions_per_step": inter, "neighbours": nb_mx,
           "neighbours_fp64": int(st64["neighbours"]),
           "stage_ms": {"build": st["ms_build"], "walk": st["ms_walk"], "force_kernel": st["ms_force"]},
           "fp64_ms_per_step": t64[0],
           "mixed_error_vs_fp64": _errors(mx[0], mx[1], f64[0], f64[1])}
    return rec, d, {"fp64": f64, "mixed": mx}


def n1mkb_leg(ctx, steps, flush):
    """The paper's N1mkb model (Sec. 7.1.1, Table 2): 10^6 stars, all in
    5 x 10^5 primordial binaries of the Kroupa (1995) period distribution
    (Eq. 39; seed 12), r_out,ref = 0.00199039, r_out/r_in = 10, theta 0.3,
    with mass-dependent changeover radii (Eq. 12, factors computed on the
    device).  Mixed and FP64 step times, mixed vs FP64 error, and the fraction
    of binaries closer than their pair radius r_out * max(s_i, s_j) whose
    members are each other's neighbours (every one of them must be)."""
    from paper_2006_16560_gb300 import binding as B
    from paper_2006_16560_gb300 import inputs
    d = inputs.kroupa95_binaries(500_000, 12)
    n = len(d["mass"])
    r_out = 0.199039e-2
    kw = dict(theta=0.3, r_in=0.1 * r_out, r_out=r_out, n_leaf=16, n_group=64, order=2, mass_dependent=1)
    pm, p64 = B.Params(precision=B.PT_MIXED, **kw), B.Params(precision=B.PT_FP64, **kw)
    pos, mass, out = _device_set(d, n)
    holder = [None]
    run_steps(ctx, holder, pos, mass, pm, out, 2, flush)
    times, st = run_steps(ctx, holder, pos, mass, pm, out, steps, flush)
    mx = (out[0].cpu().numpy().copy(), out[1].cpu().numpy().copy())
    off, idx = out[2].cpu().numpy(), out[3][: int(st["neighbours"])].cpu().numpy()
    run_steps(ctx, holder, pos, mass, p64, out, 1, flush)
    t64, st64 = run_steps(ctx, holder, pos, mass, p64, out, 2, flush)
    f64 = (out[0].cpu().numpy(), out[1].cpu().numpy())
    holder[0].free()
    # pairs closer than their pair radius (Eq. 12 factors, with a margin for
    # the device's cube root) must be neighbours of each other
    m = d["mass"]
    sfac = np.cbrt(np.maximum(1.0, m / m.mean()))
    rij = r_out * np.maximum(sfac[0::2], sfac[1::2])
    sep = np.linalg.norm(d["pos"][0::2] - d["pos"][1::2], axis=1)
    must = np.nonzero(sep < 0.999 * rij)[0]
    rows = np.repeat(np.arange(n), np.diff(off))
    have = np.zeros(n, dtype=bool)
    have[rows[idx == (rows ^ 1)]] = True
    ms, ms64 = statistics.mean(times), statistics.mean(t64)
    inter = st["cell_interactions"] + st["pp_interactions"]
    return {"workload": "N1mkb: 5x10^5 Kroupa (1995) primordial binaries (10^6 stars, seed 12), r_out,ref = "
                        "0.00199039, r_in = r_out/10, theta 0.3, n_leaf 16, n_group 64, quadrupole, mass-dependent "
                        "radii (Eq. 12)",
            "value": inter / (ms * 1e-3), "unit": "interactions/s", "ms_per_step": ms,
            "stage_ms": {"build": st["ms_build"], "walk": st["ms_walk"], "force_kernel": st["ms_force"]},
            "fp64_ms_per_step": ms64, "speedup_mixed_vs_fp64": ms64 / ms,
            "interactions_per_step": inter, "pp_changeover_interactions": st["pp_changeover_interactions"],
            "neighbours": int(st["neighbours"]), "neighbours_fp64": int(st64["neighbours"]),
            "binaries_within_pair_radius": int(len(must)),
            "companions_found": float(np.mean(have[2 * must] & have[2 * must + 1])) if len(must) else None,
            "mixed_error_vs_fp64": _errors(mx[0], mx[1], f64[0], f64[1])}


def size_sweep_leg(ctx, steps, flush, sizes=(1 << 14, 1 << 16, 1 << 18, 1 << 22)):
    """The headline workload (Kroupa Plummer, seed 2, the same tree
    parameters, FP32-mixed, neighbour lists on) at other particle counts:
    ms per step and interactions/s, timed like the headline."""
    from paper_2006_16560_gb300 import binding as B
    from paper_2006_16560_gb300 import inputs
    rows = []
    for n in sizes:
        d = inputs.plummer(n, SEED, masses="kroupa")
        pos, mass, out = _device_set(d, n)
        holder = [None]
        run_steps(ctx, holder, pos, mass, params(B.PT_MIXED), out, 2, flush)
        times, st = run_steps(ctx, holder, pos, mass, params(B.PT_MIXED), out, steps, flush)
        holder[0].free()
        ms = statistics.mean(times)
        inter = st["cell_interactions"] + st["pp_interactions"]
        rows.append({"n": n, "ms_per_step": ms, "interactions_per_s": inter / (ms * 1e-3),
                     "particles_per_s": n / (ms * 1e-3), "interactions_per_step": inter,
                     "stage_ms": {"build": st["ms_build"], "walk": st["ms_walk"],
                                  "force_kernel": st["ms_force"]}})
    return {"workload": "Plummer N=2^14..2^22, Kroupa IMF, seed 2; quadrupole tree theta=0.3, n_leaf=16, "
                        "n_group=64, r_out=0.003, r_in=0.0003; FP32-mixed, neighbour lists on",
            "rows": rows}


def binaries_leg(ctx, steps, flush):
    """Precision variant: N = 10^6 with every star in a primordial binary
    (500,000 pairs, a log-uniform in 0.005-50 AU, thermal e; seed 4) on the
    headline tree parameters.  Mixed and FP64 step times, mixed vs FP64
    error, and the fraction of stars whose companion is in their neighbour
    list (every pair is closer than r_in, so all of them must be)."""
    from paper_2006_16560_gb300 import binding as B
    from paper_2006_16560_gb300 import inputs
    d = inputs.plummer_binaries(500_000, 4)
    n = len(d["mass"])
    pos, mass, out = _device_set(d, n)
    holder = [None]
    run_steps(ctx, holder, pos, mass, params(B.PT_MIXED), out, 2, flush)
    times, st = run_steps(ctx, holder, pos, mass, params(B.PT_MIXED), out, steps, flush)
    mx = (out[0].cpu().numpy().copy(), out[1].cpu().numpy().copy())
    off, idx = out[2].cpu().numpy(), out[3][: int(st["neighbours"])].cpu().numpy()
    rows = np.repeat(np.arange(n), np.diff(off))
    found = np.zeros(n, dtype=bool)
    found[rows[idx == (rows ^ 1)]] = True
    run_steps(ctx, holder, pos, mass, params(B.PT_FP64), out, 1, flush)
    t64, st64 = run_steps(ctx, holder, pos, mass, params(B.PT_FP64), out, 2, flush)
    f64 = (out[0].cpu().numpy(), out[1].cpu().numpy())
    holder[0].free()
    ms, ms64 = statistics.mean(times), statistics.mean(t64)
    inter = st["cell_interactions"] + st["pp_interactions"]
    return {"workload": "Plummer centres N=500000 pairs (10^6 stars), Kroupa masses, a log-uniform "
                        "0.005-50 AU, thermal e (seed 4); quadrupole tree theta=0.3, n_leaf=16, n_group=64, "
                        "r_out=0.003, r_in=0.0003",
            "value": inter / (ms * 1e-3), "unit": "interactions/s", "ms_per_step": ms,
            "fp64_ms_per_step": ms64, "speedup_mixed_vs_fp64": ms64 / ms,
            "pp_changeover_interactions": st["pp_changeover_interactions"],
            "interactions_per_step": inter, "neighbours": int(st["neighbours"]),
            "neighbours_fp64": int(st64["neighbours"]),
            "companions_found": float(found.mean()),
            "mixed_error_vs_fp64": _errors(mx[0], mx[1], f64[0], f64[1])}


def tree_vs_direct(d, results, nsample, seed):
    """Tree-vs-direct truncation error: the oracle's direct O(N^2) long-range
    sum (same changeover split, float64) on nsample random targets against
    each GPU result in `results` ({name: (acc, pot)})."""
    import oracle
    n = len(d["mass"])
    tg = np.random.default_rng(seed).choice(n, min(nsample, n), replace=False)
    t0 = time.perf_counter()
    a_d, p_d = oracle.direct_force(d["pos"], d["mass"], 0.0003, 0.003, targets=tg)
    rec = {"targets": int(len(tg)), "direct_s": time.perf_counter() - t0}
    for name, (acc, pot) in results.items():
        rec[name] = _errors(acc[tg], pot[tg], a_d, p_d)
    return rec


def cpu_oracle_sample(pos, mass, nsample, seed=11):
    """Oracle tree on the host cores: full build plus the tree force on
    nsample targets; returns the interactions/s it would sustain on the whole
    set, the seconds spent and the threads used."""
    import oracle
    n = len(mass)
    nsample = min(nsample, n)
    t0 = time.perf_counter()
    T = oracle.Tree(pos, mass, 16, 64)
    t1 = time.perf_counter()
    tg = np.random.default_rng(seed).choice(n, nsample, replace=False)
    _, _, st = T.force(0.3, 0.0003, 0.003, order=2, targets=tg)
    t2 = time.perf_counter()
    inter = st[0] + st[1]
    full_time = (t1 - t0) + (t2 - t1) * n / nsample
    full_inter = inter * n / nsample
    threads = _omp_threads()
    return full_inter / full_time, t2 - t0, threads, inter


def _omp_threads(n=None):
    """The OpenMP thread count of the oracle's runtime (libgomp, loaded with
    the oracle library); with n, sets it and returns the previous count."""
    import ctypes
    g = ctypes.CDLL("libgomp.so.1")
    prev = g.omp_get_max_threads()
    if n is not None:
        g.omp_set_num_threads(int(n))
    return prev


def reference_main(args, rank, world):
    """--impl reference: the CPU oracle as it stands on the host cores."""
    if rank != 0:
        return
    from paper_2006_16560_gb300 import inputs
    n = args.n
    d = inputs.plummer(n, SEED, masses="kroupa")
    ns = args.cpu_sample
    vals, secs = [], []
    for i in range(args.warmup + args.steps):
        v, s, thr, _ = cpu_oracle_sample(d["pos"], d["mass"], ns, seed=11 + i)
        if i >= args.warmup:
            vals.append(v)
            secs.append(s)
    v = statistics.median(vals)
    sample = (f"per step: oracle tree build over all {n} particles + oracle tree force on {ns} random "
              f"targets, extrapolated to all targets")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "interactions/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * statistics.mean(secs), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(n),
            "cpu_baseline": {"value": v, "unit": "interactions/s", "cores": thr, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "interactions/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--particles", "--n", dest="n", type=int, default=N_DEFAULT)
    ap.add_argument("--cpu-sample", type=int, default=262144,
                    help="oracle targets per CPU sample (about 10 s on 16 host cores)")
    ap.add_argument("--no-sweep", action="store_true", help="skip the 2^14..2^22 size sweep")
    ap.add_argument("--no-n1mkb", action="store_true",
                    help="skip the N1mkb leg (Kroupa 1995 binaries, mass-dependent radii)")
    ap.add_argument("--cpu-sample-1core", type=int, default=4096,
                    help="oracle targets of the one-core CPU sample (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--only-mixed", action="store_true", help="skip the FP64, e2e and batch legs (profiling)")
    ap.add_argument("--no-batch", action="store_true", help="skip the 256-cluster batch leg")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--serve-seconds", type=float, default=15.0)
    ap.add_argument("--no-widened", action="store_true",
                    help="skip the orbit-neighbour and tidal-tensor legs")
    ap.add_argument("--no-10m", action="store_true", help="skip the N = 10^7 leg")
    ap.add_argument("--no-binaries", action="store_true", help="skip the primordial-binary leg")
    ap.add_argument("--tvd-sample", type=int, default=10000,
                    help="targets of the direct-sum reference at N = 2^20 (tree-vs-direct error)")
    ap.add_argument("--tvd-sample-10m", type=int, default=1000,
                    help="targets of the direct-sum reference at N = 10^7")
    ap.add_argument("--only-leg", choices=["orbit", "tidal", "batch"], default=None,
                    help="run one widened leg alone on the headline set and print its JSON (profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    rank, world, local = rank_env()
    if args.impl == "reference":
        reference_main(args, rank, world)
        return
    if args.only_leg:
        from paper_2006_16560_gb300 import binding as B
        from paper_2006_16560_gb300 import inputs
        d = inputs.plummer(args.n, SEED, masses="kroupa")
        ctx = B.Context(local)
        if args.only_leg == "batch":
            leg = batch_leg(ctx, args.steps)
        else:
            leg = orbit_leg(ctx, d, args.steps) if args.only_leg == "orbit" else tidal_leg(ctx, d, args.steps)
        print(json.dumps({"leg": args.only_leg, **leg}), flush=True)
        ctx.close()
        return

    import torch
    import torch.distributed as dist
    from paper_2006_16560_gb300 import binding as B
    from paper_2006_16560_gb300 import inputs

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    n = args.n
    d = inputs.plummer(n, SEED, masses="kroupa")
    pos = torch.from_numpy(d["pos"]).cuda()
    mass = torch.from_numpy(d["mass"]).cuda()
    ctx = B.Context(local)
    cap = 8 * n
    out = (torch.empty((n, 3), dtype=torch.float64, device="cuda"),
           torch.empty((n,), dtype=torch.float64, device="cuda"),
           torch.empty((n + 1,), dtype=torch.int64, device="cuda"),
           torch.empty((cap,), dtype=torch.int32, device="cuda"))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MiB > L2
    prm_mx, prm_64 = params(B.PT_MIXED), params(B.PT_FP64)
    holder = [None]

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- mixed precision (the headline) ----
    run_steps(ctx, holder, pos, mass, prm_mx, out, args.warmup, flush)
    barrier()
    with ClockSampler(local) as clk:
        t_wall0 = time.perf_counter()
        times, st = run_steps(ctx, holder, pos, mass, prm_mx, out, args.steps, flush)
        barrier()
        t_wall = time.perf_counter() - t_wall0
    clocks = clk.summary()
    acc_mx = out[0].cpu().numpy().copy()
    pot_mx = out[1].cpu().numpy().copy()
    res_1m = {"mixed": (acc_mx, pot_mx)}
    nb_total = int(st["neighbours"])
    ms_step = statistics.mean(times)
    ms_max = max_over_ranks(ms_step, device="cuda")
    inter = st["cell_interactions"] + st["pp_interactions"]
    value = replica_value(inter, ms_max, world)
    # force kernel alone (CUDA events on the launching stream, inside the library)
    kernel_ms = []
    for _ in range(max(3, min(args.steps, 10))):
        flush.fill_(1.0)
        _, s2 = run_steps(ctx, holder, pos, mass, prm_mx, out, 1)
        kernel_ms.append(s2["ms_force"])
    k_ms = statistics.mean(kernel_ms)
    achieved = flops_of(st, "mixed") / (k_ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32-mixed",
        "data": "synthetic", "config": workload_config(n),
        "particles_per_s": replica_value(n, ms_max, world),
        "latency_ms": {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99)),
                       "wall_per_step": 1000 * t_wall / args.steps},
        "interactions_per_step": inter, "cell_interactions": st["cell_interactions"],
        "pp_interactions": st["pp_interactions"],
        "pp_changeover_interactions": st["pp_changeover_interactions"],
        "groups": st["groups"], "nodes": st["nodes"], "max_walk_stack": st["max_walk_stack"],
        "neighbours": nb_total,
        "stage_ms": {"build": st["ms_build"], "walk": st["ms_walk"], "force_kernel": k_ms,
                     "force_call": st["ms_total"]},
        "gpu_launches": int((st["launches_build"] + st["launches_force"]) * args.steps),
        "clocks": clocks,
    }
    sms = device_sm_count(local)
    max_mhz = clocks.get("sm_max_mhz") or GB300_MAX_MHZ
    peak = fp32_peak(sms, max_mhz)
    line["roofline"] = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                        "unit": "TFLOP/s", "frac": achieved / peak,
                        "traffic": FORCE_MIXED_DRAM_BYTES,
                        "kernel": "k_force_mixed<2,true>",
                        "flops_per_interaction": {"cell_quadrupole": FLOPS[("mixed", "cell", 2)],
                                                  "pp_changeover": FLOPS[("mixed", "pp", None)],
                                                  "pp_newton": FLOPS[("mixed", "pp_newton", None)]},
                        "peak_note": f"FP32 CUDA-core peak at the {max_mhz:.0f} MHz maximum SM clock "
                                     f"({sms} SMs x 128 lanes x 2 flop; no tensor cores: not a contraction)"}
    if clocks.get("sm_mhz"):
        line["roofline"]["frac_at_measured_clock"] = achieved / fp32_peak(sms, clocks["sm_mhz"])
    rc, probe = B.pt_probe_fp32_peak(ctx.h)
    if rc == B.PT_OK and probe > 0:
        line["roofline"]["fp32_fma_probe_tflops"] = probe
        line["roofline"]["frac_of_probe"] = achieved / (probe * 1e12)

    if not args.only_mixed:
        # ---- float64 path on the same workload ----
        run_steps(ctx, holder, pos, mass, prm_64, out, 2, flush)
        t64, st64 = run_steps(ctx, holder, pos, mass, prm_64, out, max(3, args.steps // 2), flush)
        acc64 = out[0].cpu().numpy()
        pot64 = out[1].cpu().numpy()
        res_1m["fp64"] = (acc64, pot64)
        ms64 = statistics.mean(t64)
        inter64 = st64["cell_interactions"] + st64["pp_interactions"]
        e = np.linalg.norm(acc_mx - acc64, axis=1) / np.linalg.norm(acc64, axis=1)
        ep = np.abs(pot_mx - pot64) / np.abs(pot64)
        line["fp64"] = {"value": world * inter64 / (ms64 * 1e-3), "unit": "interactions/s",
                        "ms_per_step": ms64, "force_kernel_ms": st64["ms_force"],
                        "latency_ms": {"p50": float(np.percentile(t64, 50)),
                                       "p99": float(np.percentile(t64, 99))}}
        line["speedup_mixed_vs_fp64"] = ms64 / ms_step
        line["mixed_error_vs_fp64"] = {"acc_p50": float(np.percentile(e, 50)),
                                       "acc_p99": float(np.percentile(e, 99)),
                                       "acc_max": float(e.max()),
                                       "pot_p99": float(np.percentile(ep, 99))}
    if not args.no_e2e and not args.only_mixed:
        # ---- end to end through the C ABI with pinned host buffers ----
        hp = torch.from_numpy(d["pos"]).pin_memory()
        hm = torch.from_numpy(d["mass"]).pin_memory()
        ha = torch.empty((n, 3), dtype=torch.float64).pin_memory()
        hphi = torch.empty((n,), dtype=torch.float64).pin_memory()
        hoff = torch.empty((n + 1,), dtype=torch.int64).pin_memory()
        hidx = torch.empty((cap,), dtype=torch.int32).pin_memory()
        hbuf = (ha.numpy(), hphi.numpy(), hoff.numpy(), hidx.numpy())
        tree_h = B.Tree(ctx, hp.numpy(), hm.numpy(), prm_mx)
        tree_h.force(*hbuf, cap)
        for _ in range(args.warmup):          # the build's graph is captured on its first repeat
            tree_h.rebuild(hp.numpy(), hm.numpy(), prm_mx)
            tree_h.force(*hbuf, cap)
        te = []
        for _ in range(max(3, args.steps // 2)):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tree_h.rebuild(hp.numpy(), hm.numpy(), prm_mx)
            tot, ste, _ = tree_h.force(*hbuf, cap)
            te.append(time.perf_counter() - t0)
        inter_e = ste.cell_interactions + ste.pp_interactions
        line["e2e"] = {"value": world * inter_e / statistics.mean(te), "unit": "interactions/s",
                       "h2d_bytes_per_step": 32 * n,
                       "d2h_bytes_per_step": 32 * n + 8 * (n + 1) + 4 * int(tot),
                       "ms_per_step": 1000 * statistics.mean(te)}
        tree_h.free()
    if holder[0] is not None:
        holder[0].free()
    if not args.no_batch and not args.only_mixed:
        line["batch"] = batch_leg(ctx, max(3, args.steps // 2))
    if not args.no_serve and not args.only_mixed and rank == 0:
        line["serving"] = serve_leg(ctx, args.serve_seconds)
    if not args.no_widened and not args.only_mixed:
        line["orbit_neighbours"] = orbit_leg(ctx, d, args.steps)
        line["tidal"] = tidal_leg(ctx, d, max(3, args.steps // 2))
    big = None
    if not args.no_10m and not args.only_mixed:
        line["c2_10m"], d10, big = c2_10m_leg(ctx, max(3, args.steps // 4), flush)
    if not args.no_binaries and not args.only_mixed:
        line["binaries_1m"] = binaries_leg(ctx, max(3, args.steps // 4), flush)
    if not args.no_n1mkb and not args.only_mixed:
        line["n1mkb"] = n1mkb_leg(ctx, max(3, args.steps // 4), flush)
    if not args.no_sweep and not args.only_mixed:
        line["size_sweep"] = size_sweep_leg(ctx, max(3, args.steps // 2), flush)
    if rank == 0 and not args.no_cpu_baseline:
        # CPU oracle on the host cores: the direct-sum reference of the
        # tree-vs-direct error on sampled targets, then the timed baseline
        tvd = {"n_1m": tree_vs_direct(d, res_1m, args.tvd_sample, 21)}
        if big is not None:
            tvd["n_10m"] = tree_vs_direct(d10, big, args.tvd_sample_10m, 22)
            del big, d10
        line["tree_vs_direct"] = tvd
        v, secs, thr, si = cpu_oracle_sample(d["pos"], d["mass"], args.cpu_sample)
        line["cpu_baseline"] = {"value": v, "unit": "interactions/s", "cores": thr, "kind": "oracle",
                                "sample": f"oracle tree build over all {n} particles + oracle tree force "
                                          f"on {args.cpu_sample} random targets ({si} interactions, "
                                          f"{secs:.1f} s), extrapolated to all targets"}
        if args.cpu_sample_1core > 0:
            prev = _omp_threads(1)
            v1, secs1, _, si1 = cpu_oracle_sample(d["pos"], d["mass"], args.cpu_sample_1core, seed=12)
            _omp_threads(prev)
            line["cpu_baseline"]["one_core"] = {
                "value": v1, "unit": "interactions/s",
                "sample": f"the same on one core: {args.cpu_sample_1core} targets ({si1} interactions, "
                          f"{secs1:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
