"""Python handle on the native serving loop (pt_server_* in include/pt.h) and
a seeded Poisson load generator for it.

The server itself (resident state, admission by HBM budget, continuous
batching on a worker thread) is C++ inside libpt.so; this module only
marshals arguments and drives requests.
"""
from __future__ import annotations

import ctypes as C
import threading
import time

import numpy as np

from . import binding as B


class pt_server_config(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_batch_particles", C.c_int64),
                ("max_sims", C.c_int), ("neighbours", C.c_int), ("params", B.pt_params),
                ("workers", C.c_int), ("large_sim_particles", C.c_int64)]


class pt_request_info(C.Structure):
    _fields_ = [("ticket", C.c_int64), ("sim", C.c_int), ("status", C.c_int),
                ("t_submit", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double),
                ("batch_size", C.c_int), ("batch_particles", C.c_int64)]


class pt_server_stats_t(C.Structure):
    _fields_ = [("batches", C.c_int64), ("requests", C.c_int64), ("particles", C.c_int64),
                ("interactions", C.c_int64), ("busy_s", C.c_double), ("uptime_s", C.c_double),
                ("resident_bytes", C.c_int64), ("max_batch_particles", C.c_int64), ("queued", C.c_int64)]


_sigs_done = False


def _lib():
    global _sigs_done
    L = B.lib()
    if not _sigs_done:
        P, I, I64, D = C.c_void_p, C.c_int, C.c_int64, C.c_double
        for name, res, args in [
            ("pt_server_create", I, [P, C.POINTER(pt_server_config), C.POINTER(P)]),
            ("pt_server_destroy", I, [P]),
            ("pt_server_add_sim", I, [P, I64, P, P, P, D, D, C.POINTER(I)]),
            ("pt_server_remove_sim", I, [P, I]),
            ("pt_server_submit", I, [P, I, D, D, C.POINTER(I64)]),
            ("pt_server_wait", I, [P, I64, D, C.POINTER(pt_request_info)]),
            ("pt_server_read_sim", I, [P, I, P, P, P, P]),
            ("pt_server_stats", I, [P, C.POINTER(pt_server_stats_t)]),
            ("pt_server_last_error", C.c_char_p, [P]),
        ]:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _sigs_done = True
    return L


class Server:
    """Resident-state serving loop for long-range kick requests."""

    def __init__(self, ctx: B.Context, params: B.Params, hbm_budget_bytes: float = 150e9,
                 max_sims: int = 64, neighbours: bool = True, max_batch_particles: int = 0,
                 workers: int = 0, large_sim_particles: int = 0):
        self.ctx = ctx
        cfg = pt_server_config(int(hbm_budget_bytes), int(max_batch_particles), int(max_sims),
                               1 if neighbours else 0, params.c(), int(workers), int(large_sim_particles))
        h = C.c_void_p()
        rc = _lib().pt_server_create(ctx.h, C.byref(cfg), C.byref(h))
        if rc != B.PT_OK:
            raise B.PTError(rc, "pt_server_create")
        self.h = h
        self.n = {}

    def add_sim(self, pos, vel, mass, r_in: float, r_out: float) -> int:
        sid = C.c_int(-1)
        rc = _lib().pt_server_add_sim(self.h, int(mass.shape[0]), B._ptr(pos), B._ptr(vel), B._ptr(mass),
                                      float(r_in), float(r_out), C.byref(sid))
        if rc != B.PT_OK:
            raise B.PTError(rc, "pt_server_add_sim")
        self.n[sid.value] = int(mass.shape[0])
        return sid.value

    def try_add_sim(self, pos, vel, mass, r_in, r_out):
        sid = C.c_int(-1)
        rc = _lib().pt_server_add_sim(self.h, int(mass.shape[0]), B._ptr(pos), B._ptr(vel), B._ptr(mass),
                                      float(r_in), float(r_out), C.byref(sid))
        if rc == B.PT_OK:
            self.n[sid.value] = int(mass.shape[0])
        return rc, sid.value

    def remove_sim(self, sid: int):
        rc = _lib().pt_server_remove_sim(self.h, sid)
        if rc != B.PT_OK:
            raise B.PTError(rc, "pt_server_remove_sim")
        self.n.pop(sid, None)

    def submit(self, sid: int, dt_drift: float, dt_kick: float) -> int:
        t = C.c_int64(0)
        rc = _lib().pt_server_submit(self.h, sid, float(dt_drift), float(dt_kick), C.byref(t))
        if rc != B.PT_OK:
            raise B.PTError(rc, "pt_server_submit")
        return t.value

    def wait(self, ticket: int, timeout: float = -1.0) -> dict:
        info = pt_request_info()
        rc = _lib().pt_server_wait(self.h, ticket, float(timeout), C.byref(info))
        if rc != B.PT_OK:
            raise B.PTError(rc, "pt_server_wait: " + self.last_error())
        return {k: getattr(info, k) for k, _ in info._fields_}

    def read(self, sid: int):
        n = self.n[sid]
        pos, vel, acc = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
        pot = np.zeros(n)
        rc = _lib().pt_server_read_sim(self.h, sid, pos.ctypes.data, vel.ctypes.data, acc.ctypes.data,
                                       pot.ctypes.data)
        if rc != B.PT_OK:
            raise B.PTError(rc, "pt_server_read_sim")
        return pos, vel, acc, pot

    def last_error(self) -> str:
        return (_lib().pt_server_last_error(self.h) or b"").decode()

    def stats(self) -> dict:
        s = pt_server_stats_t()
        _lib().pt_server_stats(self.h, C.byref(s))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close(self):
        if getattr(self, "h", None):
            _lib().pt_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def poisson_load(server: Server, sims: list[int], rate: float, duration_s: float, seed: int,
                 dt_drift: float = 1e-4, dt_kick: float = 1e-4, timeout: float = -1.0) -> dict:
    """Submit requests at Poisson arrival times (rate per second) for
    duration_s, each on a uniformly chosen simulation; wait for all of them.
    Returns latency percentiles (submit -> done, server clock), throughput and
    the batch sizes seen."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=int(rate * duration_s * 2) + 16)
    arrivals = np.cumsum(gaps)
    arrivals = arrivals[arrivals < duration_s]
    choice = rng.integers(0, len(sims), size=len(arrivals))
    tickets = []
    lock = threading.Lock()

    def submitter():
        t0 = time.perf_counter()
        for a, c in zip(arrivals, choice):
            delay = a - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tk = server.submit(sims[c], dt_drift, dt_kick)
            with lock:
                tickets.append(tk)

    th = threading.Thread(target=submitter)
    s0 = server.stats()
    t_start = time.perf_counter()
    th.start()
    th.join()
    infos = [server.wait(t, timeout) for t in tickets]
    wall = time.perf_counter() - t_start
    s1 = server.stats()
    lat = np.array([i["t_done"] - i["t_submit"] for i in infos]) * 1e3
    qwait = np.array([i["t_start"] - i["t_submit"] for i in infos]) * 1e3
    bsz = np.array([i["batch_size"] for i in infos])
    served_particles = sum(server.n[i["sim"]] for i in infos)
    inter = s1["interactions"] - s0["interactions"]
    busy = s1["busy_s"] - s0["busy_s"]
    return {
        "requests": len(infos), "offered_rate": rate, "duration_s": duration_s, "wall_s": wall,
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "mean": float(lat.mean()), "max": float(lat.max())},
        "queue_wait_ms": {"p50": float(np.percentile(qwait, 50)), "p99": float(np.percentile(qwait, 99))},
        "throughput_req_per_s": len(infos) / wall,
        "particles_per_s": served_particles / wall,
        "interactions_per_s_busy": inter / busy if busy > 0 else None,
        "device_busy_fraction": busy / wall,
        "batches": s1["batches"] - s0["batches"],
        "batch_size": {"mean": float(bsz.mean()), "max": int(bsz.max())},
        "errors": int(sum(1 for i in infos if i["status"] not in (B.PT_OK, B.PT_ERR_CAPACITY))),
    }
