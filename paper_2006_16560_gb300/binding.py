"""ctypes binding of libpt.so (include/pt.h).

The C functions keep their names (``pt_ctx_create``, ``pt_tree_build``,
``pt_longrange_force``, ``pt_batch_longrange_force``, ...).  This module only
marshals arguments: every step of the force pipeline runs in the library's
CUDA kernels.  Buffers may be CUDA torch tensors (device pointers) or numpy
arrays (host pointers); the library stages host buffers itself.

There is no fallback: if libpt.so cannot be built or loaded, or no GPU is
usable, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import threading
from dataclasses import dataclass

import numpy as np

from . import build_lib

PT_OK, PT_ERR_ARG, PT_ERR_OOM, PT_ERR_CAPACITY, PT_ERR_TIMEOUT, PT_ERR_CUDA, PT_ERR_INTERNAL = range(7)
PT_FP64, PT_MIXED = 0, 1
PT_BATCH_GRAPH = 1
ERR_NAMES = {0: "PT_OK", 1: "PT_ERR_ARG", 2: "PT_ERR_OOM", 3: "PT_ERR_CAPACITY",
             4: "PT_ERR_TIMEOUT", 5: "PT_ERR_CUDA", 6: "PT_ERR_INTERNAL"}


class pt_params(C.Structure):
    _fields_ = [("theta", C.c_double), ("r_in", C.c_double), ("r_out", C.c_double),
                ("G", C.c_double), ("n_leaf", C.c_int), ("n_group", C.c_int),
                ("order", C.c_int), ("precision", C.c_int), ("mass_dependent", C.c_int)]


class pt_stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("nodes", C.c_int64), ("groups", C.c_int64),
                ("max_level", C.c_int64), ("cell_list_total", C.c_int64),
                ("pp_list_total", C.c_int64), ("cell_interactions", C.c_int64),
                ("pp_interactions", C.c_int64), ("neighbours", C.c_int64),
                ("energy", C.c_double), ("momentum", C.c_double * 3),
                ("ms_build", C.c_double), ("ms_walk", C.c_double), ("ms_force", C.c_double),
                ("ms_total", C.c_double), ("pp_changeover_interactions", C.c_int64),
                ("max_walk_stack", C.c_int64), ("launches_build", C.c_int64),
                ("launches_force", C.c_int64)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "momentum"}
        d["momentum"] = list(self.momentum)
        return d


class pt_cluster_desc(C.Structure):
    _fields_ = [("n", C.c_int64), ("pos", C.c_void_p), ("mass", C.c_void_p),
                ("r_in", C.c_double), ("r_out", C.c_double), ("acc", C.c_void_p),
                ("pot", C.c_void_p), ("nb_offsets", C.c_void_p), ("nb_idx", C.c_void_p),
                ("nb_capacity", C.c_int64), ("nb_total", C.c_int64), ("radius_scale", C.c_void_p)]


class pt_orbit_params(C.Structure):
    _fields_ = [("dt", C.c_double), ("C_r", C.c_double), ("C_v", C.c_double), ("mode", C.c_int)]


PT_ORBIT_ROUT, PT_ORBIT_RNB, PT_ORBIT_CANDIDATES = 0, 1, 2

_lib = None
_lock = threading.Lock()


def lib():
    """Load libpt.so, building it first if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            path = build_lib.build()
            L = C.CDLL(path)
            P, I64, I = C.c_void_p, C.c_int64, C.c_int
            sigs = {
                "pt_abi_version": (I, []),
                "pt_ctx_create": (I, [C.POINTER(P), I, P]),
                "pt_ctx_destroy": (I, [P]),
                "pt_last_error": (C.c_char_p, [P]),
                "pt_tree_build": (I, [P, I64, P, P, C.POINTER(pt_params), C.POINTER(P)]),
                "pt_tree_build_scaled": (I, [P, I64, P, P, P, C.POINTER(pt_params), C.POINTER(P)]),
                "pt_longrange_force": (I, [P, P, P, P, P, P, I64, C.POINTER(I64), C.POINTER(pt_stats)]),
                "pt_tree_free": (I, [P]),
                "pt_batch_longrange_force": (I, [P, I, C.POINTER(pt_cluster_desc), C.POINTER(pt_params), I,
                                                 C.POINTER(pt_stats)]),
                "pt_autotune": (I, [P, I, C.POINTER(pt_cluster_desc), C.POINTER(pt_params), P, I, P, I, I,
                                    C.POINTER(pt_params), C.POINTER(C.c_double)]),
                "pt_tree_info": (I, [P, P, P]),
                "pt_tree_keys": (I, [P, P, P]),
                "pt_tree_nodes": (I, [P, P, P, P]),
                "pt_tree_groups": (I, [P, P]),
                "pt_tree_lists": (I, [P, P, P, P, P]),
                "pt_orbit_neighbours": (I, [P, P, C.POINTER(pt_orbit_params), P, P, I64, C.POINTER(I64),
                                            C.POINTER(I64), P]),
                "pt_probe_fp32_peak": (I, [P, C.POINTER(C.c_double)]),
                "pt_tidal_points": (I, [P, I, I64, P, P, P]),
                "pt_tidal_tensor": (I, [P, I, I64, P, P, P]),
                "pt_tidal_eval": (I, [P, I, I64, P, P, I64, P, P, P]),
            }
            for name, (res, args) in sigs.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


# ---- the C entry points under their own names ------------------------------

def pt_ctx_create(device: int = 0, stream: int | None = None):
    h = C.c_void_p()
    rc = lib().pt_ctx_create(C.byref(h), device, stream)
    if rc != PT_OK:
        raise PTError(rc, "pt_ctx_create failed (is a CUDA device available?)")
    return h


def pt_ctx_destroy(ctx) -> int:
    return lib().pt_ctx_destroy(ctx)


def pt_last_error(ctx) -> str:
    s = lib().pt_last_error(ctx)
    return s.decode() if s else ""


def pt_tree_build(ctx, n, pos_ptr, mass_ptr, params: pt_params, tree=None):
    h = tree if tree is not None else C.c_void_p()
    rc = lib().pt_tree_build(ctx, n, pos_ptr, mass_ptr, C.byref(params), C.byref(h))
    return rc, h


def pt_tree_build_scaled(ctx, n, pos_ptr, mass_ptr, scale_ptr, params: pt_params, tree=None):
    h = tree if tree is not None else C.c_void_p()
    rc = lib().pt_tree_build_scaled(ctx, n, pos_ptr, mass_ptr, scale_ptr, C.byref(params), C.byref(h))
    return rc, h


def pt_longrange_force(ctx, tree, acc_ptr, pot_ptr, nb_off_ptr, nb_idx_ptr, nb_capacity):
    tot = C.c_int64(0)
    st = pt_stats()
    rc = lib().pt_longrange_force(ctx, tree, acc_ptr, pot_ptr, nb_off_ptr, nb_idx_ptr,
                                  nb_capacity, C.byref(tot), C.byref(st))
    return rc, tot.value, st


def pt_tree_free(tree) -> int:
    return lib().pt_tree_free(tree)


def pt_batch_longrange_force(ctx, descs, params: pt_params, flags: int = 0):
    arr = (pt_cluster_desc * len(descs))(*descs)
    st = pt_stats()
    rc = lib().pt_batch_longrange_force(ctx, len(descs), arr, C.byref(params), flags, C.byref(st))
    return rc, arr, st


def pt_autotune(ctx, descs, base: pt_params, leafs=None, groups=None, reps: int = 2):
    arr = (pt_cluster_desc * len(descs))(*descs)
    la = (C.c_int * len(leafs))(*leafs) if leafs else None
    ga = (C.c_int * len(groups))(*groups) if groups else None
    best = pt_params()
    ms = C.c_double(0.0)
    rc = lib().pt_autotune(ctx, len(descs), arr, C.byref(base), la, len(leafs) if leafs else 0,
                           ga, len(groups) if groups else 0, reps, C.byref(best), C.byref(ms))
    return rc, best, ms.value


def pt_orbit_neighbours(tree, vel_ptr, op: pt_orbit_params, nb_off_ptr, nb_idx_ptr, nb_capacity,
                        rnb_ptr=None):
    tot, cand = C.c_int64(0), C.c_int64(0)
    rc = lib().pt_orbit_neighbours(tree, vel_ptr, C.byref(op), nb_off_ptr, nb_idx_ptr, nb_capacity,
                                   C.byref(tot), C.byref(cand), rnb_ptr)
    return rc, tot.value, cand.value


def pt_probe_fp32_peak(ctx):
    """(status, measured float32 FMA throughput in TFLOP/s)."""
    v = C.c_double(0.0)
    rc = lib().pt_probe_fp32_peak(ctx, C.byref(v))
    return rc, v.value


def pt_tidal_points(ctx, order, n, r_cm_ptr, d_c_ptr, points_ptr) -> int:
    return lib().pt_tidal_points(ctx, order, n, r_cm_ptr, d_c_ptr, points_ptr)


def pt_tidal_tensor(ctx, order, n, acc_ptr, d_c_ptr, T_ptr) -> int:
    return lib().pt_tidal_tensor(ctx, order, n, acc_ptr, d_c_ptr, T_ptr)


def pt_tidal_eval(ctx, order, n_query, owner_ptr, T_ptr, n_binaries, acc_cm_ptr, rel_ptr, out_ptr) -> int:
    return lib().pt_tidal_eval(ctx, order, n_query, owner_ptr, T_ptr, n_binaries, acc_cm_ptr, rel_ptr,
                               out_ptr)


class PTError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


# ---- thin object wrappers ---------------------------------------------------

def _ptr(x):
    """Device pointer of a CUDA tensor or host pointer of a numpy array."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)}")


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # pragma: no cover
        pass
    return None


@dataclass
class Params:
    theta: float = 0.5
    r_in: float = 0.005
    r_out: float = 0.05
    G: float = 1.0
    n_leaf: int = 8
    n_group: int = 64
    order: int = 2
    precision: int = PT_FP64
    mass_dependent: int = 0

    def c(self) -> pt_params:
        return pt_params(self.theta, self.r_in, self.r_out, self.G, self.n_leaf, self.n_group,
                         self.order, self.precision, self.mass_dependent)


class Context:
    """A library context bound to one device and one CUDA stream."""

    def __init__(self, device: int = 0, stream: int | None = None):
        if stream is None:
            stream = _current_stream()
        self.h = pt_ctx_create(device, stream)

    def check(self, rc: int, what: str):
        if rc != PT_OK:
            raise PTError(rc, f"{what}: {pt_last_error(self.h)}")

    def close(self):
        if getattr(self, "h", None):
            pt_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Tree:
    """A built tree (pt_tree) over one particle set."""

    def __init__(self, ctx: Context, pos, mass, params: Params, scale=None):
        self.ctx = ctx
        self.n = int(mass.shape[0])
        self.params = params
        self._cp = params.c()
        self._scale = scale
        rc, self.h = pt_tree_build_scaled(ctx.h, self.n, _ptr(pos), _ptr(mass), _ptr(scale), self._cp)
        ctx.check(rc, "pt_tree_build")

    def rebuild(self, pos, mass, params: Params | None = None, scale=None):
        if params is not None:
            self.params = params
            self._cp = params.c()
        self.n = int(mass.shape[0])
        self._scale = scale
        rc, self.h = pt_tree_build_scaled(self.ctx.h, self.n, _ptr(pos), _ptr(mass), _ptr(scale),
                                          self._cp, self.h)
        self.ctx.check(rc, "pt_tree_build")

    def force(self, acc, pot, nb_offsets=None, nb_idx=None, nb_capacity: int = 0,
              allow_capacity_error: bool = False):
        rc, total, st = pt_longrange_force(self.ctx.h, self.h, _ptr(acc), _ptr(pot), _ptr(nb_offsets),
                                           _ptr(nb_idx), nb_capacity)
        if rc == PT_ERR_CAPACITY and allow_capacity_error:
            return total, st, rc
        self.ctx.check(rc, "pt_longrange_force")
        return total, st, rc

    def orbit_neighbours(self, vel, dt: float, C_r: float = 3.0, C_v: float = 1.5,
                         mode: int = PT_ORBIT_ROUT, nb_capacity: int | None = None, r_nb=None):
        """Orbit-dependent neighbour lists (Sec. 6.3.1, Eq. 24) for velocities
        ``vel`` (n, 3); returns (nb_offsets, nb_idx, n_candidates) on the side
        (CUDA tensor or numpy) of ``vel``, growing the capacity as needed."""
        op = pt_orbit_params(dt, C_r, C_v, mode)
        cap = nb_capacity if nb_capacity is not None else max(8 * self.n, 1024)
        for _ in range(2):
            off = _empty_like(vel, (self.n + 1,), np.int64)
            idx = _empty_like(vel, (max(cap, 1),), np.int32)
            rc, total, cand = pt_orbit_neighbours(self.h, _ptr(vel), op, _ptr(off), _ptr(idx), cap,
                                                  _ptr(r_nb))
            if rc == PT_ERR_CAPACITY:
                cap = total
                continue
            self.ctx.check(rc, "pt_orbit_neighbours")
            return off, idx[:total], cand
        self.ctx.check(rc, "pt_orbit_neighbours")

    # introspection (host numpy arrays)
    def info(self):
        info = np.zeros(5, dtype=np.int64)
        box = np.zeros(5)
        self.ctx.check(lib().pt_tree_info(self.h, info.ctypes.data, box.ctypes.data), "pt_tree_info")
        return info, box

    def keys(self):
        k = np.zeros(self.n, dtype=np.uint64)
        p = np.zeros(self.n, dtype=np.uint32)
        self.ctx.check(lib().pt_tree_keys(self.h, k.ctypes.data, p.ctypes.data), "pt_tree_keys")
        return k, p

    def nodes(self) -> dict:
        info, _ = self.info()
        nn = int(info[1])
        ints = np.zeros((nn, 8), dtype=np.int64)
        q = np.zeros((nn, 6), dtype=np.uint32)
        mom = np.zeros((nn, 10))
        self.ctx.check(lib().pt_tree_nodes(self.h, ints.ctypes.data, q.ctypes.data, mom.ctypes.data),
                       "pt_tree_nodes")
        return {"begin": ints[:, 0], "count": ints[:, 1], "level": ints[:, 2], "leaf": ints[:, 3],
                "first_child": ints[:, 4], "nchild": ints[:, 5], "qmin": q[:, :3], "qmax": q[:, 3:],
                "mass": mom[:, 0], "com": mom[:, 1:4], "quad": mom[:, 4:10]}

    def groups(self) -> dict:
        info, _ = self.info()
        ng = int(info[2])
        g = np.zeros((ng, 8), dtype=np.int64)
        self.ctx.check(lib().pt_tree_groups(self.h, g.ctypes.data), "pt_tree_groups")
        return {"begin": g[:, 0], "count": g[:, 1], "qmin": g[:, 2:5], "qmax": g[:, 5:8]}

    def lists(self, ncell_total: int, npp_total: int):
        info, _ = self.info()
        ng = int(info[2])
        co = np.zeros(ng + 1, dtype=np.int64)
        po = np.zeros(ng + 1, dtype=np.int64)
        cells = np.zeros(max(ncell_total, 1), dtype=np.uint32)
        pp = np.zeros(max(npp_total, 1), dtype=np.uint32)
        self.ctx.check(lib().pt_tree_lists(self.h, co.ctypes.data, cells.ctypes.data, po.ctypes.data,
                                           pp.ctypes.data), "pt_tree_lists")
        return co, cells[:ncell_total], po, pp[:npp_total]

    def free(self):
        if getattr(self, "h", None):
            pt_tree_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Batch:
    """Device buffers and descriptors for pt_batch_longrange_force over many sets.

    ``sets`` is a list of dicts with float64 CUDA tensors ``pos`` (n, 3) and
    ``mass`` (n,) and floats ``r_in``, ``r_out``.  Outputs live in
    ``self.acc[k]``, ``self.pot[k]``, ``self.nb_off[k]``, ``self.nb_idx[k]``.
    """

    def __init__(self, sets, neighbours: bool = True, nb_factor: int = 8):
        import torch
        self.sets = sets
        self.acc, self.pot, self.nb_off, self.nb_idx, self.descs = [], [], [], [], []
        for st in sets:
            n = int(st["mass"].shape[0])
            dev = st["pos"].device
            self.acc.append(torch.empty((n, 3), dtype=torch.float64, device=dev))
            self.pot.append(torch.empty((n,), dtype=torch.float64, device=dev))
            cap = nb_factor * n + 64
            self.nb_off.append(torch.empty((n + 1,), dtype=torch.int64, device=dev) if neighbours else None)
            self.nb_idx.append(torch.empty((cap,), dtype=torch.int32, device=dev) if neighbours else None)
            d = pt_cluster_desc()
            d.n = n
            d.pos, d.mass = _ptr(st["pos"]), _ptr(st["mass"])
            d.r_in, d.r_out = float(st["r_in"]), float(st["r_out"])
            d.acc, d.pot = _ptr(self.acc[-1]), _ptr(self.pot[-1])
            d.nb_offsets = _ptr(self.nb_off[-1])
            d.nb_idx = _ptr(self.nb_idx[-1])
            d.nb_capacity = cap if neighbours else 0
            self.descs.append(d)
        self.arr = (pt_cluster_desc * len(self.descs))(*self.descs)

    def run(self, ctx: Context, params: Params, graph: bool = False):
        st = pt_stats()
        rc = lib().pt_batch_longrange_force(ctx.h, len(self.descs), self.arr, C.byref(params.c()),
                                            PT_BATCH_GRAPH if graph else 0, C.byref(st))
        ctx.check(rc, "pt_batch_longrange_force")
        return st.as_dict()

    def autotune(self, ctx: Context, params: Params, leafs=None, groups=None, reps: int = 2):
        la = (C.c_int * len(leafs))(*leafs) if leafs else None
        ga = (C.c_int * len(groups))(*groups) if groups else None
        best = pt_params()
        ms = C.c_double(0.0)
        rc = lib().pt_autotune(ctx.h, len(self.descs), self.arr, C.byref(params.c()), la,
                               len(leafs) if leafs else 0, ga, len(groups) if groups else 0, reps,
                               C.byref(best), C.byref(ms))
        ctx.check(rc, "pt_autotune")
        out = Params(**params.__dict__)
        out.n_leaf, out.n_group = best.n_leaf, best.n_group
        return out, ms.value


def longrange_force(ctx: Context, pos, mass, params: Params, neighbours: bool = True,
                    nb_capacity: int | None = None):
    """One-shot build + force on CUDA tensors; returns (acc, pot, nb_off, nb_idx, stats).

    ``pos`` (n, 3) and ``mass`` (n,) are float64 CUDA tensors; the outputs are
    float64 / int64 / int32 CUDA tensors in the input order.
    """
    import torch
    n = int(mass.shape[0])
    dev = pos.device
    t = Tree(ctx, pos, mass, params)
    acc = torch.empty((n, 3), dtype=torch.float64, device=dev)
    pot = torch.empty((n,), dtype=torch.float64, device=dev)
    nb_off = nb_idx = None
    cap = 0
    if neighbours:
        cap = nb_capacity if nb_capacity is not None else max(4 * n, 1024)
        nb_off = torch.empty((n + 1,), dtype=torch.int64, device=dev)
        nb_idx = torch.empty((cap,), dtype=torch.int32, device=dev)
    total, st, rc = t.force(acc, pot, nb_off, nb_idx, cap, allow_capacity_error=True)
    if rc == PT_ERR_CAPACITY:
        nb_idx = torch.empty((total,), dtype=torch.int32, device=dev)
        total, st, rc = t.force(acc, pot, nb_off, nb_idx, total)
    t.free()
    if neighbours:
        nb_idx = nb_idx[:total]
    return acc, pot, nb_off, nb_idx, st.as_dict()


# ---- tidal tensor of a binary's perturbation (Sec. 6.4.1) -----------------

TIDAL_POINTS = {2: 4, 3: 8}
TIDAL_ELEMENTS = {2: 6, 3: 16}


def _empty_like(x, shape, dtype):
    """Uninitialised array on the same side (CUDA tensor or numpy) as ``x``."""
    if isinstance(x, np.ndarray):
        return np.empty(shape, dtype=dtype)
    import torch
    return torch.empty(shape, dtype=getattr(torch, np.dtype(dtype).name), device=x.device)


def tidal_points(ctx: Context, order: int, r_cm, d_c):
    """(n, P, 3) measure points of n binaries (centres ``r_cm`` (n, 3), scales ``d_c`` (n,))."""
    n = int(r_cm.shape[0])
    out = _empty_like(r_cm, (n, TIDAL_POINTS.get(order, 0), 3), np.float64)
    ctx.check(pt_tidal_points(ctx.h, order, n, _ptr(r_cm), _ptr(d_c), _ptr(out)), "pt_tidal_points")
    return out


def tidal_tensor(ctx: Context, order: int, acc, d_c):
    """(n, E) elements from ``acc`` (n, 1 + P, 3): centre of mass first, then the points."""
    n = int(acc.shape[0])
    out = _empty_like(acc, (n, TIDAL_ELEMENTS.get(order, 0)), np.float64)
    ctx.check(pt_tidal_tensor(ctx.h, order, n, _ptr(acc), _ptr(d_c), _ptr(out)), "pt_tidal_tensor")
    return out


def tidal_eval(ctx: Context, order: int, owner, T, acc_cm, rel):
    """(n_query, 3) accelerations acc_cm[owner] + expansion of T[owner] at ``rel``."""
    nq = int(owner.shape[0])
    out = _empty_like(rel, (nq, 3), np.float64)
    ctx.check(pt_tidal_eval(ctx.h, order, nq, _ptr(owner), _ptr(T), int(T.shape[0]), _ptr(acc_cm),
                            _ptr(rel), _ptr(out)), "pt_tidal_eval")
    return out
