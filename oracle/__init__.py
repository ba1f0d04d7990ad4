"""CPU oracle for the P3T long-range force -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it and
shares no code with it.  The arithmetic lives in ``pt_oracle.c`` (plain C,
float64, compiled without FMA contraction); this module compiles it with gcc
and wraps it with ctypes and numpy.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pt_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()

_i64 = C.c_int64
_dbl = C.c_double
_p = C.c_void_p


def build(force: bool = False) -> str:
    """Compile pt_oracle.c into a shared object (gcc, OpenMP, no FMA contraction)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            for name, res, args in [
                ("orc_f", _dbl, [_dbl, _dbl]),
                ("orc_W", _dbl, [_dbl, _dbl]),
                ("orc_K", _dbl, [_dbl, _dbl]),
                ("orc_direct", None, [_i64, _p, _p, _dbl, _dbl, _dbl, _i64, _p, _p, _p, C.c_int, _p]),
                ("orc_neighbours_count", None, [_i64, _p, _dbl, _i64, _p, _p, _p]),
                ("orc_neighbours_fill", None, [_i64, _p, _dbl, _i64, _p, _p, _p, _p]),
                ("orc_radius_scale", None, [_i64, _p, _p]),
                ("orc_tree_build", _p, [_i64, _p, _p, C.c_int, C.c_int, _p]),
                ("orc_tree_free", None, [_p]),
                ("orc_tree_info", None, [_p, _p, _p]),
                ("orc_tree_keys", None, [_p, _p, _p, _p]),
                ("orc_tree_nodes", None, [_p, _p, _p, _p]),
                ("orc_tree_groups", None, [_p, _p]),
                ("orc_tree_walk", C.c_int, [_p, _i64, _dbl, _dbl, _p, _i64, _p, _i64, _p, _p]),
                ("orc_cell_pull", None, [_p, _i64, _p, C.c_int, _p, _p]),
                ("orc_tree_force", None, [_p, _dbl, _dbl, _dbl, _dbl, C.c_int, _i64, _p, _p, _p, _p]),
                ("orc_pericentre", _dbl, [_p, _p, _dbl]),
                ("orc_rnb", None, [_i64, _p, _p, _dbl, _dbl, _dbl, _p]),
                ("orc_orbit_count", None, [_i64, _p, _p, _p, _p, _p, _dbl, _dbl, _dbl, C.c_int, _i64,
                                           _p, _p, _p]),
                ("orc_orbit_fill", None, [_i64, _p, _p, _p, _p, _p, _dbl, _dbl, _dbl, C.c_int, _i64,
                                          _p, _p, _p]),
                ("orc_abi_version", C.c_int, []),
            ]:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def changeover_f(x: float, lam: float) -> float:
    return lib().orc_f(float(x), float(lam))


def changeover_W(x: float, lam: float) -> float:
    return lib().orc_W(float(x), float(lam))


def changeover_K(x: float, lam: float) -> float:
    return lib().orc_K(float(x), float(lam))


def radius_scale(mass):
    """Eq. 12 radius factors s_i = max(1, m_i/<m>)^(1/3)."""
    mass = _f64(mass)
    out = np.zeros(len(mass))
    lib().orc_radius_scale(len(mass), _ptr(mass), _ptr(out))
    return out


def direct_force(pos, mass, r_in, r_out, G=1.0, targets=None, shortrange=False, scale=None):
    """Direct O(N^2) long-range (or short-range) acc (nt,3) and pot (nt,);
    ``scale`` gives per-particle radius factors (pair radii use the larger)."""
    pos = _f64(pos)
    mass = _f64(mass)
    sc = None if scale is None else _f64(scale)
    n = len(mass)
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else len(tg)
    acc = np.zeros((nt, 3))
    pot = np.zeros(nt)
    lib().orc_direct(n, _ptr(pos), _ptr(mass), G, r_in, r_out, nt, _ptr(tg),
                     _ptr(acc), _ptr(pot), 1 if shortrange else 0, _ptr(sc))
    return acc, pot


def neighbours(pos, r_out, targets=None, scale=None):
    """Brute-force r_out neighbour sets as CSR (offsets (nt+1,), idx)."""
    pos = _f64(pos)
    sc = None if scale is None else _f64(scale)
    n = len(pos)
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else len(tg)
    cnt = np.zeros(nt, dtype=np.int64)
    lib().orc_neighbours_count(n, _ptr(pos), r_out, nt, _ptr(tg), _ptr(cnt), _ptr(sc))
    off = np.zeros(nt + 1, dtype=np.int64)
    np.cumsum(cnt, out=off[1:])
    idx = np.zeros(max(int(off[-1]), 1), dtype=np.int32)
    lib().orc_neighbours_fill(n, _ptr(pos), r_out, nt, _ptr(tg), _ptr(off), _ptr(idx), _ptr(sc))
    return off, idx[: off[-1]]


ORBIT_ROUT, ORBIT_RNB, ORBIT_CANDIDATES = 0, 1, 2


def pericentre(dx, dv, mu) -> float:
    """Kepler pericentre distance of the relative orbit (Sec. 6.3.1)."""
    dx, dv = _f64(dx), _f64(dv)
    return lib().orc_pericentre(_ptr(dx), _ptr(dv), float(mu))


def neighbour_radius(vel, r_out, dt, C_r=3.0, scale=None):
    """Eq. 24: r_nb,i = s_i r_out + C_r |v_i| dt."""
    vel = _f64(vel)
    sc = None if scale is None else _f64(scale)
    out = np.zeros(len(vel))
    lib().orc_rnb(len(vel), _ptr(vel), _ptr(sc), r_out, dt, C_r, _ptr(out))
    return out


def orbit_neighbours(pos, vel, mass, r_out, dt, C_r=3.0, C_v=1.5, G=1.0, mode=ORBIT_ROUT,
                     scale=None, targets=None):
    """Two-stage orbit-dependent neighbour sets (Sec. 6.3.1) as CSR
    (offsets (nt+1,), idx) plus per-target stage-1 candidate counts.

    mode ORBIT_ROUT keeps candidates with pericentre < C_v r_out,ij (the
    reading used by the library), ORBIT_RNB the printed C_v r_nb,ij, and
    ORBIT_CANDIDATES returns the stage-1 candidates themselves."""
    pos, vel, mass = _f64(pos), _f64(vel), _f64(mass)
    sc = None if scale is None else _f64(scale)
    n = len(mass)
    rnb = neighbour_radius(vel, r_out, dt, C_r, sc)
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else len(tg)
    cnt = np.zeros(nt, dtype=np.int64)
    ncand = np.zeros(nt, dtype=np.int64)
    L = lib()
    L.orc_orbit_count(n, _ptr(pos), _ptr(vel), _ptr(mass), _ptr(sc), _ptr(rnb), r_out, G, C_v, mode,
                      nt, _ptr(tg), _ptr(cnt), _ptr(ncand))
    off = np.zeros(nt + 1, dtype=np.int64)
    np.cumsum(cnt, out=off[1:])
    idx = np.zeros(max(int(off[-1]), 1), dtype=np.int32)
    L.orc_orbit_fill(n, _ptr(pos), _ptr(vel), _ptr(mass), _ptr(sc), _ptr(rnb), r_out, G, C_v, mode,
                     nt, _ptr(tg), _ptr(off), _ptr(idx))
    return off, idx[: off[-1]], ncand


class Tree:
    """Oracle octree (keys, sort, nodes, moments, groups) over one particle set."""

    def __init__(self, pos, mass, n_leaf: int, n_group: int, scale=None):
        self._pos = _f64(pos)
        self._mass = _f64(mass)
        self._scale = None if scale is None else _f64(scale)
        self.n = len(self._mass)
        self.n_leaf = n_leaf
        self.n_group = n_group
        self._h = lib().orc_tree_build(self.n, _ptr(self._pos), _ptr(self._mass), n_leaf, n_group,
                                       _ptr(self._scale))
        info = np.zeros(4, dtype=np.int64)
        box = np.zeros(5)
        lib().orc_tree_info(self._h, _ptr(info), _ptr(box))
        self.nnodes = int(info[1])
        self.ngroups = int(info[2])
        self.max_level = int(info[3])
        self.origin = box[:3].copy()
        self.S = float(box[3])
        self.scale = float(box[4])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_tree_free(h)
            self._h = None

    def keys(self):
        """(keys per original index, grid q (n,3) per original index, perm)."""
        key = np.zeros(self.n, dtype=np.uint64)
        q = np.zeros((self.n, 3), dtype=np.uint32)
        perm = np.zeros(self.n, dtype=np.int64)
        lib().orc_tree_keys(self._h, _ptr(key), _ptr(q), _ptr(perm))
        return key, q, perm

    def nodes(self) -> dict:
        ints = np.zeros((self.nnodes, 8), dtype=np.int64)
        q = np.zeros((self.nnodes, 6), dtype=np.uint32)
        mom = np.zeros((self.nnodes, 10))
        lib().orc_tree_nodes(self._h, _ptr(ints), _ptr(q), _ptr(mom))
        return {"begin": ints[:, 0], "count": ints[:, 1], "level": ints[:, 2],
                "leaf": ints[:, 3], "first_child": ints[:, 4], "nchild": ints[:, 5],
                "qmin": q[:, :3], "qmax": q[:, 3:], "mass": mom[:, 0],
                "com": mom[:, 1:4], "quad": mom[:, 4:10]}

    def groups(self) -> dict:
        g = np.zeros((self.ngroups, 8), dtype=np.int64)
        lib().orc_tree_groups(self._h, _ptr(g))
        return {"begin": g[:, 0], "count": g[:, 1], "qmin": g[:, 2:5], "qmax": g[:, 5:8]}

    def walk(self, g: int, theta: float, r_out: float):
        """(cells as node indices, PP as sorted particle indices) of group g."""
        nc = np.zeros(1, dtype=np.int64)
        npp = np.zeros(1, dtype=np.int64)
        lib().orc_tree_walk(self._h, g, theta, r_out, None, 0, None, 0, _ptr(nc), _ptr(npp))
        cells = np.zeros(max(int(nc[0]), 1), dtype=np.int64)
        pp = np.zeros(max(int(npp[0]), 1), dtype=np.int64)
        lib().orc_tree_walk(self._h, g, theta, r_out, _ptr(cells), len(cells), _ptr(pp),
                            len(pp), _ptr(nc), _ptr(npp))
        return cells[: nc[0]], pp[: npp[0]]

    def cell_pull(self, v: int, x, order: int):
        x = _f64(x)
        acc = np.zeros(3)
        pot = np.zeros(1)
        lib().orc_cell_pull(self._h, v, _ptr(x), order, _ptr(acc), _ptr(pot))
        return acc, float(pot[0])

    def force(self, theta, r_in, r_out, G=1.0, order=2, targets=None):
        """Tree force; per original index (targets None) or per target slot.

        Returns (acc, pot, stats) with stats = (cell interactions, PP list
        interactions)."""
        tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
        nt = self.n if tg is None else len(tg)
        acc = np.zeros((nt, 3))
        pot = np.zeros(nt)
        st = np.zeros(2, dtype=np.int64)
        lib().orc_tree_force(self._h, theta, r_in, r_out, G, order, nt, _ptr(tg),
                             _ptr(acc), _ptr(pot), _ptr(st))
        return acc, pot, (int(st[0]), int(st[1]))
