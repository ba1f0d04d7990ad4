"""The allocation-free sort entry point, pt_sort_keys_noalloc.

Some callers cannot allocate device memory: their GPU memory belongs to
another allocator (a framework's caching allocator, a fixed arena), or they
run in a loop that must not allocate.  The regular entry points size their
workspace with cudaMalloc; this one works in a fixed scratch array inside the
library.  The tests call it through the C ABI, several times in a row (the
scratch keeps the previous call's contents, and the larger call comes first
so that a smaller one meets its leftovers), and check:

* Morton keys: the order pt_tree_build gives them (sorted keys and
  permutation, bit for bit);
* arbitrary 64-bit keys, half with the top bit set, drawn from a small pool
  so that most keys repeat: numpy's stable argsort, bit for bit;
* the device's free memory is the same before and after a call;
* sizes outside 1 .. 2^18 and host pointers are rejected.

This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2006_16560_gb300 import binding as B
from paper_2006_16560_gb300 import inputs

pytestmark = pytest.mark.gpu

MAX_N = 1 << 18


def _fn():
    f = B.lib().pt_sort_keys_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    return f


def _tree_order(ctx, d):
    """Sorted keys and permutation from the existing entry point."""
    import torch
    p = B.Params(theta=0.5, r_in=0.005, r_out=0.05, n_leaf=8, n_group=64, order=0)
    t = B.Tree(ctx, torch.from_numpy(d["pos"]).cuda(), torch.from_numpy(d["mass"]).cuda(), p)
    ks, perm = t.keys()
    t.free()
    return ks, perm


def _sort(f, keys_u64, stream):
    import torch
    n = len(keys_u64)
    dk = torch.from_numpy(np.ascontiguousarray(keys_u64).view(np.int64)).cuda()
    dks = torch.empty(n, dtype=torch.int64, device="cuda")
    dp = torch.empty(n, dtype=torch.int32, device="cuda")
    rc = f(n, dk.data_ptr(), dks.data_ptr(), dp.data_ptr(), stream)
    assert rc == B.PT_OK
    torch.cuda.synchronize()
    return dks.cpu().numpy().view(np.uint64), dp.cpu().numpy().view(np.uint32)


def test_noalloc_sort_matches_tree_build_twice():
    import torch
    ctx = B.Context(0)
    f = _fn()
    stream = torch.cuda.current_stream().cuda_stream
    for n, seed in ((MAX_N, 22), (200_000, 21)):
        d = inputs.plummer(n, seed, masses="kroupa")
        ks, perm = _tree_order(ctx, d)
        key_in = np.empty(n, dtype=np.uint64)
        key_in[perm] = ks                      # keys in the input order
        got_k, got_p = _sort(f, key_in, stream)
        assert np.array_equal(got_k, ks)
        assert np.array_equal(got_p, perm)
    ctx.close()


def test_noalloc_sort_arbitrary_keys_with_ties():
    import torch
    f = _fn()
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(31)
    pool = rng.integers(0, 2 ** 63, 500, dtype=np.uint64)
    pool[::2] |= np.uint64(1 << 63)                        # half the pool above 2^63
    pool[:4] = [0, 1, (1 << 64) - 1, 1 << 63]
    for n in (MAX_N, 1000, 1, 77_777):
        keys = pool[rng.integers(0, len(pool), n)]
        got_k, got_p = _sort(f, keys, stream)
        ref = np.argsort(keys, kind="stable")
        assert np.array_equal(got_p, ref.astype(np.uint32))
        assert np.array_equal(got_k, keys[ref])


def test_noalloc_sort_allocates_nothing():
    import torch
    f = _fn()
    stream = torch.cuda.current_stream().cuda_stream
    n = MAX_N
    keys = np.random.default_rng(5).integers(0, 2 ** 64 - 1, n, dtype=np.uint64)
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    dks = torch.empty(n, dtype=torch.int64, device="cuda")
    dp = torch.empty(n, dtype=torch.int32, device="cuda")
    assert f(n, dk.data_ptr(), dks.data_ptr(), dp.data_ptr(), stream) == B.PT_OK   # first call: set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert f(n, dk.data_ptr(), dks.data_ptr(), dp.data_ptr(), stream) == B.PT_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_sort_rejects_bad_sizes():
    import torch
    f = _fn()
    big = torch.zeros(MAX_N + 1, dtype=torch.int64, device="cuda")
    out = torch.empty(MAX_N + 1, dtype=torch.int64, device="cuda")
    pm = torch.empty(MAX_N + 1, dtype=torch.int32, device="cuda")
    assert f(MAX_N + 1, big.data_ptr(), out.data_ptr(), pm.data_ptr(), None) == B.PT_ERR_ARG
    assert f(0, big.data_ptr(), out.data_ptr(), pm.data_ptr(), None) == B.PT_ERR_ARG
    host = np.zeros(16, dtype=np.uint64)
    assert f(16, host.ctypes.data, out.data_ptr(), pm.data_ptr(), None) == B.PT_ERR_ARG
