"""The allocation-free sort entry point, pt_sort_keys_noalloc.

Some callers cannot allocate device memory (their GPU memory belongs to
another allocator, or they run in a loop that must not allocate); the
regular entry points size their workspace with cudaMalloc, this one works in
a fixed scratch array inside the library.  The test calls it through the C
ABI, twice in a row on different inputs (the scratch keeps the previous
call's contents), and checks that it orders the Morton keys exactly as
pt_tree_build does (sorted keys and permutation, bit for bit).  This file is
collected last on purpose.
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


def test_noalloc_sort_matches_tree_build_twice():
    import torch
    ctx = B.Context(0)
    f = _fn()
    stream = torch.cuda.current_stream().cuda_stream
    for n, seed in ((200_000, 21), (MAX_N, 22)):
        d = inputs.plummer(n, seed, masses="kroupa")
        ks, perm = _tree_order(ctx, d)
        key_in = np.empty(n, dtype=np.uint64)
        key_in[perm] = ks                      # keys in the input order
        dk = torch.from_numpy(key_in.view(np.int64)).cuda()
        dks = torch.empty(n, dtype=torch.int64, device="cuda")
        dp = torch.empty(n, dtype=torch.int32, device="cuda")
        rc = f(n, dk.data_ptr(), dks.data_ptr(), dp.data_ptr(), stream)
        assert rc == B.PT_OK
        torch.cuda.synchronize()
        assert np.array_equal(dks.cpu().numpy().view(np.uint64), ks)
        assert np.array_equal(dp.cpu().numpy().view(np.uint32), perm)
    ctx.close()


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
