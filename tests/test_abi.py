"""The C-ABI library loads on any machine with the CUDA runtime and exports
every entry point that include/pt.h declares (no GPU needed)."""
import os
import re

from paper_2006_16560_gb300 import binding as B

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "pt.h")


def declared():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pt_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared()
    for need in ("pt_ctx_create", "pt_ctx_destroy", "pt_tree_build", "pt_longrange_force",
                 "pt_tree_free", "pt_batch_longrange_force", "pt_last_error"):
        assert need in names


def test_library_exports_every_declared_symbol():
    L = B.lib()
    for name in declared():
        assert hasattr(L, name), name
    assert L.pt_abi_version() == 1


def test_no_gpu_means_error_not_fallback():
    import ctypes
    import torch
    if torch.cuda.is_available():
        return
    h = ctypes.c_void_p()
    assert B.lib().pt_ctx_create(ctypes.byref(h), 0, None) == B.PT_ERR_CUDA
