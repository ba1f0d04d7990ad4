"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and bring its tree, lists and forces back as numpy arrays."""
from __future__ import annotations

import numpy as np

from paper_2006_16560_gb300 import binding as B


def run_gpu(ctx, pos, mass, params: B.Params, neighbours=True, device_buffers=True, repeat=1):
    """Build + force through pt_tree_build / pt_longrange_force.

    Returns a dict with acc, pot (input order), CSR neighbours, stats and the
    Tree (still alive, for introspection).  repeat > 1 calls the force that
    many times on the tree (a tree's first walk sizes its lists in two passes;
    later ones run in one pass into arrays sized from the last walk)."""
    import torch
    n = len(mass)
    if device_buffers:
        tp = torch.from_numpy(np.ascontiguousarray(pos)).cuda()
        tm = torch.from_numpy(np.ascontiguousarray(mass)).cuda()
        tree = B.Tree(ctx, tp, tm, params)
        acc = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        pot = torch.empty((n,), dtype=torch.float64, device="cuda")
        cap = max(8 * n, 1024)
        nb_off = torch.empty((n + 1,), dtype=torch.int64, device="cuda") if neighbours else None
        nb_idx = torch.empty((cap,), dtype=torch.int32, device="cuda") if neighbours else None
        for _ in range(repeat):
            total, st, rc = tree.force(acc, pot, nb_off, nb_idx, cap if neighbours else 0,
                                       allow_capacity_error=True)
            if rc == B.PT_ERR_CAPACITY:          # retry with the reported size
                nb_idx = torch.empty((total,), dtype=torch.int32, device="cuda")
                cap = total
                total, st, rc = tree.force(acc, pot, nb_off, nb_idx, total)
        out = {"acc": acc.cpu().numpy(), "pot": pot.cpu().numpy()}
        if neighbours:
            out["nb_off"] = nb_off.cpu().numpy()
            out["nb_idx"] = nb_idx[:total].cpu().numpy()
    else:
        tree = B.Tree(ctx, np.ascontiguousarray(pos), np.ascontiguousarray(mass), params)
        acc = np.zeros((n, 3))
        pot = np.zeros(n)
        cap = max(8 * n, 1024)
        nb_off = np.zeros(n + 1, dtype=np.int64) if neighbours else None
        nb_idx = np.zeros(cap, dtype=np.int32) if neighbours else None
        total, st, rc = tree.force(acc, pot, nb_off, nb_idx, cap if neighbours else 0,
                                   allow_capacity_error=True)
        if rc == B.PT_ERR_CAPACITY:
            nb_idx = np.zeros(total, dtype=np.int32)
            total, st, rc = tree.force(acc, pot, nb_off, nb_idx, total)
        out = {"acc": acc, "pot": pot}
        if neighbours:
            out["nb_off"] = nb_off
            out["nb_idx"] = nb_idx[:total]
    out["stats"] = st.as_dict()
    out["tree"] = tree
    return out


def rel_err(a, b):
    """Per-particle relative error |a - b| / |b| of (n,3) vectors."""
    den = np.linalg.norm(b, axis=1)
    return np.linalg.norm(a - b, axis=1) / np.where(den > 0, den, 1.0)


def node_ids(nodes, idx):
    """(level, begin) identifiers of node indices idx."""
    return sorted(zip(nodes["level"][idx].tolist(), nodes["begin"][idx].tolist()))
