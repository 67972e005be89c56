"""Helpers shared by the GPU parity tests (conversion between the oracle's
numpy (N, k) arrays and the library's (k, N) complex64 CUDA tensors)."""
import numpy as np
import torch


def to_dev(a):
    a = np.asarray(a)
    if a.ndim == 1:
        return torch.from_numpy(a.astype(np.complex64)).cuda()
    return torch.from_numpy(np.ascontiguousarray(a.T.astype(np.complex64))).cuda()


def to_np(t):
    a = t.detach().cpu().numpy().astype(np.complex128)
    return a if a.ndim == 1 else a.T


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def hss_to_c_layout(hss):
    """Oracle HSS generators -> (ranks, U, B, D) flat complex64 arrays (column-major blocks)."""
    U = [u.flatten(order="F") for l in range(1, hss.Lh + 1) for u in hss.U[l]]
    B = [b.flatten(order="F") for l in range(hss.Lh) for b in hss.B[l]]
    D = [d.flatten(order="F") for d in hss.D]
    cat = lambda xs: (np.concatenate(xs) if xs else np.zeros(1)).astype(np.complex64)
    return list(hss.ranks), cat(U), cat(B), cat(D)
