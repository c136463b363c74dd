"""Helpers for the GPU parity tests (column-major torch tensors on cuda:0)."""
import numpy as np

U = 2.0 ** -53


def to_dev(A):
    import torch
    A = np.asfortranarray(A)
    t = torch.from_numpy(np.ascontiguousarray(A.T)).to("cuda:0")
    return t.t()  # column-major view: stride (1, n)


def to_host(t):
    if isinstance(t, np.ndarray):
        return t
    return t.detach().cpu().numpy()
