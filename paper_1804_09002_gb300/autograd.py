"""torch.autograd bridge of the CS decomposition: the forward is csd_polar
(canonical column signs, so U1, U2, V1 are functions of A), the backward is
the library's csd_polar_backward (hand-written adjoint kernels).  Argument
marshalling only: both directions run in the CUDA library.

    U1, U2, V1, theta = csd(A1, A2)        # A1, A2: float64 CUDA tensors
    loss = (theta ** 2).sum() + ((U1 - U1_ref) ** 2).sum()
    loss.backward()                        # A1.grad, A2.grad

Real, full-rank inputs only (the derivative of the rank-deficient CSD is not
provided).
"""
import torch

from . import binding as _B

_contexts = {}


def _context(device):
    idx = device.index if device.index is not None else torch.cuda.current_device()
    if idx not in _contexts:
        c = _B.Context(idx)
        c.set_sign_convention(1)
        _contexts[idx] = c
    return _contexts[idx]


class CSDPolar(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A1, A2):
        c = _context(A1.device)
        R = c.csd_polar(A1.detach(), A2.detach())
        n = A1.shape[1]
        if R["rank"] != n:
            raise ValueError(f"csd: rank {R['rank']} < n = {n}; the derivative needs a full-rank input")
        U1, U2, V1, th = R["U1"], R["U2"], R["V1"], R["theta"]
        ctx.save_for_backward(U1, U2, V1, th)
        return U1, U2, V1, th

    @staticmethod
    def backward(ctx, gU1, gU2, gV1, gth):
        U1, U2, V1, th = ctx.saved_tensors
        c = _context(U1.device)
        gA1, gA2 = c.csd_backward(U1, U2, V1, th, gU1, gU2, gV1, gth)
        return gA1, gA2


def csd(A1, A2):
    """(U1, U2, V1, theta) of [A1; A2] with a backward pass to A1, A2."""
    return CSDPolar.apply(A1, A2)


def csd_many(pairs):
    """CS decompositions of a list of (A1, A2) pairs of any sizes; each
    result carries its own backward."""
    return [CSDPolar.apply(a1, a2) for a1, a2 in pairs]
