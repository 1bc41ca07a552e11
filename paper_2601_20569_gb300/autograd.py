"""torch.autograd bridge of the refit adjoint.

``refit_chi2(tracker, clusters, tracks, coeff)`` returns the per-track refit
chi2 as a tensor that is differentiable with respect to the correction-map
control points ``coeff``: backward calls the library's hand-written adjoint
(tpc_refit_backward), with the fit's references and decisions held fixed.
This is what a distortion calibration minimising the summed chi2 needs.

The library differentiates the most recent refit of a context.  The forward
records the context's refit generation and the backward refuses (TpcError,
TPC_ERR_STATE) when another refit ran on that context in between; ``coeff``
is saved for backward, so an in-place change of the map after the forward
is caught by torch's version check.
"""
from __future__ import annotations

import torch

TPC_ERR_STATE = 7


class RefitChi2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coeff, tracker, clusters, tracks):
        c = coeff.detach().contiguous()
        out = tracker.refit(clusters, tracks, c)
        ctx.tracker = tracker
        ctx.generation = tracker.refit_generation()
        ctx.shape = tuple(coeff.shape)
        ctx.save_for_backward(coeff)
        return out["chi2"].clone()

    @staticmethod
    def backward(ctx, grad_chi2):
        from .tpc import TpcError

        (_coeff,) = ctx.saved_tensors  # raises if coeff was modified in place
        if ctx.tracker.refit_generation() != ctx.generation:
            raise TpcError(TPC_ERR_STATE, "another refit ran on this tracker after this "
                           "forward; its backward would differentiate that refit")
        g = ctx.tracker.refit_backward(grad_chi2, ctx.shape)
        return g, None, None, None


def refit_chi2(tracker, clusters, tracks, coeff):
    return RefitChi2.apply(coeff, tracker, clusters, tracks)
