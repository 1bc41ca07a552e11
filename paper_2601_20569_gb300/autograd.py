"""torch.autograd bridge of the refit adjoint.

``refit_chi2(tracker, clusters, tracks, coeff)`` returns the per-track refit
chi2 as a tensor that is differentiable with respect to the correction-map
control points ``coeff``: backward calls the library's hand-written adjoint
(tpc_refit_backward), with the fit's references and decisions held fixed.
This is what a distortion calibration minimising the summed chi2 needs.
"""
from __future__ import annotations

import torch


class RefitChi2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coeff, tracker, clusters, tracks):
        out = tracker.refit(clusters, tracks, coeff.detach().contiguous())
        ctx.tracker = tracker
        ctx.shape = tuple(coeff.shape)
        return out["chi2"].clone()

    @staticmethod
    def backward(ctx, grad_chi2):
        g = ctx.tracker.refit_backward(grad_chi2, ctx.shape)
        return g, None, None, None


def refit_chi2(tracker, clusters, tracks, coeff):
    return RefitChi2.apply(coeff, tracker, clusters, tracks)
