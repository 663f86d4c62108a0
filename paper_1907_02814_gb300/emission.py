"""Differentiable expected-emission operator.

``expected_emission(ctx, Z, params, gamma, w)`` returns, per cell, the
expected photon rate, pair rate and radiated power of its electron samples
(rate form of the thin-target yield, Eq. N_br_theo1/2, and the radiative
stopping power of Sec. III.B) for plasma parameters
params[c] = (n_i, T_e, Z*, s_TF, s_D).  Forward and backward run in the
library's CUDA kernels (pcc_expected_emission_fwd / _bwd); the gradient
flows to ``params`` only.
"""
from __future__ import annotations

import torch

from . import pcc


class ExpectedEmission(torch.autograd.Function):
    @staticmethod
    def forward(fctx, lib_ctx, Z, params, gamma, w, n_quad):
        for name, t in (("params", params), ("gamma", gamma), ("w", w)):
            if t.dtype != torch.float32 or not t.is_cuda:
                raise TypeError(f"expected_emission: {name} must be a float32 CUDA tensor")
        params, gamma, w = params.contiguous(), gamma.contiguous(), w.contiguous()
        out = pcc.expected_emission_fwd(lib_ctx, Z, params, gamma, w, n_quad=n_quad)
        fctx.save_for_backward(params, gamma, w)
        fctx.lib_ctx, fctx.Z, fctx.n_quad = lib_ctx, Z, n_quad
        return out

    @staticmethod
    def backward(fctx, grad_out):
        params, gamma, w = fctx.saved_tensors
        g = pcc.expected_emission_bwd(fctx.lib_ctx, fctx.Z, params, gamma, w, grad_out.float().contiguous(),
                                      n_quad=fctx.n_quad)
        return None, None, g, None, None, None


def expected_emission(lib_ctx, Z, params, gamma, w, n_quad=64):
    """[n_cells, 3] float32: (R_gamma, R_pair, P_rad) per cell."""
    return ExpectedEmission.apply(lib_ctx, int(Z), params, gamma, w, int(n_quad))
