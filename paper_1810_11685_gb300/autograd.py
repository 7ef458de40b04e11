"""torch.autograd bindings of the composite maps.

``qpat_data(ctx, mu, illum)`` returns the sensor series P-hat = H_a H_o[mu]
(eq. com_des) as a differentiable function of the absorption map mu:

* backward (reverse mode) is J^T w = J_o^* H_a^*(w) (Lemma 1 mu row, Lemma 2),
  computed by ``qpat_vjp`` from the fluence saved by the forward call;
* forward mode (``torch.func.jvp`` / ``torch.autograd.forward_ad``) is
  J v = H_a J_o v (eq. J_des) through ``qpat_jvp``.

``acoustic(ctx, p0)`` is the linear map H_a with H_a^* as its backward.
All arithmetic runs in the CUDA library; mu, its gradient and tangents are
float64, the sensor series has the context's precision.
"""
from __future__ import annotations

import torch


class _QpatData(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mu, qctx, illum):
        data, phi = qctx.forward(mu, illum, return_phi=True)
        ctx.qctx, ctx.illum = qctx, illum
        ctx.save_for_backward(mu, phi)
        ctx.save_for_forward(mu, phi)
        return data

    @staticmethod
    def backward(ctx, grad_data):
        mu, phi = ctx.saved_tensors
        g = ctx.qctx.vjp(mu, grad_data.to(ctx.qctx.dtype).contiguous(), ctx.illum, phi0=phi)
        return g.reshape(mu.shape), None, None

    @staticmethod
    def jvp(ctx, mu_t, qctx_t, illum_t):
        mu, phi = ctx.saved_tensors
        return ctx.qctx.jvp(mu, mu_t.contiguous(), ctx.illum, phi0=phi)


def qpat_data(qctx, mu: torch.Tensor, illum: int) -> torch.Tensor:
    """Differentiable P-hat = H_a H_o[mu] for illumination mask ``illum``.
    mu: CUDA float64 [n1][n0] or [B][n1][n0]; returns [B][nt][ns]."""
    return _QpatData.apply(mu, qctx, illum)


class _Acoustic(torch.autograd.Function):
    @staticmethod
    def forward(ctx, p0, qctx):
        ctx.qctx = qctx
        ctx.shape = p0.shape
        return qctx.acoustic_forward(p0)

    @staticmethod
    def backward(ctx, grad):
        return ctx.qctx.acoustic_adjoint(grad.contiguous()).reshape(ctx.shape), None

    @staticmethod
    def jvp(ctx, p0_t, qctx_t):
        return ctx.qctx.acoustic_forward(p0_t.contiguous())


def acoustic(qctx, p0: torch.Tensor) -> torch.Tensor:
    """Differentiable H_a (linear): p0 [n1][n0] or [B][n1][n0] -> [B][nt][ns]."""
    return _Acoustic.apply(p0, qctx)
