"""torch.autograd bindings of the hand-written REINFORCE backward (sg_grad).

The paper trains with PyTorch autograd on the objective of Eq. loss1, whose
gradient is the score-function estimator
    grad F_q  ~  (1/B) sum_b (L_b - Lbar) grad log q(sigma_b),   L = beta E + ln q,
with the coefficients (L_b - Lbar)/B held constant (Methods "Training
strategy").  Here the derivative of log q with respect to the weights is the
library's hand-written backward, exposed to autograd in two forms:

* ``LogQ`` -- log q(sigma_b) of given configurations as a differentiable
  function of the model's FP32 weight blob.  Forward: sg_logprob.  Backward:
  the vector-Jacobian product sum_b g_b d log q_b / d theta, which is exactly
  sg_grad with coefficients g = the incoming gradient.  Any loss built from
  log q (the REINFORCE surrogate, Eq. loss2's likelihood term) backpropagates
  through it.
* ``ReinforceLoss`` -- the surrogate sum_b c_b log q(sigma_b) with fixed
  coefficients c in one fused call: its forward runs sg_grad once, which
  returns log q and the gradient together (the activations are recomputed
  inside the call, chunk by chunk), and its backward scales that stored
  gradient by the incoming scalar.  This is the training path: no second
  forward pass.

Both take the weight blob as their first argument so that autograd attaches
the gradient to it: pass ``Model.weights()`` with ``requires_grad_(True)``.
Python does argument marshalling only; the arithmetic runs in libsg kernels.
"""
from __future__ import annotations

import torch

from . import sg


def _check_weights(weights, model):
    if weights.data_ptr() != model.weights().data_ptr():
        raise ValueError("weights must be the model's own blob (Model.weights())")


class LogQ(torch.autograd.Function):
    """log q(sigma_b) (Algorithm 1, teacher-forced) with the hand-written
    backward as its vector-Jacobian product."""

    @staticmethod
    def forward(ctx, weights, model, spins):
        _check_weights(weights, model)
        ctx.model = model
        ctx.save_for_backward(spins)
        return model.logprob(spins)

    @staticmethod
    def backward(ctx, grad_logq):
        (spins,) = ctx.saved_tensors
        g = ctx.model.grad(spins, grad_logq.detach().to(torch.float32).contiguous())
        return g, None, None


class ReinforceLoss(torch.autograd.Function):
    """sum_b coeff_b log q(sigma_b) with coeff held constant (Eq. loss1's
    surrogate); forward and backward in one sg_grad call."""

    @staticmethod
    def forward(ctx, weights, model, spins, coeff):
        _check_weights(weights, model)
        coeff = coeff.detach().to(torch.float32).contiguous()
        logq = torch.empty(spins.shape[0], dtype=torch.float32, device=spins.device)
        ctx.g = model.grad(spins, coeff, logq=logq)
        ctx.logq = logq
        # the surrogate's value, reported only (its gradient is g)
        return torch.dot(coeff, logq)

    @staticmethod
    def backward(ctx, grad_out):
        return ctx.g * grad_out, None, None, None


def logq(model: "sg.Model", spins: torch.Tensor, weights: torch.Tensor | None = None):
    """Differentiable teacher-forced log q of ``spins`` [B][N] int8."""
    w = model.weights() if weights is None else weights
    return LogQ.apply(w, model, spins)


def reinforce_loss(model: "sg.Model", spins: torch.Tensor, coeff: torch.Tensor,
                   weights: torch.Tensor | None = None):
    """The REINFORCE surrogate sum_b coeff_b log q(sigma_b); ``loss.backward()``
    puts sum_b coeff_b grad log q(sigma_b) into ``weights.grad``."""
    w = model.weights() if weights is None else weights
    return ReinforceLoss.apply(w, model, spins, coeff)
