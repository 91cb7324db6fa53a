"""Linear response through torch.autograd.

The SETD step (Sec. II schemes, Sec. IV boxed algorithm) maps the state phi_t
to phi_{t+n} along one noise path.  Its derivative with respect to a
perturbation of phi_t -- the dynamic linear response to a field kick
h(x, t) = eps f(x) delta(t - t0), which displaces phi(t0) by Gamma eps f(x) --
is a linear map J (the noise enters additively and drops out of it).

``SETDPropagate`` exposes J as an autograd Function:
  forward(dphi0)  = J dphi0        (tangent map, ``sft_tangent_step``)
  backward(g)     = J^T g          (adjoint, ``sft_adjoint``, checkpointed with
                                    Philox noise regeneration)
Both run in the library's CUDA kernels; this module only marshals tensors.
Every case the library differentiates: the cubic term (d = 1..3), the KPZ and
CGL terms (d = 1, 2), every scheme.  Complex fields (CGL) take complex64
tensors; J is then only real-linear (the linearised |A|^2 A term holds
conj(dA)), and backward returns its transpose for the real inner product
Re sum conj(u) v, which is the vector-Jacobian product of torch's convention
for a real loss (grad = dL/dRe + i dL/dIm).
"""
from __future__ import annotations

import torch

from . import Stepper, sft_adjoint, sft_tangent_step


def _device_fields(x: torch.Tensor, stepper: Stepper, what: str) -> torch.Tensor:
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % what)
    shape = (stepper.R,) + tuple(stepper.shape)
    if tuple(x.shape) != shape:
        raise ValueError("%s must have shape %s (replicas, lattice), got %s" % (what, shape, tuple(x.shape)))
    return x.detach().to(torch.complex64 if stepper.complex_field else torch.float32).contiguous()


class SETDPropagate(torch.autograd.Function):
    """dphi(t + n) = J dphi(t) for the stepper's current state and noise path.

    The primal advances by ``nsteps`` (as a plain step would).  The backward
    pass rewinds the stepper to the forward's start state, runs the adjoint
    over the same steps and puts the stepper back where it was.
    """

    @staticmethod
    def forward(ctx, dphi0: torch.Tensor, stepper: Stepper, nsteps: int):
        x = _device_fields(dphi0, stepper, "dphi0")
        start = stepper.checkpoint()
        out = torch.empty_like(x)
        torch.cuda.current_stream(x.device).synchronize()  # x is complete before the library stream reads it
        sft_tangent_step(stepper.ctx, x.data_ptr(), int(nsteps), out.data_ptr())
        stepper.sync()
        ctx.stepper, ctx.nsteps, ctx.start = stepper, int(nsteps), start
        return out

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        st: Stepper = ctx.stepper
        g = _device_fields(grad_out, st, "grad_out")
        here = st.checkpoint()
        st.restore(ctx.start)
        grad = torch.empty_like(g)
        torch.cuda.current_stream(g.device).synchronize()
        sft_adjoint(st.ctx, g.data_ptr(), ctx.nsteps, grad.data_ptr())
        st.sync()
        st.restore(here)
        return grad, None, None


def propagate(dphi0: torch.Tensor, stepper: Stepper, nsteps: int) -> torch.Tensor:
    """J dphi0 over ``nsteps`` steps, differentiable with respect to dphi0."""
    return SETDPropagate.apply(dphi0, stepper, nsteps)
