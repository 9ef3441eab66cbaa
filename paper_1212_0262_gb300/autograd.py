"""torch.autograd.Function over md_grad: a final-time observable of an md_step
rollout, differentiable with respect to the initial positions, momenta and eps.

The forward pass calls md_grad once, which integrates forward (storing FP64
checkpoints) and runs the hand-written discrete adjoint backward; the gradients
are kept for the backward pass, which only scales them by the incoming
gradient.  All arithmetic runs in libmd's CUDA kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import binding as B
from .system import System


def _to_numpy(t: torch.Tensor) -> np.ndarray:
    return np.ascontiguousarray(t.detach().to("cpu", torch.float64).numpy())


class Rollout(torch.autograd.Function):
    """value = O(state after `nsteps` steps from (q0, p0)) of `system` with softening eps.

    q0, p0: float64 tensors of dim*N elements (any device); eps: 0-d tensor.
    observable: 0 = kinetic energy, 1 = |M| (HMF, Ring).
    """

    @staticmethod
    def forward(ctx, q0, p0, eps, system: System, nsteps: int, observable: int = 0,
                checkpoint_every: int = 20):
        system._chk(B.load().md_set_eps(system._h, float(eps)))
        system.set_state(_to_numpy(q0), _to_numpy(p0))
        val, gq, gp, ge = system.grad(int(nsteps), int(observable), int(checkpoint_every))
        dev = q0.device
        ctx.save_for_backward(torch.from_numpy(gq).to(dev), torch.from_numpy(gp).to(dev),
                              torch.tensor(ge, dtype=torch.float64, device=dev))
        return torch.tensor(val, dtype=torch.float64, device=dev)

    @staticmethod
    def backward(ctx, g):
        gq, gp, ge = ctx.saved_tensors
        return g * gq, g * gp, g * ge, None, None, None, None


def rollout(q0, p0, eps, system: System, nsteps: int, observable: int = 0, checkpoint_every: int = 20):
    """Functional form of Rollout.apply."""
    if not torch.is_tensor(eps):
        eps = torch.tensor(float(eps), dtype=torch.float64)
    return Rollout.apply(q0, p0, eps, system, nsteps, observable, checkpoint_every)


def rollout_model(q0, p0, eps, model, nsteps: int, dt: float, observable: int = 0, precision: str = "fp64",
                  checkpoint_every: int = 20):
    """Rollout by model: a context of `model` with N taken from q0 (dim*N elements) and
    time step dt is made for the call; the gradient flows to q0, p0 and eps."""
    from . import system as S

    m = S._model(model)
    n = int(q0.numel()) // {2: 2, 3: 3}.get(m, 1)
    e = float(eps.detach()) if torch.is_tensor(eps) else float(eps)
    with System(m, n, e, float(dt), 0, precision=precision) as s:
        return rollout(q0, p0, eps, s, nsteps, observable, checkpoint_every)
