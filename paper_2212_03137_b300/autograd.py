"""torch.autograd front end of the library's gradient kernels.

``bead_energy(system, x, theta)`` is U_P = (1/P) sum_b V(x_b) (Eq. (3)) of the bead
positions x (CUDA float64 [P, N, 3]) and the force-field parameters theta
(float64 [5]: eps, sigma, q_O, k_b, k_theta).  Its backward is the library's
hand-written gradient kernel (dU_P/dx = -F/P and dU_P/dtheta), not torch's tape.

``segment_average(system, theta, K, observable, block)`` is the time average of an
observable over K BAOAB steps from the system's current state with the thermostat
noise held fixed; its gradient is the library's checkpointed adjoint of the step,
evaluated together with the forward value (one call returns both).

Both only marshal arguments: every arithmetic step runs in libqhp.so.  Evaluating
``bead_energy`` makes x the system's bead positions (momenta are kept).
"""
from __future__ import annotations

import numpy as np
import torch

from . import qhp


def _bind_stream(system, device):
    qhp.qhp_set_stream(system.h, torch.cuda.current_stream(device).cuda_stream)


def _set_theta(system, theta):
    th = theta.detach().cpu().numpy().astype(np.float64)
    if not np.array_equal(th, qhp.ff_params(system.ff)):
        system.set_params(th)


class _BeadEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, theta, system):
        if x.dtype != torch.float64 or not x.is_cuda or tuple(x.shape) != (system.P, system.n_atoms, 3):
            raise ValueError("x must be a CUDA float64 tensor of shape [P, N, 3]")
        x = x.contiguous()
        _set_theta(system, theta)
        _bind_stream(system, x.device)
        e, _ = qhp.qhp_energy_grad_device(system.h, x.data_ptr(), None, want_theta=False)
        ctx.save_for_backward(x, theta)
        ctx.system = system
        return torch.tensor(e, dtype=torch.float64, device=x.device)

    @staticmethod
    def backward(ctx, g):
        x, theta = ctx.saved_tensors
        system = ctx.system
        _set_theta(system, theta)
        _bind_stream(system, x.device)
        gx = torch.empty_like(x)
        _, gt = qhp.qhp_energy_grad_device(system.h, x.data_ptr(), gx.data_ptr(), want_theta=True)
        gth = torch.as_tensor(gt, dtype=theta.dtype, device=theta.device)
        return g * gx, g.to(theta.device) * gth, None


def bead_energy(system, x: torch.Tensor, theta: torch.Tensor) -> torch.Tensor:
    return _BeadEnergy.apply(x, theta, system)


class _SegmentAverage(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, system, K, observable, block):
        _set_theta(system, theta)
        J, g = qhp.qhp_segment_grad(system.h, K, block, observable)
        ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
        return torch.tensor(J, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, gJ):
        (g,) = ctx.saved_tensors
        return gJ * g, None, None, None, None


def segment_average(system, theta: torch.Tensor, K: int, observable: int, block: int | None = None) -> torch.Tensor:
    """Differentiable J(theta); block defaults to ceil(sqrt(K)) steps between checkpoints."""
    if block is None:
        block = max(1, int(np.ceil(np.sqrt(K))))
    return _SegmentAverage.apply(theta, system, int(K), int(observable), int(block))
