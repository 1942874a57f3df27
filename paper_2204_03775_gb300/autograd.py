"""Receiver traces as a differentiable torch function of the squared slowness.

``traces(m, shot)`` runs one shot of the stepper from rest and returns its
traces [nrec][nt]; its backward pass is the library's discrete adjoint
(``ws_adjoint_gradient`` in residual mode), so gradients of any loss of the
traces with respect to m = 1/V^2 flow through the same kernels. Marshalling
only: the forward and the backward pass both run in libwavestep.
"""

from __future__ import annotations

import numpy as np
import torch

from . import binding as b


class Shot:
    """One source gather: its own handle (sources, receivers, taper, tiling)."""

    def __init__(self, shape, h: float, dt: float, nt: int, sources, receivers,
                 sponge=(0, 0.0), kernel: int = b.WS_KERNEL_AUTO):
        nz, ny, nx = shape
        self.shape = (nz, ny, nx)
        self.nt = int(nt)
        self.receivers = np.ascontiguousarray(np.asarray(receivers, np.int32).reshape(-1, 3))
        self.ws = b.ws_create(nx, ny, nz, h, dt)
        b.ws_set_sponge(self.ws, *sponge)
        b.ws_set_kernel(self.ws, kernel)
        for s in sources:
            b.ws_add_source(self.ws, *s)
        b.ws_set_receivers(self.ws, self.receivers, self.nt)

    def _bind(self, m: torch.Tensor) -> None:
        """Give the handle the model m, unless it already holds this very tensor
        unmodified (then the checkpoints of its last forward run stay usable)."""
        if not (m.is_cuda and m.dtype == torch.float32 and tuple(m.shape) == self.shape):
            raise TypeError(f"m: a float32 CUDA tensor of shape {self.shape}")
        b.ws_set_stream(self.ws, torch.cuda.current_stream(m.device))
        # the reference to the bound tensor keeps its memory from being reused
        # by another tensor that would then look identical
        if getattr(self, "_bound", None) is not m or self._bound_version != m._version:
            b.ws_set_slowness2(self.ws, m.contiguous())
            self._bound, self._bound_version = m, m._version


class _Traces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m: torch.Tensor, shot: Shot) -> torch.Tensor:
        shot._bind(m)
        b.ws_forward(shot.ws)          # traces + the checkpoints the backward reuses
        out = torch.empty((len(shot.receivers), shot.nt), dtype=torch.float32, device=m.device)
        b.ws_read_traces(shot.ws, out)
        ctx.save_for_backward(m)
        ctx.shot = shot
        return out

    @staticmethod
    def backward(ctx, grad_traces: torch.Tensor):
        (m,) = ctx.saved_tensors
        shot = ctx.shot
        shot._bind(m)
        r = grad_traces.detach().to(torch.float32).contiguous()
        grad = torch.empty_like(m)
        b.ws_adjoint_gradient(shot.ws, r, b.WS_ADJ_RESIDUAL, grad)
        return grad, None


def traces(m: torch.Tensor, shot: Shot) -> torch.Tensor:
    """Traces [nrec][nt] of `shot` in the model m = 1/V^2 (float32 CUDA, [nz][ny][nx])."""
    return _Traces.apply(m, shot)
