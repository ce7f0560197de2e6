"""Reverse-mode differentiation of whole IMEX trajectories for PyTorch.

``IMEXTrajectory`` is a ``torch.autograd.Function`` whose forward advances a
grid nsteps IMEX PD-ARS steps (He, Wibking & Krumholz 2024, Sec. 3.2) and whose
backward is the library's hand-written adjoint (``rhd_step_record`` +
``rhd_adjoint``): the transposed PLM/HLL transport of Sec. 3.3/4.3 and the
implicit-function-theorem adjoint of the local solve.  The paper has no
adjoint; this is the derivative of the step it defines.

Memory: the forward keeps one checkpoint of the 8 evolved fields every
``checkpoint_every`` steps.  The backward re-runs each segment from its
checkpoint with recording (two states per step: y(n) and y(n+1/2)) and then
walks it backwards, so the tape never holds more than one segment.

Everything runs on torch's current CUDA stream; the tensors are float64 on
the context's device.  This module is marshalling only: every step and every
adjoint step runs in the library's kernels.
"""
from __future__ import annotations

import torch

from . import rhd as R

#: evolved fields in the tape's slot order (Egas, mx, my, mz, E, Fx, Fy, Fz)
EVOLVED = (R.RHD_F_EGAS, R.RHD_F_MX, R.RHD_F_MY, R.RHD_F_MZ,
           R.RHD_F_ERAD, R.RHD_F_FX, R.RHD_F_FY, R.RHD_F_FZ)


def set_evolved(ctx: R.RHDContext, y: torch.Tensor):
    """Copy an (8, ncell) device tensor into the context's evolved fields."""
    for s, f in enumerate(EVOLVED):
        ctx.set_field(f, y[s])


def get_evolved(ctx: R.RHDContext, out: torch.Tensor | None = None) -> torch.Tensor:
    """The context's evolved fields as an (8, ncell) device tensor."""
    if out is None:
        out = torch.empty((8, ctx.ncell), dtype=torch.float64, device="cuda")
    for s, f in enumerate(EVOLVED):
        ctx.get_field(f, out[s])
    return out


class IMEXTrajectory(torch.autograd.Function):
    """y(nsteps) = step^nsteps(y0; kappa), differentiable in y0 and kappa.

    Arguments of ``apply``: y0 (8, ncell) and kappa (ncell) float64 CUDA
    tensors, the ``RHDContext`` (its rho must already be set), nsteps, dt
    (<= 0: the CFL step) and checkpoint_every."""

    @staticmethod
    def forward(fctx, y0, kappa, ctx, nsteps, dt, checkpoint_every):
        ctx.set_stream(torch.cuda.current_stream())
        y0 = y0.detach().contiguous()
        kappa = kappa.detach().contiguous()
        ctx.set_field(R.RHD_F_KAPPA, kappa)
        set_evolved(ctx, y0)
        dt = float(dt) if dt > 0 else ctx.default_dt()
        every = max(1, int(checkpoint_every))
        ckpts = [y0.clone()]
        done = 0
        while done < nsteps:
            k = min(every, nsteps - done)
            ctx.step(k, dt)
            done += k
            if done < nsteps:
                ckpts.append(get_evolved(ctx))
        out = get_evolved(ctx)
        fctx.rctx = ctx
        fctx.ckpts = ckpts
        fctx.nsteps = int(nsteps)
        fctx.dt = dt
        fctx.every = every
        fctx.save_for_backward(kappa)
        return out

    @staticmethod
    def backward(fctx, ybar_out):
        (kappa,) = fctx.saved_tensors
        ctx = fctx.rctx
        ctx.set_stream(torch.cuda.current_stream())
        n, every, dt = fctx.nsteps, fctx.every, fctx.dt
        ybar = ybar_out.detach().contiguous().clone()
        kbar = torch.zeros(ctx.ncell, dtype=torch.float64, device=ybar.device)
        ctx.set_field(R.RHD_F_KAPPA, kappa)
        tape = torch.empty((2 * min(every, n) + 1) * 8 * ctx.ncell, dtype=torch.float64,
                           device=ybar.device)
        for seg in reversed(range(len(fctx.ckpts))):
            k = min(every, n - seg * every)
            set_evolved(ctx, fctx.ckpts[seg])
            t = tape[: (2 * k + 1) * 8 * ctx.ncell]
            ctx.step_record(k, dt, t)
            ctx.adjoint(t, k, dt, ybar, kbar)
        return ybar, kbar, None, None, None, None


def trajectory(ctx: R.RHDContext, y0: torch.Tensor, kappa: torch.Tensor, nsteps: int,
               dt: float = 0.0, checkpoint_every: int = 20) -> torch.Tensor:
    """Differentiable y(nsteps) of the grid of ``ctx`` from (y0, kappa)."""
    return IMEXTrajectory.apply(y0, kappa, ctx, int(nsteps), float(dt), int(checkpoint_every))
