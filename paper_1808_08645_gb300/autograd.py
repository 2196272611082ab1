"""torch.autograd binding of the receiver traces: c^2 -> traces, with the
library's discrete adjoint as the backward (argument marshalling only; every
step runs in libbbwadg through ``binding.Solver``).

    traces = receiver_traces(solver, c2, q0, dt, nsteps, checkpoint_every)
    loss = 0.5 * ((traces - data) ** 2).sum()
    loss.backward()          # c2.grad = d loss / d c2 (bbw_adjoint)

``solver`` carries the mesh, degree, penalties, source and receivers; ``c2``
is a [K, M_p] tensor of Bernstein coefficients (any device; it is copied to
the host for the ABI), ``q0`` the initial state [4, K, N_p] (numpy or tensor).
The solver keeps one recorded run; when several forwards share a solver, the
backward of an earlier one records its run again (from the c2 and q0 it kept)
before the adjoint, and leaves the solver in that run's state.
"""
from __future__ import annotations

import numpy as np
import torch

__all__ = ["ReceiverTraces", "receiver_traces"]


def _host(x) -> np.ndarray:
    if isinstance(x, torch.Tensor):
        return x.detach().to("cpu", torch.float64).numpy()
    return np.asarray(x, dtype=np.float64)


class ReceiverTraces(torch.autograd.Function):
    """traces[n, r] = pressure at receiver r after step n, as a function of c2."""

    @staticmethod
    def forward(ctx, c2, solver, q0, dt, nsteps, checkpoint_every, t0):
        c2h, q0h = _host(c2), _host(q0)
        solver.set_c2(c2h)
        solver.set_state(q0h, None, float(t0))
        tr = solver.record(float(dt), int(nsteps), int(checkpoint_every))
        ctx.solver = solver
        # the run this output came from: the solver differentiates only its
        # latest recorded run, so backward re-records if another run came since
        ctx.run = solver.runs
        ctx.inputs = (c2h, q0h, float(dt), int(nsteps), int(checkpoint_every), float(t0))
        return torch.from_numpy(tr).to(dtype=c2.dtype, device=c2.device)

    @staticmethod
    def backward(ctx, grad_traces):
        s = ctx.solver
        if s.runs != ctx.run:
            c2h, q0h, dt, nsteps, every, t0 = ctx.inputs
            s.set_c2(c2h)
            s.set_state(q0h, None, t0)
            s.record(dt, nsteps, every)
            ctx.run = s.runs
        gc, _ = s.adjoint(_host(grad_traces))
        return (torch.from_numpy(gc).to(dtype=grad_traces.dtype, device=grad_traces.device),
                None, None, None, None, None, None)


def receiver_traces(solver, c2, q0, dt: float, nsteps: int, checkpoint_every: int = 1, t0: float = 0.0):
    """Differentiable receiver traces [nsteps, nrec] of ``solver`` for ``c2``."""
    return ReceiverTraces.apply(c2, solver, q0, dt, nsteps, checkpoint_every, t0)
