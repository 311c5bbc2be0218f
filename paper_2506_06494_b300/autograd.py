"""torch.autograd wrappers of the JGS2 step and its adjoint (argument marshalling only).

JGS2Step.apply(mesh, x_t, v_t, E) -> (x_{t+1}, v_{t+1}): forward = jgs2_step with per-tet
Young's moduli E; backward = jgs2_step_adjoint (dL/dx_t, dL/dv_t, dL/dE).

rollout(mesh, x0, v0, E, n_steps, checkpoint_every) runs n_steps steps keeping only every
checkpoint_every-th state; its backward recomputes each segment forward from its
checkpoint and runs the step adjoints in reverse.

The adjoint is the implicit-function theorem at grad E(x_{t+1}) = 0, so it is only the
derivative of the step when the forward step converged. A forward step that stops on its
sweep cap (JGS2_ENOTCONVERGED) or on the position-change test raises NotConvergedError,
unless allow_unconverged=True (e.g. for timing runs; the gradient then has no meaning).
"""
from __future__ import annotations

import numpy as np
import torch

from . import jgs2 as J


def _set_E(mesh, E):
    mesh.set_youngs(E.detach().to("cpu", torch.float64).numpy())


class NotConvergedError(RuntimeError):
    """A forward step did not reach its residual tolerance: its adjoint would be wrong."""


def _step(mesh, x, v, opts, allow_unconverged=False):
    x = x.detach().clone().contiguous()
    v = v.detach().clone().contiguous()
    rep = mesh.step(x, v, opts)
    if not rep.converged and not allow_unconverged:
        raise NotConvergedError(f"forward step stopped after {rep.sweeps} sweeps at relative residual "
                                f"{rep.rel_residual:.3e} without reaching rel_tol: the implicit-function "
                                "adjoint needs a converged step")
    return x, v, rep


class JGS2Step(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mesh, x_t, v_t, E, opts=None, adj_opts=None, allow_unconverged=False):
        _set_E(mesh, E)
        x1, v1, _ = _step(mesh, x_t, v_t, opts, allow_unconverged)
        ctx.mesh, ctx.adj_opts = mesh, adj_opts
        ctx.save_for_backward(x_t.detach(), v_t.detach(), x1, E.detach())
        return x1, v1

    @staticmethod
    def backward(ctx, gx1, gv1):
        x_t, v_t, x1, E = ctx.saved_tensors
        mesh = ctx.mesh
        _set_E(mesh, E)
        gx1 = torch.zeros_like(x1) if gx1 is None else gx1.contiguous()
        gv1 = torch.zeros_like(x1) if gv1 is None else gv1.contiguous()
        gx, gv, gE, _ = mesh.step_adjoint(x_t, v_t, x1, gx1, gv1, opts=ctx.adj_opts)
        return None, gx, gv, gE, None, None, None


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mesh, x0, v0, E, n_steps, every, opts, adj_opts, allow_unconverged):
        _set_E(mesh, E)
        ckpt = [(x0.detach().clone(), v0.detach().clone())]
        x, v = ckpt[0]
        for k in range(n_steps):
            x, v, _ = _step(mesh, x, v, opts, allow_unconverged)
            if (k + 1) % every == 0 and k + 1 < n_steps:
                ckpt.append((x.clone(), v.clone()))
        ctx.mesh, ctx.n, ctx.every, ctx.opts, ctx.adj_opts = mesh, n_steps, every, opts, adj_opts
        ctx.allow = allow_unconverged
        ctx.ckpt = ckpt
        ctx.save_for_backward(E.detach())
        return x, v

    @staticmethod
    def backward(ctx, gxn, gvn):
        (E,) = ctx.saved_tensors
        mesh = ctx.mesh
        _set_E(mesh, E)
        gx = torch.zeros_like(ctx.ckpt[0][0]) if gxn is None else gxn.contiguous().clone()
        gv = torch.zeros_like(ctx.ckpt[0][0]) if gvn is None else gvn.contiguous().clone()
        gE = torch.zeros(mesh.T, dtype=torch.float64, device=gx.device)
        n, every = ctx.n, ctx.every
        for seg in reversed(range(len(ctx.ckpt))):
            start = seg * every
            stop = min(start + every, n)
            # recompute the segment's states from its checkpoint
            states = [ctx.ckpt[seg]]
            for _ in range(start, stop):
                states.append(_step(mesh, *states[-1], ctx.opts, ctx.allow)[:2])
            for k in reversed(range(stop - start)):
                (xt, vt), (x1, _) = states[k], states[k + 1]
                gx, gv, gE, _ = mesh.step_adjoint(xt, vt, x1, gx, gv, gE=gE, opts=ctx.adj_opts)
        return None, gx, gv, gE, None, None, None, None, None


def rollout(mesh, x0, v0, E, n_steps, checkpoint_every=5, opts=None, adj_opts=None, allow_unconverged=False):
    return _Rollout.apply(mesh, x0, v0, E, int(n_steps), int(checkpoint_every), opts, adj_opts,
                          bool(allow_unconverged))


__all__ = ["JGS2Step", "rollout", "NotConvergedError", "np", "J"]
