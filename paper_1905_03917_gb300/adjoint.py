"""Gradients through the single-time-step method.

``FrozenSteps`` is a ``torch.autograd.Function`` from the primitive
initial fields of both fluids to the conserved state after ``nsteps``
single-time-step RK2 steps.  Its backward is the discrete adjoint of each
step with that step's schedule frozen (dt, Lax-Friedrichs speeds, level
sets: the interface topology does not move under the perturbation),
computed by libsif's ``sif_adjoint_step`` and ``sif_adjoint_init``.

Memory: the forward keeps a checkpoint every ``every`` steps (host bytes of
``sif_save``) and records the tape of its last segment (device memory,
36 planes of the padded grid a step); the backward walks that segment's adjoint steps in
reverse straight away, then for every earlier segment restores its
checkpoint, re-runs it while recording its tape (bitwise the same steps)
and walks its adjoint steps.  ``every >= nsteps`` records the whole run in
the forward and recomputes nothing: on a GB300 the tape of 200 steps of a
512^2 grid takes 16 GB of its HBM.

Arithmetic runs in libsif; this module only orders the calls and holds
device buffers.
"""
from __future__ import annotations

import torch

from . import sif


class FrozenSteps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, prim_N, prim_P, solver, phi, nsteps, every):
        if prim_N.device.type != "cuda":
            raise ValueError("FrozenSteps runs on CUDA tensors")
        prim_N = prim_N.detach().contiguous()
        prim_P = prim_P.detach().contiguous()
        phi = phi.detach().contiguous()
        solver.tape_reset(0)
        solver.init_fluids(phi, prim_N, prim_P)
        ckpts, lengths = [], []
        done = 0
        while done < nsteps:
            n = min(every, nsteps - done)
            ckpts.append(solver.save())
            lengths.append(n)
            if done + n == nsteps:
                solver.tape_reset(n)  # the last segment is recorded as it runs
            solver.step_single_dt(n)
            done += n
        ny, nx = solver.ny, solver.nx
        q = torch.empty((2, 4, ny, nx), dtype=torch.float64, device=prim_N.device)
        phi_end = torch.empty((ny, nx), dtype=torch.float64, device=prim_N.device)
        solver.state_into(q[0], q[1], phi_end)
        ctx.solver, ctx.ckpts, ctx.lengths, ctx.every = solver, ckpts, lengths, every
        ctx.save_for_backward(prim_N, prim_P, phi)
        ctx.mark_non_differentiable(phi_end)
        return q, phi_end

    @staticmethod
    def backward(ctx, grad_q, grad_phi):
        solver = ctx.solver
        prim_N, prim_P, phi = ctx.saved_tensors
        lam = grad_q.detach().contiguous().clone()
        end_state = solver.save()
        last = True
        for ckpt, n in zip(reversed(ctx.ckpts), reversed(ctx.lengths)):
            # the last segment's tape is still there from the forward
            if not (last and n > 0 and solver.tape_length == n):
                solver.load_checkpoint(ckpt)
                solver.tape_reset(max(n, 1))
                solver.step_single_dt(n)
            last = False
            for s in reversed(range(n)):
                solver.adjoint_step(s, lam, lam)
        solver.tape_reset(0)
        lam_prim = torch.empty_like(lam)
        solver.adjoint_init(phi, prim_N, prim_P, lam, lam_prim)
        solver.load_checkpoint(end_state)
        return lam_prim[0], lam_prim[1], None, None, None, None


def frozen_steps(solver: "sif.Solver", phi, prim_N, prim_P, nsteps: int, every: int = 20):
    """State (2, 4, ny, nx) and level set after nsteps single-dt steps from
    the primitive fields; differentiable with respect to prim_N and prim_P."""
    return FrozenSteps.apply(prim_N, prim_P, solver, phi, int(nsteps), int(every))


def wall_pressure(q, cfg):
    """J = sum over the cells of the +x wall column of the fluid-P pressure
    times dy, for a wall column that holds fluid P only (volume fraction
    one), from the conserved state q (2, 4, ny, nx)."""
    g, pi = cfg["gamma"][1], cfg["pinf"][1]
    w = q[1, :, :, -1]
    rho, mx, my, E = w[0], w[1], w[2], w[3]
    p = (g - 1.0) * (E - 0.5 * (mx * mx + my * my) / rho) - g * pi
    return p.sum() * cfg["dy"]
