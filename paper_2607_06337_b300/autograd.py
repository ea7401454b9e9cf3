"""Differentiable rollout: torch.autograd.Function over ot_rollout / ot_rollout_backward.

``tip_rollout(sim, k, kd, q0, qd0, n_steps, ckpt_every)`` runs ``n_steps`` steps of every world
of ``sim`` from the initial joint state (q0, qd0) with per-body stiffness k and damping kd
(Sec. IV-A, Eq. 4) and returns the recorded tip positions [n_steps, n_tips, 3]. Its backward
is the hand-written adjoint kernel, with the break and detach masks frozen as the forward
recorded them (the paper simulates forward only; differentiating the step is an addition of
this library): each checkpoint segment is recomputed forward and swept in reverse, or with
``ckpt_every`` 0 the forward keeps the full tape (ot_tape_bytes of device memory) and the
backward sweeps it in reverse without recomputing any step.

Apples start from the forest's initial apple state; all four inputs are float32 CUDA tensors.
The forward overwrites the model's k and kd and the state of ``sim``; the backward writes the
gains saved by its forward back into the model before it runs, so other rollouts may run
between the two.
"""
from __future__ import annotations

import numpy as np
import torch


class TipRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sim, k, kd, q0, qd0, n_steps: int, ckpt_every: int, step0: int = 0, tape_steps: int = 0):
        dev = sim.device
        for t in (k, kd, q0, qd0):
            if t.device != dev or t.dtype != torch.float32:
                raise ValueError("tip_rollout inputs must be float32 tensors on the simulator's device")
        k = k.detach().contiguous()
        kd = kd.detach().contiguous()
        q0c = q0.detach().contiguous()
        qd0c = qd0.detach().contiguous()
        f = sim.forest
        ax = torch.as_tensor(np.asarray(f.apple_x0, np.float32).reshape(-1, 3), device=dev).contiguous()
        av = torch.as_tensor(np.asarray(f.apple_v0, np.float32).reshape(-1, 3), device=dev).contiguous()
        sim.set_gains(k, kd)
        sim.reset_from_device(q0c, qd0c, ax, av)
        tips, buffers, rec = sim.record_buffers(n_steps, ckpt_every, tape_steps=tape_steps)
        sim.rollout(n_steps, step0=step0, record=rec)
        ctx.sim = sim
        ctx.rec = rec
        ctx.buffers = buffers  # the record's device memory, alive until the backward
        ctx.meta = (n_steps, step0)
        ctx.save_for_backward(k, kd)
        return tips

    @staticmethod
    def backward(ctx, dtips):
        k, kd = ctx.saved_tensors
        sim = ctx.sim
        n_steps, step0 = ctx.meta
        sim.set_gains(k, kd)
        dk, dkd, dq0, dqd0 = sim.backward(n_steps, ctx.rec, dtips.to(torch.float32).contiguous(), step0=step0)
        return None, dk, dkd, dq0, dqd0, None, None, None, None


def tip_rollout(sim, k, kd, q0, qd0, n_steps: int, ckpt_every=None, step0: int = 0):
    """Tip positions [n_steps, n_tips, 3] of a rollout, differentiable in k, kd, q0 and qd0.

    ckpt_every: checkpoint interval of the record, or 0 for the forward's full tape. None takes
    the full tape when it needs at most a quarter of the free device memory, else a tape of as
    many final steps as fit there with checkpoints every 20 steps before them (or checkpoints
    alone when not even one step fits)."""
    tape_steps = 0
    if ckpt_every is None:
        from .orchard import tape_bytes
        free, _ = torch.cuda.mem_get_info(sim.device)
        budget = free // 4
        if tape_bytes(sim.model, int(n_steps)) <= budget:
            ckpt_every = 0
        else:
            ckpt_every = 20
            tape_steps = max(0, min(int(n_steps) - 1, budget // tape_bytes(sim.model, 0) - 1))
    return TipRollout.apply(sim, k, kd, q0, qd0, int(n_steps), int(ckpt_every), int(step0), int(tape_steps))


def tip_loss(tips, target, tip_off):
    """Tip-tracking loss summed over worlds: per world, sum over steps and tips of |p - p*|^2
    divided by (n_steps * that world's tip count). tip_off: per-world tip offsets [W+1]."""
    n_steps = tips.shape[0]
    counts = np.diff(np.asarray(tip_off))
    scale = 1.0 / (n_steps * np.maximum(counts, 1))
    w = torch.as_tensor(np.repeat(scale, counts), dtype=tips.dtype, device=tips.device)
    return (((tips - target) ** 2).sum(-1) * w).sum()
