"""Algorithmic work of one step, counted from the CUDA step's arithmetic (an FMA counts 2 flops;
add, multiply, divide, square root and each of sine and cosine count 1).

Per world and step, with n_b bodies, n_v DOFs, n_a apples, E = sum_i d_i strict-ancestor
entries of the mass-matrix rows and P = sum_i d_i (d_i + 1) / 2 ancestor pairs (d_i the number
of DOF ancestors of DOF i):

  forward sweep   466 / body   (kinematics, velocities, bias acceleration, inertia, own force)
                  140 / apple  (tether loads, reaction, coupling point mass)
  backward sweep  106 / body   (child force and composite inertia shifts, bias, right-hand side)
  mass matrix      33 / DOF + 20 / ancestor entry
  LDL^T + L^T      3 / pair + 2 / ancestor entry + 2 / DOF
  L sweep, update  13 / DOF + 2 / ancestor entry + 17 / body + 42 / apple

  flops = 589 n_b + 182 n_a + 48 n_v + 24 E + 3 P.

Adjoint, per world and step of the backward pass (n_t tips): with checkpoints the segment
replay runs the forward step once more and saves its records (factors and kinematics
included), so the reverse recomputes nothing; with the forward's tape no step runs again. Then

  tape             51 / body + 19 / DOF   (the joint-acceleration and virtual-velocity parts; the
                                           kinematics come from the step's record)
  reverse sweep   978 / body + 189 / DOF + 246 / apple + 21 / tip
  apple update, springs, hang-load sweep and the solve with the step's factors:
                   21 / body + 30 / DOF + 48 / apple + 5 / ancestor entry

  flops = [1 x forward with checkpoints] + 1050 n_b + 238 n_v + 294 n_a + 5 E + 21 n_t.

Bytes: the persistent rollout keeps a world's temporaries on chip and re-reads its model from
L2, so the unavoidable HBM traffic per rollout is one read of the model and one read and write
of the state.
"""
from __future__ import annotations

import numpy as np

F_BODY = 589
F_APPLE = 182
F_DOF = 48
F_ENTRY = 24
F_PAIR = 3

A_BODY = 1050
A_DOF = 238
A_APPLE = 294
A_ENTRY = 5
A_TIP = 21

MODEL_BYTES_PER_BODY = 7 * 16   # 2 int4 (topology, joint rows) + 5 float4
MODEL_BYTES_PER_DOF = 0         # (the DOFs' rows are found through their body)
MODEL_BYTES_PER_ENTRY = 2       # uint16 ancestor id
MODEL_BYTES_PER_APPLE = 36      # 2 float4 + int
STATE_BYTES_PER_DOF = 8         # q, qd
STATE_BYTES_PER_BODY = 12       # broken, counter, break step
STATE_BYTES_PER_APPLE = 40      # x, v, detached, two counters, detach step


def dof_depths(forest) -> np.ndarray:
    """Number of DOF ancestors of every DOF (world-local trees, packed)."""
    out = np.zeros(forest.n_dofs, np.int64)
    i = 0
    for w in range(forest.n_worlds):
        b0, b1 = forest.body_off[w], forest.body_off[w + 1]
        par = forest.parent[b0:b1]
        nd = forest.ndof[b0:b1]
        top = np.full(b1 - b0, -1, np.int64)  # depth of the deepest DOF on the path to b
        for b in range(b1 - b0):
            d = top[par[b]] if par[b] >= 0 else -1
            for _ in range(nd[b]):
                d += 1
                out[i] = d
                i += 1
            top[b] = d
    return out


def world_terms(forest):
    """Per-world (n_b, n_v, n_a, E, P)."""
    d = dof_depths(forest)
    do = forest.dof_off
    nb, nv, na = forest.world_sizes()
    E = np.add.reduceat(d, do[:-1]) if forest.n_dofs else np.zeros(forest.n_worlds, np.int64)
    P = np.add.reduceat(d * (d + 1) // 2, do[:-1]) if forest.n_dofs else np.zeros(forest.n_worlds, np.int64)
    E = np.where(nv > 0, E, 0)
    P = np.where(nv > 0, P, 0)
    return nb.astype(np.int64), nv.astype(np.int64), na.astype(np.int64), E, P


def flops_per_step(forest) -> float:
    nb, nv, na, E, P = world_terms(forest)
    return float(np.sum(F_BODY * nb + F_APPLE * na + F_DOF * nv + F_ENTRY * E + F_PAIR * P))


def adjoint_flops_per_step(forest, replay=True) -> float:
    """Flops of one step of the backward pass: the reverse terms, plus with checkpoints the
    segment replay's forward step (whose records the reverse reads, so the step runs once more,
    not twice); with the forward's full tape (replay=False) no step runs again."""
    nb, nv, na, E, P = world_terms(forest)
    nt = np.diff(forest.tip_off).astype(np.int64)
    rev = float(np.sum(A_BODY * nb + A_DOF * nv + A_APPLE * na + A_ENTRY * E + A_TIP * nt))
    return (flops_per_step(forest) if replay else 0.0) + rev


def hbm_bytes_per_rollout(forest) -> float:
    nb, nv, na, E, P = world_terms(forest)
    model = MODEL_BYTES_PER_BODY * nb + MODEL_BYTES_PER_DOF * nv + MODEL_BYTES_PER_ENTRY * (E + nv) + \
        MODEL_BYTES_PER_APPLE * na
    state = STATE_BYTES_PER_DOF * nv + STATE_BYTES_PER_BODY * nb + STATE_BYTES_PER_APPLE * na
    return float(np.sum(model + 2 * state))


def body_count(forest) -> int:
    """Bodies of the metric: segment bodies plus apples."""
    return int(forest.n_bodies + forest.n_apples)
