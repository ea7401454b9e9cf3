"""Adjoint kernel (ot_rollout_backward, and the autograd wrapper over it) against the FP64
oracle's complex-step derivative and central finite differences of the tip-tracking loss.

Tolerances, per kind of coordinate (k, kd, q0, qd0) and per world, relative to the largest
sampled magnitude of that kind:

* far target (tips + 1 cm noise): 1e-3 against the complex-step derivative. With residuals of
  1 cm the FP32 tip error (~1e-7 m) is irrelevant, so this bounds the adjoint's own rounding;
  the serial FP32 evaluation of the same arithmetic lands within 2.4e-4.
* the differentiation workload's target (the oracle's rollout with k scaled by U(0.8, 1.2)):
  residuals are only ~2e-4 m, so the loss is resolved only to the ratio r of the FP32 tips'
  error to the residual (rms over the rollout, measured per world, ~3e-4), and the gradient is
  a sum of per-step residual-weighted terms that cancel heavily for some coordinates (q0
  above all), which multiplies the adjoint's own ~1e-4 rounding. Measured: up to 4.4e-3 on
  q0 with r = 2.9e-4. The oracle's own gradient evaluated with every operation in FP32
  (single-precision complex step, tests/test_oracle_grad.py) is off by 2.6e-3 on the same
  worlds and coordinates, against 2.0e-4 for the far target: that rounding floor, not the
  adjoint, sets the bound. Bound: 1e-2 against complex step, 1.5e-2 against central
  differences (which add their own O(h^2) error). The far-target test above is the sharp
  check of the adjoint.
"""

import numpy as np
import pytest

import oracle as O
from paper_2607_06337_b300 import inputs as I
from tests import parity as PAR
from tests.test_oracle_grad import fd_steps, perturbed_target, sample_coords

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("oracle_lib")]

TOL_FAR = 1e-3


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def tip_cotangent(f, tips, target):
    """dL/dtips (float64 tensors) of L = sum over worlds of sum_t sum_tips |p - p*|^2 / (n_steps
    n_tips_of_world)."""
    torch = _torch()
    n = tips.shape[0]
    counts = np.diff(f.tip_off)
    scale = torch.as_tensor(np.repeat(1.0 / (n * np.maximum(counts, 1)), counts), device=tips.device)
    return 2.0 * (tips - target) * scale[None, :, None]


def gpu_gradients(f, fl, n, ckpt_every, target, sim=None, tape_steps=0):
    torch = _torch()
    from paper_2607_06337_b300.orchard import Simulator
    sim = sim or Simulator(f, fl)
    sim.reset()
    tips, ck, rec = sim.record_buffers(n, ckpt_every, tape_steps=tape_steps)
    sim.rollout(n, record=rec)
    tg = torch.as_tensor(np.asarray(target, np.float32), device="cuda")
    dt = tip_cotangent(f, tips.double(), tg.double()).float()
    grads = sim.backward(n, rec, dt)
    torch.cuda.synchronize()
    sim.last_tips = tips.cpu().numpy().astype(np.float64)
    g = [x.cpu().numpy().astype(np.float64) for x in grads]
    ev = dict(broken=sim.broken.cpu().numpy(), break_step=sim.break_step.cpu().numpy(),
              detached=sim.detached.cpu().numpy(), detach_step=sim.detach_step.cpu().numpy())
    return g, ev, sim


def pick(f, w, g, kinds, idx):
    b0, d0 = f.body_off[w], f.dof_off[w]
    return np.array([g[k][(b0 if k < 2 else d0) + i] for k, i in zip(kinds, idx)])


def assert_close_per_kind(got, ref, kinds, tol, what, dt=0.0):
    """Per kind of coordinate, the error against its largest sampled magnitude. With dt > 0 the
    scale of the qd0 kind is at least dt times the q0 kind's: a velocity at step 0 is, to first
    order, a displacement dt later, so dL/dqd0 holds dt dL/dq0 and inherits dt times q0's
    rounding floor (on the +-20% target the qd0 gradients are about that size)."""
    for kind in range(4):
        s = kinds == kind
        if not s.any():
            continue
        scale = np.abs(ref[s]).max()
        if kind == 3 and dt > 0 and (kinds == 2).any():
            scale = max(scale, dt * np.abs(ref[kinds == 2]).max())
        err = np.abs(got[s] - ref[s]).max()
        assert err <= tol * scale + 1e-30, (
            f"{what}: {['k', 'kd', 'q0', 'qd0'][kind]} max err {err:.3e} vs scale {scale:.3e}\n"
            f"got {got[s]}\nref {ref[s]}")


def test_adjoint_differentiation_workload_against_oracle():
    """Four worlds of the differentiation workload (200 bodies, 30 apples, a fixed 5 N pull),
    200 steps, checkpoints every 20 steps; target from the oracle with k perturbed by +-20%."""
    f = I.make_forest(I.DIFF, worlds=[0, 1, 2, 3])
    fl = I.Flags()
    n = 200
    target = perturbed_target(f, fl, n)
    _, rec0 = O.rollout(f, fl, n, record_tips=True)
    g, _, sim = gpu_gradients(f, fl, n, 20, target)
    rng = np.random.default_rng(5)
    for w in range(f.n_worlds):
        t0, t1 = f.tip_off[w], f.tip_off[w + 1]
        tw = target[:, t0:t1]
        tips_gpu = sim.last_tips[:, t0:t1]
        r = np.sqrt(((tips_gpu - rec0["tips"][:, t0:t1]) ** 2).mean() / ((rec0["tips"][:, t0:t1] - tw) ** 2).mean())
        assert r < 2e-3, f"world {w}: FP32 tips off by {r:.2e} of the residual"
        tol = 1e-2
        kinds, idx = sample_coords(f, w, 4, rng)
        g_cs, _ = O.grad(f, fl, w, n, tw, kinds, idx, np.full(len(kinds), 1e-20), mode=0)
        got = pick(f, w, g, kinds, idx)
        assert_close_per_kind(got, g_cs, kinds, tol, f"world {w} vs complex step (r = {r:.2e})")
        if w == 0:
            g_fd, _ = O.grad(f, fl, w, n, tw, kinds, idx, fd_steps(f, w, kinds, idx), mode=1)
            assert_close_per_kind(got, g_fd, kinds, 1.5 * tol, f"world {w} vs central differences")


@pytest.mark.parametrize("target_kind", ["far", "perturbed"])
def test_adjoint_eight_worlds_64_coordinates_against_central_differences(target_kind):
    """The differentiation workload's gradient check at its stated size: 8 worlds x 64 random
    coordinates (16 each of k, kd, q0, qd0), against FP64 central differences of the oracle
    (1e-3 relative steps), with checkpoints every 20 steps. Far target (tips + 1 cm noise):
    1e-3 per kind, the sharp check. The workload's own +-20% stiffness target: 1.5e-2 per kind,
    the 1e-2 rounding floor of that gradient (module docstring) plus the differences' own
    O(h^2) error. qd0 is scaled as in assert_close_per_kind (dt times q0's floor)."""
    f = I.make_forest(I.DIFF, worlds=[0, 1, 2, 3, 200, 401, 702, 1023])
    fl = I.Flags()
    n = 200
    if target_kind == "far":
        _, rec0 = O.rollout(f, fl, n, record_tips=True)
        target = rec0["tips"] + np.random.default_rng(31).normal(0.0, 0.01, rec0["tips"].shape)
        tol = TOL_FAR
    else:
        target = perturbed_target(f, fl, n)
        tol = 1.5e-2
    g, _, _ = gpu_gradients(f, fl, n, 20, target)
    rng = np.random.default_rng(64)
    for w in range(f.n_worlds):
        tw = target[:, f.tip_off[w]:f.tip_off[w + 1]]
        kinds, idx = sample_coords(f, w, 16, rng)
        assert len(kinds) == 64
        g_fd, _ = O.grad(f, fl, w, n, tw, kinds, idx, fd_steps(f, w, kinds, idx), mode=1)
        assert_close_per_kind(pick(f, w, g, kinds, idx), g_fd, kinds, tol, f"world {w} vs central differences",
                              dt=fl.dt)


def test_adjoint_far_target_bounds_the_adjoint_rounding():
    """The same worlds against a target 1 cm away (noise on the oracle's own tips): the loss is
    well resolved in FP32, so the adjoint must match the complex-step derivative to 1e-3."""
    f = I.make_forest(I.DIFF, worlds=[0, 1, 2, 3])
    fl = I.Flags()
    n = 200
    _, rec0 = O.rollout(f, fl, n, record_tips=True)
    rng = np.random.default_rng(3)
    target = rec0["tips"] + rng.normal(0.0, 0.01, rec0["tips"].shape)
    g, _, _ = gpu_gradients(f, fl, n, 20, target)
    for w in range(f.n_worlds):
        kinds, idx = sample_coords(f, w, 6, rng)
        tw = target[:, f.tip_off[w]:f.tip_off[w + 1]]
        g_cs, _ = O.grad(f, fl, w, n, tw, kinds, idx, np.full(len(kinds), 1e-20), mode=0)
        assert_close_per_kind(pick(f, w, g, kinds, idx), g_cs, kinds, TOL_FAR, f"world {w} far target")


def test_adjoint_with_breaks_and_detaches_masks_frozen():
    """Worlds of the batching workload in which a branch breaks and apples detach within 200
    steps: with the masks frozen as recorded, the adjoint matches the oracle's complex-step
    derivative (whose real part, and so every event, is that of the unperturbed rollout)."""
    f = I.make_forest(I.BATCH, worlds=[23, 79])
    fl = I.Flags()
    n = 200
    st, rec = O.rollout(f, fl, n, record_tips=True, near_eps=PAR.NEAR)
    assert st.broken.sum() > 0 and (st.detached > 0).sum() > 0
    rng = np.random.default_rng(2)
    target = rec["tips"] + rng.normal(0.0, 0.02, rec["tips"].shape)
    g, ev, _ = gpu_gradients(f, fl, n, 25, target)
    for w in range(f.n_worlds):
        ref_ev = PAR.events(st.broken, st.break_step, st.detached, st.detach_step, f, w)
        got_ev = PAR.events(ev["broken"], ev["break_step"], ev["detached"], ev["detach_step"], f, w)
        assert got_ev == ref_ev, f"world {w}: event sets differ, the gradients are not comparable"
        kinds, idx = sample_coords(f, w, 4, rng)
        tw = target[:, f.tip_off[w]:f.tip_off[w + 1]]
        g_cs, _ = O.grad(f, fl, w, n, tw, kinds, idx, np.full(len(kinds), 1e-20), mode=0)
        assert_close_per_kind(pick(f, w, g, kinds, idx), g_cs, kinds, 2e-3, f"world {w} with events")


def test_adjoint_with_body_damping_and_events():
    """Velocity-proportional body damping on (Sec. IV-A), with the linear part reduced on snapped
    sub-trees (Sec. IV-B), in worlds where branches break and apples detach: the adjoint of the
    damping wrench against the oracle's complex-step derivative, masks frozen."""
    f = I.make_forest(I.BATCH, worlds=[23, 79])
    fl = I.Flags(lin_damping=3.0, ang_damping=2.0, snapped_lin_damping=0.2)
    n = 200
    st, rec = O.rollout(f, fl, n, record_tips=True, near_eps=PAR.NEAR)
    assert st.broken.sum() > 0
    rng = np.random.default_rng(4)
    target = rec["tips"] + rng.normal(0.0, 0.02, rec["tips"].shape)
    g, ev, _ = gpu_gradients(f, fl, n, 25, target)
    for w in range(f.n_worlds):
        ref_ev = PAR.events(st.broken, st.break_step, st.detached, st.detach_step, f, w)
        got_ev = PAR.events(ev["broken"], ev["break_step"], ev["detached"], ev["detach_step"], f, w)
        assert got_ev == ref_ev, f"world {w}: event sets differ, the gradients are not comparable"
        kinds, idx = sample_coords(f, w, 4, rng)
        tw = target[:, f.tip_off[w]:f.tip_off[w + 1]]
        g_cs, _ = O.grad(f, fl, w, n, tw, kinds, idx, np.full(len(kinds), 1e-20), mode=0)
        assert_close_per_kind(pick(f, w, g, kinds, idx), g_cs, kinds, 2e-3, f"world {w} with damping")


def test_adjoint_through_the_applied_force_rails():
    """The rails' Jacobian in the adjoint: a low speed limit (2 cm/s) puts the pulled apple of
    each differentiation-workload tree in the cap, fade and brake regimes while attached; the
    gradients against the oracle's complex-step derivative (far target)."""
    f = I.make_forest(I.DIFF, worlds=[0, 1])
    fl = I.Flags(rail_speed=0.02, rail_fade_speed=0.005, rail_brake=20.0)
    n = 100
    _, rec = O.rollout(f, fl, n, record_tips=True)
    off, _ = O.rollout(f, I.Flags(), n)
    on, _ = O.rollout(f, fl, n)
    assert np.abs(on.av - off.av).max() > 1e-3  # the rails act
    rng = np.random.default_rng(6)
    target = rec["tips"] + rng.normal(0.0, 0.01, rec["tips"].shape)
    g, _, _ = gpu_gradients(f, fl, n, 20, target)
    for w in range(f.n_worlds):
        kinds, idx = sample_coords(f, w, 5, rng)
        tw = target[:, f.tip_off[w]:f.tip_off[w + 1]]
        g_cs, _ = O.grad(f, fl, w, n, tw, kinds, idx, np.full(len(kinds), 1e-20), mode=0)
        assert_close_per_kind(pick(f, w, g, kinds, idx), g_cs, kinds, TOL_FAR, f"world {w} with rails")


def test_damper_gradient_of_a_joint_without_damper():
    """dL/dkd of a joint whose kd is 0 (the compliant root of a small tree): the step's damper
    is kd' = kd (times the post-break factor), so the derivative is that of kd', not zero."""
    from tests import _trees as T
    f = T.small_random_tree(2, n_b=7, depth=3, ndof=2, root_ndof=2)
    assert f.kd[0] == 0.0
    fl = I.Flags()
    n = 60
    _, rec = O.rollout(f, fl, n, record_tips=True)
    target = rec["tips"] + np.random.default_rng(8).normal(0.0, 0.01, rec["tips"].shape)
    g, _, _ = gpu_gradients(f, fl, n, 20, target)
    kinds = np.array([1] * f.n_bodies)
    idx = np.arange(f.n_bodies)
    g_cs, _ = O.grad(f, fl, 0, n, target, kinds, idx, np.full(len(kinds), 1e-20), mode=0)
    assert abs(g_cs[0]) > 1e-3 * np.abs(g_cs).max()
    assert_close_per_kind(pick(f, 0, g, kinds, idx), g_cs, kinds, TOL_FAR, "kd with a zero damper")


def test_checkpoint_interval_does_not_change_the_gradient():
    """Every checkpoint interval, including one that does not divide the step count and one
    longer than the rollout, gives the same gradient: the replayed segments run the forward's
    step code (compiled into another kernel, so equal up to the last bits of each step, not
    bitwise), and the gradients agree to 1e-5 of each kind's largest entry."""
    f = I.make_forest(I.DIFF, worlds=[7, 8])
    fl = I.Flags()
    n = 50
    target = perturbed_target(f, fl, n)
    ref, _, sim = gpu_gradients(f, fl, n, 1, target)
    for ce in (7, 20, 50, 64):
        got, _, _ = gpu_gradients(f, fl, n, ce, target, sim=sim)
        for a, b in zip(got, ref):
            np.testing.assert_allclose(a, b, rtol=0, atol=1e-5 * np.abs(b).max())


@pytest.mark.parametrize("worlds,workload,n", [([7, 8], I.DIFF, 120), ([23, 79], I.BATCH, 120),
                                                ([0, 4096, 8000], I.STRESS, 30)])
def test_tape_gives_the_checkpointed_gradient(worlds, workload, n):
    """The forward's full tape (no step run again), and a tape of the final third of the steps
    with checkpoints before it, against checkpoints every step and every 25 steps: the same gradient up to the last bits of each step (the backward's replay is
    compiled into another kernel and may run at another group size), within 1e-5 of each
    kind's largest entry. The batching worlds break branches and drop apples on the way; the
    stress worlds (50, 400 and 2000 bodies) include one whose step temporaries are in global
    memory, with FP64 pivots on twigs under 5 mm."""
    f = I.make_forest(workload, worlds=worlds)
    fl = I.Flags(fp64_twig_diam=0.005 if workload == I.STRESS else 0.0)
    _, rec0 = O.rollout(f, fl, n, record_tips=True)
    target = rec0["tips"] + np.random.default_rng(9).normal(0.0, 0.01, rec0["tips"].shape)
    tape, _, sim = gpu_gradients(f, fl, n, 0, target)
    # the hybrid record: a tape of the final steps (a number that splits a checkpoint segment),
    # checkpoints every 25 steps before them
    hybrid, _, _ = gpu_gradients(f, fl, n, 25, target, sim=sim, tape_steps=n // 3 + 1)
    for ce in (1, 25):
        ref, _, _ = gpu_gradients(f, fl, n, ce, target, sim=sim)
        for got in (tape, hybrid):
            for a, b in zip(got, ref):
                np.testing.assert_allclose(a, b, rtol=0, atol=1e-5 * np.abs(b).max())


@pytest.mark.parametrize("n,step0,tape_steps", [(40, 137, 0), (1, 0, 0), (9, 3, 1)])
def test_tape_edge_cases_against_checkpoints(n, step0, tape_steps):
    """The tape's records keep absolute step indices (the pull schedule reads them): a rollout
    starting at step 137; a one-step rollout; a hybrid with a single taped step. Each against
    the checkpointed gradient of the same rollout (checkpoints every 4 steps), to 1e-5 of each
    kind's largest entry."""
    torch = _torch()
    from paper_2607_06337_b300.orchard import Simulator
    f = I.make_forest(I.DIFF, worlds=[3, 4])
    fl = I.Flags()
    sim = Simulator(f, fl)
    _, rec0 = O.rollout(f, fl, n, record_tips=True, step0=step0)
    target = torch.as_tensor(rec0["tips"] + 0.01, device="cuda")

    def grads(ce, k):
        sim.reset()
        tips, buf, rec = sim.record_buffers(n, ce, tape_steps=k)
        sim.rollout(n, step0=step0, record=rec)
        dt = tip_cotangent(f, tips.double(), target).float()
        g = sim.backward(n, rec, dt, step0=step0)
        torch.cuda.synchronize()
        return [x.cpu().numpy().astype(np.float64) for x in g], tips.cpu().numpy()

    ref, tips_ref = grads(4, 0)
    got, tips_got = grads(4 if tape_steps else 0, tape_steps)
    np.testing.assert_array_equal(tips_got, tips_ref)
    for a, b in zip(got, ref):
        assert np.abs(b).max() > 0
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-5 * np.abs(b).max())


def test_tape_of_a_frozen_world_gives_nan_gradients_only_there():
    """A world whose state is non-finite from the start is frozen by the forward: with the tape
    its gradients are NaN, and the other world's are those of the checkpointed backward."""
    torch = _torch()
    f = I.make_forest(I.PLAIN, worlds=[0, 1])
    f.q0 = f.q0.copy()
    f.q0[f.dof_off[1] + 3] = np.nan
    fl = I.Flags()
    n = 30
    _, rec0 = O.rollout(f.subset([0]), fl, n, record_tips=True)
    target = np.zeros((n, f.n_tips, 3))
    target[:, :f.tip_off[1]] = rec0["tips"] + 0.01
    tape, _, sim = gpu_gradients(f, fl, n, 0, target)
    ref, _, _ = gpu_gradients(f, fl, n, 10, target, sim=sim)
    b1, d1 = f.body_off[1], f.dof_off[1]
    for k, (a, b) in enumerate(zip(tape, ref)):
        cut = b1 if k < 2 else d1
        assert np.all(np.isnan(a[cut:])), k
        np.testing.assert_allclose(a[:cut], b[:cut], rtol=0, atol=1e-5 * np.abs(b[:cut]).max())


def test_tape_buffer_checks():
    """A tape one float too small, or not on a 16-byte boundary, is refused (OT_EINVAL) by the
    rollout and by the backward before any work is queued; so is a tape of the final steps
    without checkpoints, or of more steps than the rollout."""
    torch = _torch()
    from paper_2607_06337_b300 import orchard as B
    f = I.make_forest(I.DIFF, worlds=[0])
    sim = B.Simulator(f, I.Flags())
    n = 8
    need = B.tape_bytes(sim.model, n)
    assert need > 0 and need % 16 == 0
    buf = torch.empty(need + 64, dtype=torch.uint8, device="cuda")
    tips = torch.empty((n, sim.counts.tips, 3), dtype=torch.float32, device="cuda")
    for ptr, nbytes in ((buf.data_ptr(), need - 4), (buf.data_ptr() + 4, need)):
        rec = B.Record(tips.data_ptr(), None, 0, 0, ptr, nbytes, 0)
        with pytest.raises(B.OrchardError) as e:
            sim.rollout(n, record=rec)
        assert e.value.status == B.OT_EINVAL
        with pytest.raises(B.OrchardError) as e:
            sim.backward(n, rec, torch.zeros_like(tips))
        assert e.value.status == B.OT_EINVAL
    # a tape of the final steps only needs checkpoints for the others; more steps than the
    # rollout are refused
    for steps in (3, n + 1):
        rec = B.Record(tips.data_ptr(), None, 0, 0, buf.data_ptr(), need, steps)
        with pytest.raises(B.OrchardError) as e:
            sim.rollout(n, record=rec)
        assert e.value.status == B.OT_EINVAL
    sim.rollout(n, record=B.Record(tips.data_ptr(), None, 0, 0, buf.data_ptr(), need, 0))
    torch.cuda.synchronize()


def test_autograd_function_matches_the_direct_call():
    """tip_rollout + tip_loss + loss.backward() gives the gradients of ot_rollout_backward, and
    the forward returns the tips of a plain recorded rollout."""
    torch = _torch()
    from paper_2607_06337_b300.autograd import tip_loss, tip_rollout
    f = I.make_forest(I.DIFF, worlds=[9, 10, 11])
    fl = I.Flags()
    n = 60
    target = perturbed_target(f, fl, n).astype(np.float32).astype(np.float64)  # same bits on both paths
    g_ref, _, sim = gpu_gradients(f, fl, n, 20, target)
    dev = "cuda"
    k = torch.tensor(f.k, dtype=torch.float32, device=dev, requires_grad=True)
    kd = torch.tensor(f.kd, dtype=torch.float32, device=dev, requires_grad=True)
    q0 = torch.tensor(f.q0, dtype=torch.float32, device=dev, requires_grad=True)
    qd0 = torch.tensor(f.qd0, dtype=torch.float32, device=dev, requires_grad=True)
    tips = tip_rollout(sim, k, kd, q0, qd0, n, ckpt_every=20)
    loss = tip_loss(tips.double(), torch.as_tensor(target, device=dev), f.tip_off)
    loss.backward()
    for t, r in zip((k, kd, q0, qd0), g_ref):
        np.testing.assert_allclose(t.grad.cpu().numpy(), r, rtol=0, atol=1e-5 * np.abs(r).max())
    # the loss itself agrees with the oracle's at the unperturbed gains
    lo = sum(O.grad(f, fl, w, n, target[:, f.tip_off[w]:f.tip_off[w + 1]], [2], [0], [1e-20], mode=0)[1]
             for w in range(f.n_worlds))
    assert float(loss.detach()) == pytest.approx(lo, rel=1e-3)
    # a second forward with scaled gains changes the tips; its backward uses its own gains
    k2 = (k.detach() * 1.1).requires_grad_(True)
    tips2 = tip_rollout(sim, k2, kd.detach(), q0.detach(), qd0.detach(), n, ckpt_every=20)
    assert not torch.equal(tips2, tips)
    # the full tape (ckpt_every 0): the same tips and gradients
    grads = [t.grad.clone() for t in (k, kd, q0, qd0)]
    for t in (k, kd, q0, qd0):
        t.grad = None
    tips3 = tip_rollout(sim, k, kd, q0, qd0, n, ckpt_every=0)
    assert torch.equal(tips3, tips)
    assert torch.equal(tip_rollout(sim, k.detach(), kd.detach(), q0.detach(), qd0.detach(), n), tips)  # default
    tip_loss(tips3.double(), torch.as_tensor(target, device=dev), f.tip_off).backward()
    for t, r in zip((k, kd, q0, qd0), grads):
        np.testing.assert_allclose(t.grad.cpu().numpy(), r.cpu().numpy(), rtol=0, atol=1e-5 * r.abs().max().item())
    # the hybrid record (a tape of the last 25 steps, checkpoints every 20 before them), the
    # default's choice when the full tape does not fit
    from paper_2607_06337_b300.autograd import TipRollout
    for t in (k, kd, q0, qd0):
        t.grad = None
    tips4 = TipRollout.apply(sim, k, kd, q0, qd0, n, 20, 0, 25)
    assert torch.equal(tips4, tips)
    tip_loss(tips4.double(), torch.as_tensor(target, device=dev), f.tip_off).backward()
    for t, r in zip((k, kd, q0, qd0), grads):
        np.testing.assert_allclose(t.grad.cpu().numpy(), r.cpu().numpy(), rtol=0, atol=1e-5 * r.abs().max().item())


@pytest.mark.parametrize("ckpt_every", [16, 0])
def test_full_gradient_against_the_oracle_reverse_mode(ckpt_every):
    """Every coordinate of the gradient against the oracle's own FP64 adjoint (its reverse-mode
    tape): six generated 24-body trees with 6 apples each and a 12-body tree in which a joint
    breaks and an apple detaches (masks frozen as recorded), 150 steps, checkpoints every 16 or
    the forward's full tape (0), a target 1 cm away. Per world and kind: |g - g_ref|_2 <= 1e-3
    |g_ref|_2, and the largest entry error within 2e-3 of the kind's largest entry."""
    from tests import _trees as T
    from tests.test_oracle_grad import event_tree
    trees = []
    for seed in range(20, 26):
        t = T.small_random_tree(seed, n_b=24, depth=5, n_a=6)
        t.qd0[:] = np.random.default_rng(seed).uniform(-0.3, 0.3, t.n_dofs)
        trees.append(t)
    trees.append(event_tree())
    f = T.concat(trees)
    fl = I.Flags()
    n = 150
    st, rec0 = O.rollout(f, fl, n, record_tips=True)
    target = rec0["tips"] + np.random.default_rng(4).normal(0.0, 0.01, rec0["tips"].shape)
    g, ev, _ = gpu_gradients(f, fl, n, ckpt_every, target)
    for w in range(f.n_worlds):
        assert PAR.events(ev["broken"], ev["break_step"], ev["detached"], ev["detach_step"], f, w) == \
            PAR.events(st.broken, st.break_step, st.detached, st.detach_step, f, w)
        ref = O.grad_full(f, fl, w, n, target[:, f.tip_off[w]:f.tip_off[w + 1]])
        b0, b1, d0, d1 = f.body_off[w], f.body_off[w + 1], f.dof_off[w], f.dof_off[w + 1]
        for name, got in (("dk", g[0][b0:b1]), ("dkd", g[1][b0:b1]), ("dq0", g[2][d0:d1]), ("dqd0", g[3][d0:d1])):
            r = ref[name]
            nrm = np.linalg.norm(r)
            assert nrm > 0
            assert np.linalg.norm(got - r) <= 1e-3 * nrm, f"world {w} {name}: normwise {np.linalg.norm(got - r) / nrm:.2e}"
            assert np.abs(got - r).max() <= 2e-3 * np.abs(r).max(), f"world {w} {name}"


@pytest.mark.parametrize("world,n,per_kind", [(0, 60, 4), (4096, 60, 4), (8000, 30, 2)])
def test_adjoint_stress_size_classes(world, n, per_kind):
    """One world per size class of the stress workload (50, 400 and 2000 bodies), with FP64
    pivots on twigs under 5 mm, against the oracle's complex-step derivative (1 cm target).
    Per kind of coordinate the error must stay within 2e-3 of the largest sampled entry (the
    serial FP32 evaluation of the same arithmetic: at most 1.1e-3); the error is printed per
    size class."""
    f = I.make_forest(I.STRESS, worlds=[world])
    fl = I.Flags(fp64_twig_diam=0.005)
    _, rec0 = O.rollout(f, fl, n, record_tips=True)
    rng = np.random.default_rng(world + 1)
    target = rec0["tips"] + rng.normal(0.0, 0.01, rec0["tips"].shape)
    g, _, _ = gpu_gradients(f, fl, n, 20, target)
    kinds, idx = sample_coords(f, 0, per_kind, rng)
    g_cs, _ = O.grad(f, fl, 0, n, target, kinds, idx, np.full(len(kinds), 1e-20), mode=0)
    got = pick(f, 0, g, kinds, idx)
    errs = {["k", "kd", "q0", "qd0"][k]: float(np.abs(got[kinds == k] - g_cs[kinds == k]).max() /
                                              np.abs(g_cs[kinds == k]).max()) for k in range(4)}
    print(f"stress adjoint, {int(np.diff(f.body_off)[0])} bodies: relative error per kind {errs}")
    assert_close_per_kind(got, g_cs, kinds, 2e-3, f"stress world {world}")


@pytest.mark.parametrize("ckpt_every", [0, 10])
def test_backward_schedules_give_the_same_gradients(ckpt_every):
    """Two size classes (50- and 400-body stress trees), 40 steps, the forward's tape or
    checkpoints: every backward threads-per-world candidate, and the one the backward autotuner
    picks, give the default plan's gradients (the work of each joint and each scan does not
    depend on which warp takes it)."""
    torch = _torch()
    from paper_2607_06337_b300 import orchard as B
    f = I.make_forest(I.STRESS, worlds=[0, 1, 4096, 4097])
    fl = I.Flags(fp64_twig_diam=0.005)
    n = 40
    sim = B.Simulator(f, fl)
    assert sim.counts.classes >= 2
    sim.reset()
    tips, _, rec = sim.record_buffers(n, ckpt_every)
    sim.rollout(n, record=rec)
    dtips = (1e-3 * torch.sin(torch.arange(tips.numel(), device="cuda", dtype=torch.float32))).view_as(tips)
    ref = [g.cpu().numpy() for g in sim.backward(n, rec, dtips)]

    def same(got, what):
        for a, b, name in zip(got, ref, ("dk", "dkd", "dq0", "dqd0")):
            np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max(), err_msg=f"{what} {name}")

    for t in (64, 128, 256):
        for k in range(sim.counts.classes):
            B.set_backward_schedule(sim.model, k, t)
        assert sim.backward_schedules() == [t] * sim.counts.classes
        same([g.cpu().numpy() for g in sim.backward(n, rec, dtips)], f"{t} threads per world")
    sim.autotune_backward(n, rec, dtips)
    assert all(t in (64, 128, 256) for t in sim.backward_schedules())
    same([g.cpu().numpy() for g in sim.backward(n, rec, dtips)], "autotuned")
