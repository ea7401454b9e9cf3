"""GPU step (through the C ABI) against the FP64 oracle, element by element."""
import numpy as np
import pytest

import oracle as O
from paper_2607_06337_b300 import inputs as I
from tests import parity as PAR

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("oracle_lib")]


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _gpu_state(sim):
    return dict(q=sim.q.cpu().numpy().astype(np.float64), qd=sim.qd.cpu().numpy().astype(np.float64),
                ax=sim.apple_x.cpu().numpy().astype(np.float64), broken=sim.broken.cpu().numpy(),
                break_step=sim.break_step.cpu().numpy(), detached=sim.detached.cpu().numpy(),
                detach_step=sim.detach_step.cpu().numpy(), status=sim.status.cpu().numpy())


def _run(f, flags, n_steps, form="batched", record_tips=False):
    torch = _torch()
    from paper_2607_06337_b300.orchard import Record, Simulator
    sim = Simulator(f, flags)
    sim.reset()
    tips = None
    rec = None
    if record_tips:
        tips = torch.zeros((n_steps, f.n_tips, 3), dtype=torch.float32, device="cuda")
        rec = Record(tips.data_ptr(), None, 0, 0)
    if form == "batched":
        sim.rollout(n_steps, record=rec)
    elif form == "plain":
        sim.rollout_plain(n_steps)
    elif form == "step":
        for t in range(n_steps):
            sim.step(t)
    torch.cuda.synchronize()
    out = _gpu_state(sim)
    if tips is not None:
        out["tips"] = tips.cpu().numpy().astype(np.float64)
    return out


@pytest.mark.parametrize("form", ["batched", "plain"])
def test_config0_plain_parity_1000_steps(form):
    """16 worlds x 64 bodies x 8 apples, gravity only, 1000 steps (the plain-form workload)."""
    f = I.make_forest(I.PLAIN)
    fl = I.Flags()
    g = _run(f, fl, 1000, form)
    st, rec = O.rollout(f, fl, 1000, near_eps=PAR.NEAR)
    rep = PAR.compare(f, fl, g, st, rec["near"])
    PAR.assert_parity(rep)
    assert max(r["ratio"] for r in rep) < 0.1  # ample margin in the smooth regime
    assert (g["status"] == 0).all()


def test_body_damping_with_pulls_and_events():
    """Velocity-proportional body damping on (Sec. IV-A), reduced linear drag on snapped
    sub-trees (Sec. IV-B): uneven trees with random pulls, q gate and identical event sets."""
    f = I.make_forest(I.BATCH, worlds=[0, 1, 2, 3, 17, 33])
    fl = I.Flags(lin_damping=3.0, ang_damping=2.0, snapped_lin_damping=0.2)
    g = _run(f, fl, 1000)
    st, rec = O.rollout(f, fl, 1000, near_eps=PAR.NEAR)
    rep = PAR.compare(f, fl, g, st, rec["near"])
    PAR.assert_parity(rep)
    assert sum(r["n_events"] for r in rep) > 5  # breaks put bodies on snapped sub-trees
    st0, _ = O.rollout(f, I.Flags(), 1000)
    assert np.abs(st.q - st0.q).max() > 1e-3  # the damping does change the motion


def test_applied_force_rails_with_pulls_and_events():
    """The rails of App. B on the apples' applied forces (impulse cap, power fade, speed brake)
    in uneven trees with random pulls up to 60 N: q gate and identical event sets, and the
    detached apples' speeds against the oracle's (they fly under their pull, so the rails act on
    them while it lasts)."""
    torch = _torch()
    from paper_2607_06337_b300.orchard import Simulator
    f = I.make_forest(I.BATCH, worlds=[0, 1, 2, 3, 17, 33])
    fl = I.Flags(rail_speed=3.0, rail_fade_speed=1.5, rail_brake=10.0)
    n = 1000
    sim = Simulator(f, fl)
    sim.reset()
    sim.rollout(n)
    torch.cuda.synchronize()
    g = _gpu_state(sim)
    gv = sim.apple_v.cpu().numpy().astype(np.float64)
    st, rec = O.rollout(f, fl, n, near_eps=PAR.NEAR)
    rep = PAR.compare(f, fl, g, st, rec["near"])
    PAR.assert_parity(rep)
    det = (st.detached > 0) & (g["detached"] > 0)
    assert det.sum() >= 5
    s_ref = np.linalg.norm(st.av[det], axis=1)
    s_gpu = np.linalg.norm(gv[det], axis=1)
    # the rails hold the flying apples near v_lim: gravity is not an applied force, so under a
    # pull the brake balances it at v_lim + g / c_b at most
    assert s_ref.max() < 3.0 + 9.81 / 10.0 + 1e-6
    np.testing.assert_allclose(s_gpu, s_ref, rtol=1e-3, atol=1e-4)
    off, _ = O.rollout(f, I.Flags(), n)
    assert np.linalg.norm(off.av[det], axis=1).max() > 10.0  # without the rails they run away


def test_model_variants_with_pulls_and_events():
    """Generated-model variants (pipe exponent 2.3, capsule links, the paper's Kd = c_d Kp with
    c_d = 0.1 s) on uneven trees with random pulls: q gate and identical event sets."""
    var = I.ModelVariant(pipe_exponent=2.3, capsule=True, damping_cd=0.1)
    f = I.make_forest(I.BATCH, worlds=[0, 1, 2, 17], variant=var)
    fl = I.Flags()
    g = _run(f, fl, 1000)
    st, rec = O.rollout(f, fl, 1000, near_eps=PAR.NEAR)
    rep = PAR.compare(f, fl, g, st, rec["near"])
    PAR.assert_parity(rep)


def test_per_level_stiffness_variant():
    """The per-level exponential stiffness (k = 2000 N m / rad x 0.3^(depth - 1)) on the plain
    workload's trees under gravity: q gate."""
    var = I.ModelVariant(level_k0=2000.0, level_gamma=0.3)
    f = I.make_forest(I.PLAIN, variant=var)
    fl = I.Flags()
    g = _run(f, fl, 500)
    st, rec = O.rollout(f, fl, 500, near_eps=PAR.NEAR)
    rep = PAR.compare(f, fl, g, st, rec["near"])
    PAR.assert_parity(rep)


def test_device_domain_randomisation_against_the_host_build():
    """ot_model_randomize (per-world lengths, diameters, density, modulus, rupture strength and
    c_d; every derived record rebuilt on the GPU) against its host counterpart inputs.randomize:
    the GPU rollout of the device-randomised model and the oracle's rollout of the host-randomised
    forest, with the same (float32) factors: q gate and identical event sets."""
    torch = _torch()
    from paper_2607_06337_b300.orchard import Simulator
    f = I.make_forest(I.BATCH, worlds=[0, 1, 2, 17])
    rng = np.random.default_rng(9)
    fac = np.column_stack([rng.uniform(0.85, 1.15, (f.n_worlds, 5)), rng.uniform(0.05, 0.15, f.n_worlds)])
    fac = fac.astype(np.float32)
    fl = I.Flags()
    n = 600
    sim = Simulator(f, fl)
    sim.randomize(torch.as_tensor(fac, device="cuda"))
    sim.reset()
    sim.rollout(n)
    torch.cuda.synchronize()
    g = _gpu_state(sim)
    h = I.randomize(f, fac.astype(np.float64))
    st, rec = O.rollout(h, fl, n, near_eps=PAR.NEAR)
    rep = PAR.compare(h, fl, g, st, rec["near"])
    PAR.assert_parity(rep)
    plain, _ = O.rollout(f, fl, n)
    assert np.abs(plain.q - st.q).max() > 1e-3  # the randomisation does change the worlds


def test_domain_randomisation_needs_the_material():
    torch = _torch()
    from paper_2607_06337_b300.orchard import Simulator
    from tests import _trees as T
    f, _, _ = T.single_hinge()
    sim = Simulator(f, I.Flags())
    with pytest.raises(RuntimeError):
        sim.randomize(torch.ones((1, 6), dtype=torch.float32, device="cuda"))


def test_step_by_step_equals_rollout():
    f = I.make_forest(I.BATCH, worlds=[5, 6, 7])
    fl = I.Flags()
    a = _run(f, fl, 60, "batched")
    b = _run(f, fl, 60, "step")
    np.testing.assert_array_equal(a["q"], b["q"])
    np.testing.assert_array_equal(a["broken"], b["broken"])


def test_config1_subset_with_pulls_and_events():
    """Uneven trees (100-600 bodies) with random pulls: q gate and identical event sets."""
    f = I.make_forest(I.BATCH, worlds=[0, 1, 2, 3, 17, 33, 64, 101])
    fl = I.Flags()
    g = _run(f, fl, 1000)
    st, rec = O.rollout(f, fl, 1000, near_eps=PAR.NEAR)
    rep = PAR.compare(f, fl, g, st, rec["near"])
    PAR.assert_parity(rep)
    assert sum(r["n_events"] for r in rep) > 10  # the workload does exercise breaks and detaches


def _stratified(f, n):
    """n worlds at evenly spaced ranks of the size order (bodies plus apples)."""
    sizes = np.diff(f.body_off) + np.diff(f.apple_off)
    order = np.argsort(sizes, kind="stable")
    return np.unique(order[np.linspace(0, len(order) - 1, n).round().astype(np.int64)])


def test_config1_stratified_64_worlds_1000_steps():
    """The batching workload's parity sample: 64 of its 4096 trees stratified by size (100-600
    bodies, with their random pulls), 1000 steps, through the autotuned batched rollout; q gate
    and identical event sets on every world."""
    from paper_2607_06337_b300.orchard import Simulator
    torch = _torch()
    full = I.make_forest(I.BATCH, processes=8)
    f = full.subset(_stratified(full, 64))
    fl = I.Flags()
    sim = Simulator(f, fl)
    sim.autotune(n_steps=10)
    sim.reset()
    sim.rollout(1000)
    torch.cuda.synchronize()
    g = _gpu_state(sim)
    st, rec = O.rollout(f, fl, 1000, near_eps=PAR.NEAR)
    rep = PAR.compare(f, fl, g, st, rec["near"])
    PAR.assert_parity(rep)
    assert len(rep) == 64 and sum(r["n_events"] for r in rep) > 100
    print("batch4096 stratified 64: max q-error / gate", round(max(r["ratio"] for r in rep), 4))


def test_config4_stress_four_worlds_per_class_500_steps():
    """The stress workload's parity sample: four worlds of each size class (50, 400 and 2000
    bodies, the last with its temporaries in global memory) over the workload's full 500 steps,
    FP64 pivots on twigs under 5 mm as the workload runs them; the error against the oracle
    per size class."""
    f = I.make_forest(I.STRESS, worlds=[0, 1365, 2730, 4095, 4096, 5461, 6826, 8191 - 820, 7373, 7782, 8000, 8191])
    sizes = np.diff(f.body_off)
    assert sorted(np.unique(sizes).tolist()) == [50, 400, 2000] and all((sizes == s).sum() == 4 for s in (50, 400, 2000))
    fl = I.Flags(fp64_twig_diam=0.005)
    g = _run(f, fl, 500)
    st, rec = O.rollout(f, fl, 500, near_eps=PAR.NEAR)
    rep = PAR.compare(f, fl, g, st, rec["near"])
    PAR.assert_parity(rep)
    for s in (50, 400, 2000):
        print(f"stress {s} bodies: max q-error / gate",
              round(max(r["ratio"] for r, n in zip(rep, sizes) if n == s), 4))


@pytest.mark.parametrize("workload,worlds,stage", [(I.BATCH, list(range(0, 60, 3)), -1),
                                                   (I.PLAIN, list(range(16)), 127)])
def test_staged_model_records_give_the_same_states(workload, worlds, stage):
    """The staged instantiation (model records copied into shared memory per world: stage -1
    takes every part that fits, 127 all of them) reads the same values as the unstaged one, so
    every class's states after a rollout are bit-identical: uneven batch trees with pulls, breaks
    and detaches (automatic staging), and the plain-form trees with every part staged."""
    torch = _torch()
    from paper_2607_06337_b300 import orchard as B
    f = I.make_forest(workload, worlds=worlds)
    fl = I.Flags()
    out = []
    for st in (0, stage):
        sim = B.Simulator(f, fl)
        for k, sc in enumerate(sim.schedules()):
            # one world per block at 64 threads: room for the records of most of these trees
            B.set_schedule(sim.model, k, B.Schedule(64, 1, 0, sc.global_workspace, st))
        infos = sim.class_infos()
        if st == -1:
            assert any(ci["stage_mask"] for ci in infos)
        if st == 127:
            assert all(ci["stage_mask"] == 127 for ci in infos)
        sim.reset()
        sim.rollout(300)
        torch.cuda.synchronize()
        out.append(_gpu_state(sim))
        sim.close()
    for key in ("q", "qd", "ax", "broken", "break_step", "detached", "detach_step", "status"):
        np.testing.assert_array_equal(out[1][key], out[0][key], err_msg=key)
    if workload == I.BATCH:
        assert out[0]["broken"].sum() + out[0]["detached"].sum() > 0


def test_lean_placement_gives_the_same_states():
    """The lean placement (schedule global_workspace 2: the state, the apple records and the
    snapped flags in global memory, the rest of the workspace in shared memory) computes what the
    whole-workspace placement does: the six largest batch trees and two small ones, with pulls,
    breaks and detaches, bit-identical states and tips after 300 steps with checkpoints written
    on the way; and a rollout that writes the adjoint's tape under a lean schedule (run in the
    whole-workspace placement) gives the same states again."""
    torch = _torch()
    from paper_2607_06337_b300 import orchard as B
    full = I.make_forest(I.BATCH, processes=8)
    order = np.argsort(np.diff(full.body_off), kind="stable")
    f = full.subset(sorted(order[-6:].tolist() + order[:2].tolist()))
    fl = I.Flags()
    n = 300
    out = []
    for lean, ce in ((False, 50), (True, 50), (True, 0)):
        sim = B.Simulator(f, fl)
        taken = 0
        for k, sc in enumerate(sim.schedules()):
            if lean and not sc.global_workspace:
                try:
                    B.set_schedule(sim.model, k, B.Schedule(256, 1, 0, 2, 0))
                    taken += 1
                except B.OrchardError:
                    pass  # a class that fits two worlds per SM is not offered the lean placement
        if lean:
            assert taken >= 1
            assert any(ci["workspace_bytes"] < 140 * 1024 for ci in sim.class_infos() if ci["max_bodies"] > 550)
            for k, sc in enumerate(sim.schedules()):
                if sc.global_workspace == 2:  # instantiated for 128-512 threads per world only
                    with pytest.raises(B.OrchardError):
                        B.set_schedule(sim.model, k, B.Schedule(64, 1, 0, 2, 0))
                elif not sc.global_workspace:  # classes of several worlds per SM: not offered
                    with pytest.raises(B.OrchardError):
                        B.set_schedule(sim.model, k, B.Schedule(256, 1, 0, 2, 0))
        tips, buf, rec = sim.record_buffers(n, ce)
        sim.reset()
        sim.rollout(n, record=rec)
        torch.cuda.synchronize()
        st = _gpu_state(sim)
        st["tips"] = tips.cpu().numpy()
        st["ckpt"] = buf.cpu().numpy() if ce else None
        out.append(st)
        sim.close()
    for o in out[1:]:
        for key in ("q", "qd", "ax", "broken", "break_step", "detached", "detach_step", "status", "tips"):
            np.testing.assert_array_equal(o[key], out[0][key], err_msg=key)
    np.testing.assert_array_equal(out[1]["ckpt"], out[0]["ckpt"], err_msg="checkpoints")
    assert out[0]["broken"].sum() + out[0]["detached"].sum() > 0


def test_autotune_leaves_the_state_as_it_found_it():
    """ot_autotune times every launch from a device copy of the state it was given and restores
    the state at the end: uneven batch trees advanced 50 steps (pulls, a break or detach on the
    way), then autotuned, hold bit-identical state arrays, status words included."""
    torch = _torch()
    from paper_2607_06337_b300 import orchard as B
    f = I.make_forest(I.BATCH, worlds=[0, 700, 1400, 2100, 2800, 3500, 4095])
    fl = I.Flags()
    sim = B.Simulator(f, fl)
    sim.reset()
    sim.rollout(50)
    torch.cuda.synchronize()
    before = _gpu_state(sim)
    B.autotune(sim.model, sim.state, 5, fl.dt)
    torch.cuda.synchronize()
    after = _gpu_state(sim)
    sim.close()
    for key in ("q", "qd", "ax", "broken", "break_step", "detached", "detach_step", "status"):
        np.testing.assert_array_equal(after[key], before[key], err_msg=key)


def test_tip_record_matches_oracle():
    f = I.make_forest(I.DIFF, worlds=[0, 1, 2])
    fl = I.Flags()
    g = _run(f, fl, 200, record_tips=True)
    st, rec = O.rollout(f, fl, 200, record_tips=True)
    err = np.abs(g["tips"] - rec["tips"]).max()
    assert err < 1e-5, err


@pytest.mark.parametrize("twig", [0.0, 0.005])
def test_stress_classes_including_global_workspace(twig):
    """50 / 400 / 2000-body worlds (the 2000-body class runs with its workspace in global memory),
    with FP32 pivots throughout and with FP64 pivots on the joints of twigs under 5 mm (the
    stress workload's setting); the oracle is FP64 either way."""
    f = I.make_forest(I.STRESS, worlds=[0, 4096, 8000])  # one world per size class
    assert sorted(np.diff(f.body_off)) == [50, 400, 2000]
    if twig:
        assert (f.diam < twig).sum() > 100  # the setting reaches many joints
    fl = I.Flags(fp64_twig_diam=twig)
    g = _run(f, fl, 150)
    st, rec = O.rollout(f, fl, 150, near_eps=PAR.NEAR)
    rep = PAR.compare(f, fl, g, st, rec["near"])
    PAR.assert_parity(rep)
    print("stress q-error / gate per world:", [round(r["ratio"], 4) for r in rep], "twig", twig)


def test_edge_cases_single_body_and_chain():
    """Degenerate worlds in one batch: a welded post with an apple (no DOFs), a one-body hinge,
    a 1-DOF chain, and a regular tree."""
    from tests import _trees as T
    post = I.from_bodies([dict(parent=-1, ndof=0, mass=1.0, com=(0, 0, 0.5), inertia=(0.1, 0.1, 0.01))],
                         apples=[dict(body=0, hang_local=(0, 0, 1.0), mass=0.2, k_s=1000.0, c_s=5.0, f_detach=20.0,
                                      x0=(0.0, 0.0, -0.01), v0=(0.0, 0.0, 0.0))])
    hinge, _, _ = T.single_hinge(k=0.5, kd=0.01, gravity=(0.0, 0.0, -9.81))
    hinge.q0[:] = 0.3
    chain, _ = T.chain(12, 0.1, 0.01, 700.0, 1e9, kd=0.05, gravity=(0.0, 0.0, -9.81))
    chain.q0[:] = np.linspace(0.05, -0.05, 12)
    tree = I.make_forest(I.PLAIN, worlds=[0])
    f = T.concat([post, hinge, chain, tree])
    fl = I.Flags()
    g = _run(f, fl, 300)
    st, rec = O.rollout(f, fl, 300, near_eps=PAR.NEAR)
    rep = PAR.compare(f, fl, g, st, rec["near"])
    PAR.assert_parity(rep)
    np.testing.assert_allclose(g["ax"], st.ax, atol=1e-5)


def test_nonfinite_world_is_frozen_others_continue():
    f = I.make_forest(I.PLAIN, worlds=[0, 1])
    f.q0 = f.q0.copy()
    f.q0[f.dof_off[1] + 3] = np.nan
    fl = I.Flags()
    g = _run(f, fl, 50)
    assert g["status"][1] & 1 and g["status"][0] == 0
    st, _ = O.rollout(f.subset([0]), fl, 50)
    a, b = f.dof_off[0], f.dof_off[1]
    assert np.abs(g["q"][a:b] - st.q).max() < 1e-4 * np.abs(st.q).max() + 1e-7


def test_classes_sharing_a_kernel_instantiation():
    """Several size classes launched with the same threads-per-world (default schedules, then
    one uniform schedule set through the ABI) must all run and agree with the oracle."""
    torch = _torch()
    from paper_2607_06337_b300 import orchard as B
    f = I.make_forest(I.BATCH, worlds=list(range(0, 96, 2)))
    fl = I.Flags()
    st, rec = O.rollout(f, fl, 30, near_eps=PAR.NEAR)
    sim = B.Simulator(f, fl)
    assert sim.counts.classes >= 2
    for uniform in (False, True):
        if uniform:
            for k, sc in enumerate(sim.schedules()):
                B.set_schedule(sim.model, k, B.Schedule(64, 1, 0, sc.global_workspace))
        sim.reset()
        sim.rollout(30)
        torch.cuda.synchronize()
        rep = PAR.compare(f, fl, _gpu_state(sim), st, rec["near"])
        PAR.assert_parity(rep)
