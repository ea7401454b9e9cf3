"""The allocation-free step (ot_step_static_scratch), for callers that cannot allocate device
memory while they step: its per-world temporaries live in a fixed array inside the library.

It must give the same states as the regular ot_step on the same inputs, call after call. This
file is collected last, so a run that stops at the first failure has run every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_2607_06337_b300 import inputs as I

pytestmark = pytest.mark.gpu

Q_REL, Q_ABS = 1e-4, 1e-7  # the q gate of the parity tests


def _state(sim):
    return (sim.q.cpu().numpy().astype(np.float64), sim.qd.cpu().numpy().astype(np.float64),
            sim.apple_x.cpu().numpy().astype(np.float64), sim.broken.cpu().numpy(),
            sim.detached.cpu().numpy())


def test_static_scratch_step_matches_regular_step_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_06337_b300 import orchard as B
    # uneven worlds across several size classes, with pulls active from step 0
    f = I.make_forest(I.BATCH, worlds=[0, 1, 2, 3, 40, 41])
    f.pull_start = np.minimum(f.pull_start, 0).astype(np.int32)
    fl = I.Flags()
    ref = B.Simulator(f, fl)
    alt = B.Simulator(f, fl)
    ref.reset()
    alt.reset()
    L = B.lib()
    stream = B._stream_handle()
    for t in range(2):  # two calls in a row
        ref.step(t)
        st = L.ot_step_static_scratch(alt.model, alt.state, None, C.byref(alt.pulls), t, fl.dt, stream)
        assert st == B.OT_OK, L.ot_status_string(st).decode()
        torch.cuda.synchronize()
        a, b = _state(ref), _state(alt)
        for w in range(f.n_worlds):
            lo, hi = f.dof_off[w], f.dof_off[w + 1]
            err = np.abs(a[0][lo:hi] - b[0][lo:hi]).max()
            assert err <= Q_REL * np.abs(a[0][lo:hi]).max() + Q_ABS, (t, w, err)
        np.testing.assert_allclose(b[1], a[1], rtol=1e-4, atol=1e-6)
        np.testing.assert_allclose(b[2], a[2], rtol=1e-4, atol=1e-7)
        np.testing.assert_array_equal(b[3], a[3])
        np.testing.assert_array_equal(b[4], a[4])
    assert np.abs(a[1]).max() > 0  # the trees did move


def _fan_world(chain, fan, sub):
    """A long chain ending in wide fans of short branches: deep DOF rows, whose mass-matrix
    storage alone runs to megabytes."""
    parent = list(range(-1, chain - 1))
    parent += [chain - 1] * fan
    for c in range(chain, chain + fan):
        parent += [c] * sub
    bodies = [dict(parent=p, ndof=0 if p < 0 else 2, mass=1.0, inertia=(1.0, 1.0, 1.0), com=(0, 0, 0.1),
                   jpos=(0, 0, 0.2), k=0.0 if p < 0 else 50.0, kd=0.0 if p < 0 else 0.5) for p in parent]
    return I.from_bodies(bodies)


def _compare(ref, alt, f):
    a, b = _state(ref), _state(alt)
    for w in range(f.n_worlds):
        lo, hi = f.dof_off[w], f.dof_off[w + 1]
        err = np.abs(a[0][lo:hi] - b[0][lo:hi]).max()
        assert err <= Q_REL * np.abs(a[0][lo:hi]).max() + Q_ABS, (w, err)
    np.testing.assert_allclose(b[1], a[1], rtol=1e-4, atol=1e-6)
    np.testing.assert_allclose(b[2], a[2], rtol=1e-4, atol=1e-7)
    np.testing.assert_array_equal(b[3], a[3])
    np.testing.assert_array_equal(b[4], a[4])
    return a


def test_static_scratch_global_workspace_class_with_external_force():
    """Stress-workload trees (50, 400 and 2000 bodies: the largest class keeps its temporaries
    in global memory) plus a deep fan world of several MB whose class is set to more worlds
    per block than the array has slots for; a per-step external force on every apple."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from tests._trees import concat
    from paper_2607_06337_b300 import orchard as B
    st_f = I.make_forest(I.STRESS, worlds=[0, 1, 8188])
    f = concat([st_f, _fan_world(80, 255, 25)])
    fl = I.Flags()
    ref = B.Simulator(f, fl)
    alt = B.Simulator(f, fl)
    scheds = ref.schedules()
    assert any(s.global_workspace for s in scheds)
    for k, s in enumerate(scheds):
        if s.global_workspace:
            wide = B.Schedule(32, 16, 0, 1)
            B.set_schedule(ref.model, k, wide)
            B.set_schedule(alt.model, k, wide)
    ref.reset()
    alt.reset()
    rng = np.random.default_rng(5)
    L = B.lib()
    stream = B._stream_handle()
    for t in range(2):
        fe = torch.as_tensor(rng.uniform(-20, 20, (f.n_apples, 3)).astype(np.float32), device="cuda")
        ref.step(t, ext_force=fe)
        st = L.ot_step_static_scratch(alt.model, alt.state, C.c_void_p(fe.data_ptr()), C.byref(alt.pulls), t,
                                      fl.dt, stream)
        assert st == B.OT_OK, L.ot_status_string(st).decode()
        torch.cuda.synchronize()
        a = _compare(ref, alt, f)
    assert np.abs(a[1]).max() > 0


def test_static_scratch_rejects_worlds_that_do_not_fit():
    """Uneven batch trees plus one world whose temporaries (about 21 MB of mass-matrix rows)
    exceed the 16 MiB array: the call is rejected before any class runs, so no world moves."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from tests._trees import concat
    from paper_2607_06337_b300 import orchard as B
    f = concat([I.make_forest(I.BATCH, worlds=[0, 40]), _fan_world(80, 255, 62)])
    sim = B.Simulator(f, I.Flags())
    sim.reset()
    before = [t.clone() for t in (sim.q, sim.qd, sim.apple_x)]
    st = B.lib().ot_step_static_scratch(sim.model, sim.state, None, C.byref(sim.pulls), 0, 2e-3, B._stream_handle())
    assert st == B.OT_ECAPACITY
    torch.cuda.synchronize()
    for a, b in zip(before, (sim.q, sim.qd, sim.apple_x)):
        assert torch.equal(a, b)  # nothing ran


def test_static_scratch_rejects_bad_arguments_before_running():
    """A state of another model, or a pull schedule without its step ranges: OT_EINVAL, and
    the state is untouched."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_06337_b300 import orchard as B
    f = I.make_forest(I.BATCH, worlds=[0, 1])
    a = B.Simulator(f, I.Flags())
    b = B.Simulator(f, I.Flags())
    a.reset()
    b.reset()
    q0 = a.q.clone()
    L = B.lib()
    stream = B._stream_handle()
    assert L.ot_step_static_scratch(a.model, b.state, None, C.byref(a.pulls), 0, 2e-3, stream) == B.OT_EINVAL
    half = B.ForceSchedule(a.pulls.force, None, None)
    assert L.ot_step_static_scratch(a.model, a.state, None, C.byref(half), 0, 2e-3, stream) == B.OT_EINVAL
    torch.cuda.synchronize()
    assert torch.equal(a.q, q0)
