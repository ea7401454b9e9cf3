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


def test_static_scratch_rejects_worlds_that_do_not_fit():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_06337_b300 import orchard as B
    # a long chain ending in wide fans: ~32000 DOFs at depth ~160, whose mass-matrix rows alone
    # (about 21 MB) exceed the 16 MiB array
    chain, fan, sub = 80, 255, 62
    parent = list(range(-1, chain - 1))
    parent += [chain - 1] * fan
    for c in range(chain, chain + fan):
        parent += [c] * sub
    bodies = [dict(parent=p, ndof=0 if p < 0 else 2, mass=1.0, inertia=(1.0, 1.0, 1.0), com=(0, 0, 0.1),
                   jpos=(0, 0, 0.2)) for p in parent]
    f = I.from_bodies(bodies)
    sim = B.Simulator(f, I.Flags())
    sim.reset()
    q_before = sim.q.clone()
    st = B.lib().ot_step_static_scratch(sim.model, sim.state, None, C.byref(sim.pulls), 0, 2e-3, B._stream_handle())
    assert st == B.OT_ECAPACITY
    torch.cuda.synchronize()
    assert torch.equal(sim.q, q_before)  # nothing ran
