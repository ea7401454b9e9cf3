"""Pins of the oracle's velocity-proportional body damping (Sec. IV-A: force -c_v m v and torque
-c_omega I omega at each body's centre of mass; Sec. IV-B: a snapped sub-tree's linear drag is
reduced).

A single hinge with no spring, no gravity and no joint damper reduces the step to an exact
scalar recurrence. The damping is taken explicitly at the step's start velocity, so with J the
inertia about the hinge axis, I_a the inertia about the parallel axis through the centre of
mass, d the centre of mass's distance from the axis and s the snapped factor (1 unless the
joint is broken):

    qd_(n+1) = rho qd_n,  rho = 1 - dt (c_omega I_a + s c_v m d^2) / J,  q_(n+1) = q_n + dt qd_(n+1).

The velocity products vanish (the axis is principal and the centre of mass moves on a circle
about it), so any other term would show up as a departure from rho.
"""
import numpy as np
import pytest

import oracle as O
from paper_2607_06337_b300 import inputs as I

from tests import _trees as T

pytestmark = pytest.mark.filterwarnings("ignore")


def _expected_q(rho, dt, qd0, n):
    """q_n = dt qd0 (rho + rho^2 + ... + rho^n)."""
    k = np.arange(1, n + 1)
    if rho == 1.0:
        return dt * qd0 * k
    return dt * qd0 * rho * (1.0 - rho ** k) / (1.0 - rho)


def _run(f, fl, n, state=None):
    st, rec = O.rollout(f, fl, n, state=state, record_q=True, n_threads=1)
    return st, rec["q"][:, 0]


def test_angular_damping_alone_on_an_axis_through_the_centre_of_mass():
    """Centre of mass on the hinge axis: v_c = 0, J = I_a, rho = 1 - dt c_omega exactly."""
    f, _, m = T.single_hinge(k=0.0, kd=0.0)
    f.com[0] = (0.0, 0.0, 0.0)
    f.qd0[0] = 1.0
    Ia = float(f.inertia[0][0])
    fl = I.Flags(lin_damping=3.0, ang_damping=0.7)   # c_v must not matter here
    n = 300
    st, q = _run(f, fl, n)
    rho = 1.0 - fl.dt * 0.7 * Ia / Ia
    np.testing.assert_allclose(q, _expected_q(rho, fl.dt, 1.0, n), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(st.qd[0], rho ** n, rtol=1e-12)


@pytest.mark.parametrize("cv,cw", [(0.0, 0.0), (2.0, 0.0), (0.0, 1.5), (2.0, 1.5)])
def test_linear_and_angular_damping_on_an_offset_centre_of_mass(cv, cw):
    """Segment hinged at its end (d = l / 2): both terms, J = I_a + m d^2."""
    f, J, m = T.single_hinge(k=0.0, kd=0.0)
    f.qd0[0] = 1.0
    Ia = float(f.inertia[0][0])
    d = 0.5 * float(f.length[0])
    fl = I.Flags(lin_damping=cv, ang_damping=cw)
    n = 300
    st, q = _run(f, fl, n)
    rho = 1.0 - fl.dt * (cw * Ia + cv * m * d * d) / J
    np.testing.assert_allclose(q, _expected_q(rho, fl.dt, 1.0, n), rtol=1e-12, atol=1e-15)


def test_snapped_body_has_reduced_linear_drag_only():
    """A broken joint: the body is on a snapped sub-tree, so c_v is scaled by the snapped factor
    while c_omega is not (the spring is gone with the break; the joint has no damper here)."""
    f, J, m = T.single_hinge(k=50.0, kd=0.0)
    f.qd0[0] = 1.0
    Ia = float(f.inertia[0][0])
    d = 0.5 * float(f.length[0])
    fl = I.Flags(lin_damping=2.0, ang_damping=1.5, snapped_lin_damping=0.25)
    s0 = O.OracleState.initial(f)
    s0.broken[0] = 1
    s0.break_step[0] = -10 ** 6
    n = 300
    st, q = _run(f, fl, n, state=s0)
    rho = 1.0 - fl.dt * (1.5 * Ia + 0.25 * 2.0 * m * d * d) / J
    np.testing.assert_allclose(q, _expected_q(rho, fl.dt, 1.0, n), rtol=1e-12, atol=1e-15)


def test_damping_dissipates_on_a_random_tree():
    """Invariant: with damping on, no gravity and no springs, the kinetic energy 1/2 qd^T M qd
    of a random tree never grows from step to step (explicit damping at dt c << 1)."""
    f = T.small_random_tree(3, n_b=7, depth=3, ndof=2, root_ndof=2)
    f.gravity[:] = 0.0
    f.k[:] = 0.0
    f.kd[:] = 0.0
    rng = np.random.default_rng(5)
    f.qd0 = rng.normal(0.0, 1.0, f.n_dofs)
    fl = I.Flags(lin_damping=4.0, ang_damping=4.0)
    st = O.OracleState.initial(f)
    energies = []
    for _ in range(60):
        M = O.evaluate(f, fl, 0, st.q, st.qd)["M"]
        energies.append(0.5 * st.qd @ M @ st.qd)
        st, _ = O.rollout(f, fl, 1, state=st, n_threads=1)
    e = np.array(energies)
    assert np.all(np.diff(e) <= 1e-12 * e[0]), np.diff(e).max()
    assert e[-1] < 0.9 * e[0]
