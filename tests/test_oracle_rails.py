"""Pins of the oracle's applied-force rails (App. B), read as: (1) impulse cap, dt |f| / m <= v_lim;
(2) power fade, the component of f along the velocity, when it pushes along it, scaled by
phi(|v|) = (v_lim - |v|) / (v_lim - v_fade) between v_fade and v_lim (1 below, 0 above); (3) speed
brake, -c_b m (|v| - v_lim) v / |v| added above v_lim; all at the step's start velocity, on an
apple's applied force.

A detached apple in zero gravity under a constant force along its velocity is a scalar
recurrence v' = v + dt f'(v) / m, whose solutions in closed form are the pins:
* inside the fade band, the deficit u = v_lim - v decays as u_n = u_0 (1 - kappa)^n with
  kappa = dt F / (m (v_lim - v_fade)): the speed approaches v_lim from below and never reaches it;
* a force above the cap lifts an apple at rest to exactly v_lim in one step, and the fade then
  holds it there;
* against an opposing force F above v_lim the brake gives u_n = (u_0 + F / (m c_b))
  (1 - dt c_b)^n - F / (m c_b), u = v - v_lim.
"""
import numpy as np
import pytest

import oracle as O
from paper_2607_06337_b300 import inputs as I

MASS = 0.2


def _free_apple(force, v0):
    """One hinge body at rest and one apple, detached, at the origin with velocity v0 along x,
    pulled by `force` (3-vector) from step 0; no gravity."""
    mb, com, inertia = I.cylinder(0.02, 0.2, 700.0)
    body = dict(parent=-1, ndof=1, jpos=(0.0, 0.0, 0.0), qrel=(1.0, 0.0, 0.0, 0.0), mass=mb, com=com,
                inertia=inertia, k=50.0, kd=0.0, length=0.2, diam=0.02)
    apple = dict(body=0, hang_local=(0.0, 0.0, 0.2), attach_local=(0.0, 0.0, 0.2), mass=MASS, k_s=1000.0,
                 c_s=1.0, f_detach=1e9, x0=(0.0, 0.0, 0.0), v0=(v0, 0.0, 0.0))
    f = I.from_bodies([body], apples=[apple], tips=[(0, (0.0, 0.0, 0.2))], gravity=(0.0, 0.0, 0.0))
    f.pull_force[0] = force
    f.pull_start[0] = 0
    f.pull_end[0] = 1 << 30
    st = O.OracleState.initial(f)
    st.detached[0] = 1
    return f, st


def _speeds(f, fl, st, n):
    out = []
    for _ in range(n):
        st, _ = O.rollout(f, fl, 1, state=st, n_threads=1, step0=len(out))
        out.append(st.av[0].copy())
    return np.array(out)


FL = dict(rail_speed=4.0, rail_fade_speed=2.0, rail_brake=8.0)


def test_power_fade_approaches_the_speed_limit_geometrically():
    F = 3.0
    fl = I.Flags(**FL)
    v0 = 3.0
    f, st = _free_apple((F, 0.0, 0.0), v0)
    v = _speeds(f, fl, st, 400)
    kappa = fl.dt * F / (MASS * (FL["rail_speed"] - FL["rail_fade_speed"]))
    u = (FL["rail_speed"] - v0) * (1.0 - kappa) ** np.arange(1, 401)
    np.testing.assert_allclose(FL["rail_speed"] - v[:, 0], u, rtol=1e-10)
    assert np.all(v[:, 0] < FL["rail_speed"]) and np.all(v[:, 1:] == 0.0)


def test_rails_off_the_same_force_accelerates_without_bound():
    fl = I.Flags()
    f, st = _free_apple((3.0, 0.0, 0.0), 3.0)
    v = _speeds(f, fl, st, 100)
    np.testing.assert_allclose(v[:, 0], 3.0 + fl.dt * 3.0 / MASS * np.arange(1, 101), rtol=1e-12)


def test_impulse_cap_lifts_an_apple_at_rest_to_the_limit_and_holds_it():
    fl = I.Flags(**FL)
    cap = MASS * FL["rail_speed"] / fl.dt
    f, st = _free_apple((10.0 * cap, 0.0, 0.0), 0.0)
    v = _speeds(f, fl, st, 50)
    np.testing.assert_allclose(v[:, 0], FL["rail_speed"], rtol=1e-13)


def test_speed_brake_against_an_opposing_force():
    F = 0.5
    fl = I.Flags(**FL)
    vl, cb = FL["rail_speed"], FL["rail_brake"]
    u0 = 6.0
    f, st = _free_apple((-F, 0.0, 0.0), vl + u0)
    n = 60
    v = _speeds(f, fl, st, n)
    k = np.arange(1, n + 1)
    u = (u0 + F / (MASS * cb)) * (1.0 - fl.dt * cb) ** k - F / (MASS * cb)
    assert np.all(u > 0)  # still above the limit: the brake acts on every step
    np.testing.assert_allclose(v[:, 0] - vl, u, rtol=1e-10)


def test_rails_do_not_touch_slow_loading():
    """The differentiation workload's apples (a fixed 5 N pull, no detachment) stay far below
    v_fade: with the rails on, every state is bitwise that of the rails off."""
    f = I.make_forest(I.DIFF, worlds=[0, 1])
    a, _ = O.rollout(f, I.Flags(), 200)
    b, _ = O.rollout(f, I.Flags(rail_speed=5.0, rail_fade_speed=2.5, rail_brake=10.0), 200)
    for k in ("q", "qd", "ax", "av"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k))


def test_rails_derivative_complex_step_vs_central_differences():
    """The oracle's complex-step derivative through the rails (cap, fade and brake all active on
    the pulled apple: v_lim of 2 cm/s), with the body damping on as well, matches central
    differences to their own truncation error."""
    from tests.test_oracle_grad import fd_steps, sample_coords
    f = I.make_forest(I.DIFF, worlds=[5])
    fl = I.Flags(rail_speed=0.02, rail_fade_speed=0.005, rail_brake=20.0, lin_damping=3.0, ang_damping=2.0)
    n = 60
    st, rec = O.rollout(f, fl, n, record_tips=True)
    off, _ = O.rollout(f, I.Flags(lin_damping=3.0, ang_damping=2.0), n)
    assert np.abs(st.av - off.av).max() > 1e-3  # the rails did act
    rng = np.random.default_rng(12)
    target = rec["tips"] + rng.normal(0.0, 0.01, rec["tips"].shape)
    kinds, idx = sample_coords(f, 0, 3, rng)
    g_cs, _ = O.grad(f, fl, 0, n, target, kinds, idx, np.full(len(kinds), 1e-20), mode=0)
    g_fd, _ = O.grad(f, fl, 0, n, target, kinds, idx, fd_steps(f, 0, kinds, idx), mode=1)
    for kind in range(4):
        s = kinds == kind
        scale = np.abs(g_cs[s]).max()
        assert scale > 0
        np.testing.assert_allclose(g_fd[s], g_cs[s], rtol=0, atol=1e-4 * scale)
