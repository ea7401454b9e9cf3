"""Pins of the oracle's apple tether, detachment, rupture and energy behaviour (CPU only)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2607_06337_b300 import inputs as I
from tests import _trees as T
from tests.test_oracle_pins import _closed_form_hinge

pytestmark = pytest.mark.usefixtures("oracle_lib")


def _without_apples(f):
    g = f.subset(range(f.n_worlds))
    g.apple_off = np.zeros_like(f.apple_off)
    for name in ("apple_body", "hang_local", "attach_local", "apple_mass", "k_s", "c_s", "f_detach",
                 "apple_x0", "apple_v0", "pull_force", "pull_start", "pull_end"):
        a = getattr(f, name)
        setattr(g, name, a[:0].copy())
    return g


# ------------------------------------------------------------------------------------------
# Apple at rest: the reaction vanishes, the tree behaves as if it bore no fruit (Sec. IV-C)
# ------------------------------------------------------------------------------------------
def test_reaction_vanishes_at_rest_sag():
    f = I.make_forest(I.PLAIN, worlds=[0])
    ev = O.evaluate(f, I.Flags(), 0, np.zeros(f.n_dofs), np.zeros(f.n_dofs), ax=f.apple_x0, av=f.apple_v0,
                    detached=np.zeros(f.n_apples, np.int32), fext=np.zeros((f.n_apples, 3)))
    assert np.abs(ev["fapp"]).max() < 1e-12
    np.testing.assert_allclose(ev["tension"], f.apple_mass * I.GRAVITY, rtol=1e-12)


@pytest.mark.parametrize("implicit", [0, 1])
def test_apples_at_rest_sag_do_not_load_a_tree_at_rest(implicit):
    """Sec. IV-C: only the elastic perturbation beyond rest is transmitted, so apples hanging at
    their rest sag below a tree in equilibrium leave its trajectory that of the bare tree (to
    rounding), with the reaction taken explicitly or implicitly."""
    f = I.make_forest(I.PLAIN, worlds=[1])
    bare = _without_apples(f)
    settle = I.Flags(dt=0.01)
    sb, _ = O.rollout(bare, settle, 4000, n_threads=1)
    assert np.abs(sb.qd).max() < 1e-10
    fl = I.Flags(tether_implicit=implicit)
    bare.q0 = sb.q.copy()
    f.q0 = sb.q.copy()
    f.apple_x0 = -(f.apple_mass * I.GRAVITY / f.k_s)[:, None] * np.array([0.0, 0.0, 1.0])
    _, ra = O.rollout(f, fl, 300, record_q=True, n_threads=1)
    _, rb = O.rollout(bare, fl, 300, record_q=True, n_threads=1)
    np.testing.assert_allclose(ra["q"], rb["q"], atol=1e-12 * np.abs(rb["q"]).max())


def test_implicit_tether_keeps_the_bare_tree_rest_pose():
    """With the coupled backward-Euler tether the dynamics feel the apple's inertia, but the
    settled pose under gravity is still exactly the bare tree's."""
    f = I.make_forest(I.PLAIN, worlds=[2])
    fl = I.Flags(tether_implicit=1, dt=0.01)
    sa, _ = O.rollout(f, fl, 4000, n_threads=1)
    sb, _ = O.rollout(_without_apples(f), fl, 4000, n_threads=1)
    assert np.abs(sa.qd).max() < 1e-10 and np.abs(sb.qd).max() < 1e-10
    np.testing.assert_allclose(sa.q, sb.q, atol=1e-9 * np.abs(sb.q).max())
    # and the apples sit at the rest sag below their (moved) hang points
    ev = O.evaluate(f, fl, 0, sa.q, sa.qd, ax=sa.ax, av=sa.av, detached=sa.detached,
                    fext=np.zeros((f.n_apples, 3)))
    np.testing.assert_allclose(ev["tension"], f.apple_mass * I.GRAVITY, rtol=1e-8)


# ------------------------------------------------------------------------------------------
# Apple dynamics in closed form
# ------------------------------------------------------------------------------------------
def _one_apple_on_a_post(m=0.2, k_s=1000.0, c_s=None, x0=(0, 0, 0), v0=(0, 0, 0), f_detach=1e9,
                         gravity=(0.0, 0.0, -I.GRAVITY)):
    """An apple on a welded post; x0 is its stem elongation (its world position if detached)."""
    c_s = 2 * 0.2 * math.sqrt(k_s * m) if c_s is None else c_s
    mm, com, inertia = I.cylinder(0.05, 1.0, 700.0)
    post = dict(parent=-1, ndof=0, mass=mm, com=com, inertia=inertia, length=1.0, diam=0.05)
    apple = dict(body=0, hang_local=(0.0, 0.0, 1.0), attach_local=(0.0, 0.0, 1.0), mass=m, k_s=k_s, c_s=c_s,
                 f_detach=f_detach, x0=x0, v0=v0)
    return I.from_bodies([post], apples=[apple], gravity=gravity)


def test_attached_apple_is_the_implicit_damped_oscillator():
    """Hang point fixed (welded post): (m + dt c + dt^2 k) v' = m v - dt k y, y' = y + dt v' about
    the sag equilibrium; closed form by Sylvester's formula."""
    m, k, c = 0.2, 1000.0, 0.8
    sag = m * I.GRAVITY / k
    y0 = -0.004
    f = _one_apple_on_a_post(m=m, k_s=k, c_s=c, x0=(0.0, 0.0, -sag + y0))
    fl = I.Flags()
    n = 300
    ys = []
    st = None
    for t in range(n):
        st, _ = O.rollout(f, fl, 1, state=st, step0=t, n_threads=1)
        ys.append(st.ax[0, 2] + sag)  # the state is the elongation below the hang point
    # the apple recurrence is the single-hinge one with J -> m, kd -> c, k -> k, alpha = 1
    ref = _closed_form_hinge(m, k, c, fl.dt, 1, y0, 0.0, n)
    np.testing.assert_allclose(ys, ref, atol=1e-13)
    assert np.abs(st.ax[0, :2]).max() < 1e-15


def test_detached_apple_is_a_discrete_projectile():
    v0 = np.array([0.3, -0.2, 1.5])
    f = _one_apple_on_a_post(x0=(0.1, 0.2, 0.5), v0=tuple(v0))
    st = O.OracleState.initial(f)
    st.detached[:] = 1
    fl = I.Flags()
    n = 250
    st, _ = O.rollout(f, fl, n, state=st, n_threads=1)
    g = f.gravity[0]
    expect = np.array([0.1, 0.2, 0.5]) + n * fl.dt * v0 + fl.dt ** 2 * g * n * (n + 1) / 2
    np.testing.assert_allclose(st.ax[0], expect, atol=1e-12)
    np.testing.assert_allclose(st.av[0], v0 + n * fl.dt * g, atol=1e-12)


# ------------------------------------------------------------------------------------------
# Detachment (Sec. IV-C): pull path and tension path with their hysteresis
# ------------------------------------------------------------------------------------------
def test_pull_path_detach_step_from_ramp():
    """Pull P_n = rate * n; the counter first passes f_det at n1 = floor(f_det / rate) + 1 and the
    stem breaks N_p steps of P > f_det later: detach step n1 + N_p - 1."""
    fdet, rate = 14.3, 0.05
    m = 0.2
    sag = m * I.GRAVITY / 1000.0
    f = _one_apple_on_a_post(m=m, x0=(0.0, 0.0, -sag), f_detach=fdet)
    fl = I.Flags()
    st = None
    for t in range(400):
        f.pull_force[0] = (rate * t, 0.0, 0.0)
        f.pull_start[0], f.pull_end[0] = 0, 1 << 30
        st, _ = O.rollout(f, fl, 1, state=st, step0=t, n_threads=1)
    n1 = math.floor(fdet / rate) + 1
    assert st.detached[0] == 1
    assert st.detach_step[0] == n1 + fl.n_pull - 1


def test_tension_path_detach_step_from_oscillator():
    """No pull; a downward kick stretches the stem. The stem tension T_n = k |x_n - x_hang| follows
    the implicit oscillator closed form, and the stem breaks after N_t consecutive steps with
    T > gamma f_det."""
    m, k, c = 0.2, 1000.0, 0.8
    fdet = 10.0
    sag = m * I.GRAVITY / k
    vkick = -1.25
    f = _one_apple_on_a_post(m=m, k_s=k, c_s=c, x0=(0.0, 0.0, -sag), v0=(0.0, 0.0, vkick), f_detach=fdet)
    fl = I.Flags()
    st, _ = O.rollout(f, fl, 200, n_threads=1)
    # closed form of the displacement from the sag equilibrium, state before each step
    n = 200
    H = m + fl.dt * c + fl.dt ** 2 * k
    a = fl.dt * (fl.dt * k + c) / H
    A = np.array([[1 - fl.dt ** 2 * k / H, fl.dt * (1 - a)], [-fl.dt * k / H, 1 - a]])
    x = np.array([0.0, vkick])
    thr = fl.gamma_tension * fdet
    cnt, expect = 0, None
    for t in range(n):
        tension = k * abs(x[0] - sag)  # stretch below the hang point is sag - y
        cnt = cnt + 1 if tension > thr else 0
        if cnt >= fl.n_tension:
            expect = t
            break
        x = A @ x
    assert expect is not None and expect > fl.n_tension
    assert st.detached[0] == 1 and st.detach_step[0] == expect


# ------------------------------------------------------------------------------------------
# Rupture (Sec. IV-B): quasi-static break step and the freed hinge swinging at gravity rate
# ------------------------------------------------------------------------------------------
def test_quasi_static_break_step():
    """A single compliant segment loaded at its tip through a light apple by a slow ramp F = rho t:
    past the transients the joint moment follows the static balance k theta = F l cos(theta)
    delayed by the ramp lag of the damped system, (kd + c_s l^2) / k (plus one step for the
    implicit spring), so the first step with k |theta| > M_max is predicted; the break lands N_b steps
    later, to within one step."""
    d, l, rho_w, E, sigma = 0.01, 0.2, 700.0, 1e9, 1e6
    m, com, inertia = I.cylinder(d, l, rho_w)
    k = I.beam_stiffness(E, d, l)
    J = inertia[0] + m * (l / 2) ** 2
    kd = 2 * 1.0 * math.sqrt(k * J)
    mmax = I.rupture_moment(sigma, d)
    body = dict(parent=-1, ndof=1, mass=m, com=com, inertia=inertia, k=k, kd=kd, m_max=mmax, length=l, diam=d)
    ma, ks = 0.002, 1000.0
    apple = dict(body=0, hang_local=(0.0, 0.0, l), attach_local=(0.0, 0.0, l), mass=ma, k_s=ks,
                 c_s=2 * math.sqrt(ks * ma), f_detach=1e9, x0=(0.0, 0.0, 0.0))
    f = I.from_bodies([body], apples=[apple], gravity=(0.0, 0.0, 0.0))
    fl = I.Flags(clamp_factor=1e9)
    rate = 0.02 * mmax / l / fl.dt / 100  # reaches the break load in about 5000 steps
    st = None
    for t in range(8000):
        f.pull_force[0] = (0.0, rate * t * fl.dt, 0.0)
        f.pull_start[0], f.pull_end[0] = 0, 1 << 30
        st, _ = O.rollout(f, fl, 1, state=st, step0=t, n_threads=1)
        if st.broken[0]:
            break
    # static balance k theta = F l cos(theta) at theta = M_max / k; ramp lag of the damped system,
    # whose rotational damping is kd plus the apple's damper c_s at lever l, plus one step
    theta = mmax / k
    t_cross = mmax / (l * math.cos(theta) * rate) + (kd + apple["c_s"] * l * l) / k + fl.dt
    n_cross = math.ceil(t_cross / fl.dt)
    assert st.broken[0] == 1
    assert abs(st.break_step[0] - (n_cross + fl.n_break - 1)) <= 1


def test_broken_joint_swings_as_a_physical_pendulum():
    """A broken joint is a free hinge (gain rows zeroed, Sec. IV-B): a segment hanging from it
    swings at the small-angle period 2 pi sqrt(J / (m g l / 2)), J about the hinge."""
    d, l = 0.01, 0.2
    m, com, inertia = I.cylinder(d, l, 700.0)
    down = (0.0, 1.0, 0.0, 0.0)  # 180 degrees about x: the segment hangs straight down
    body = dict(parent=-1, ndof=1, qrel=down, mass=m, com=com, inertia=inertia, k=50.0, kd=0.0, m_max=1e30,
                length=l, diam=d)
    f = I.from_bodies([body], gravity=(0.0, 0.0, -I.GRAVITY))
    f.q0[0] = 0.01
    st = O.OracleState.initial(f)
    st.broken[:] = 1
    fl = I.Flags(dt=5e-4)
    J = inertia[0] + m * (l / 2) ** 2
    period = 2 * math.pi * math.sqrt(J / (m * I.GRAVITY * l / 2))
    n = int(5 * period / fl.dt)
    _, rec = O.rollout(f, fl, n, state=st, record_q=True, n_threads=1)
    q = np.concatenate([[0.01], rec["q"][:, 0]])
    idx = np.nonzero((q[:-1] > 0) & (q[1:] <= 0))[0]
    tc = (idx + q[idx] / (q[idx] - q[idx + 1])) * fl.dt
    assert np.mean(np.diff(tc)) == pytest.approx(period, rel=2e-3)
    assert np.abs(q).max() == pytest.approx(0.01, rel=1e-3)  # no spring, no damper: no decay


# ------------------------------------------------------------------------------------------
# Energy: damping off, no events, gravity on
# ------------------------------------------------------------------------------------------
def _energy(f, fl, q, qd):
    ev = O.evaluate(f, fl, 0, q, qd)
    g = f.gravity[0]
    k = np.concatenate([np.full(f.ndof[b], f.k[b]) for b in range(f.n_bodies)])
    return 0.5 * qd @ ev["M"] @ qd + 0.5 * np.sum(k * q * q) - np.sum(f.mass * (ev["com"] @ g))


def test_energy_bounded_and_first_order_in_dt():
    f = T.small_random_tree(11, n_b=9, depth=4)
    f.k = f.k * 1e-3
    f.kd[:] = 0.0
    errs = []
    for dt, n in ((2e-4, 2000), (1e-4, 4000)):
        fl = I.Flags(alpha_implicit_spring=0, dt=dt)
        _, rec = O.rollout(f, fl, n, record_q=True, n_threads=1)
        qs = np.vstack([np.zeros(f.n_dofs), rec["q"]])
        qd = np.diff(qs, axis=0) / dt
        E0 = _energy(f, fl, np.zeros(f.n_dofs), np.zeros(f.n_dofs))
        Es = np.array([_energy(f, fl, qs[i + 1], qd[i]) for i in range(0, n, 10)])
        scale = np.ptp(-np.array([np.sum(f.mass * (O.evaluate(f, fl, 0, qs[i], qd[0])["com"] @ f.gravity[0]))
                                  for i in range(0, n, 100)]))
        errs.append(np.abs(Es - E0).max())
        assert errs[-1] < 0.05 * scale
    assert errs[0] / errs[1] == pytest.approx(2.0, rel=0.2)


def test_post_break_friction_ramp():
    """After a break the joint keeps only the torn-fibre friction, read as an implicit viscous
    damper ramping from kd to 5 kd over 1.5 s (Sec. IV-B). A single broken hinge hanging under
    gravity then follows the scalar recurrence (J + dt c_n) D = dt (-m g (l/2) sin q - c_n qd),
    c_n = kd (1 + 4 min(n dt / 1.5, 1)), with n counted from the break step."""
    d, l, kd = 0.01, 0.2, 2e-3
    m, com, inertia = I.cylinder(d, l, 700.0)
    down = (0.0, 1.0, 0.0, 0.0)
    body = dict(parent=-1, ndof=1, qrel=down, mass=m, com=com, inertia=inertia, k=50.0, kd=kd, m_max=1e30,
                length=l, diam=d)
    f = I.from_bodies([body], gravity=(0.0, 0.0, -I.GRAVITY))
    f.q0[0] = 0.5
    st = O.OracleState.initial(f)
    st.broken[:] = 1
    st.break_step[:] = -100
    fl = I.Flags(dt=2e-3)
    n = 1200
    _, rec = O.rollout(f, fl, n, state=st, record_q=True, n_threads=1)
    J = inertia[0] + m * (l / 2) ** 2
    q, qd = 0.5, 0.0
    ref = []
    for t in range(n):
        c = kd * (1 + 4 * min((t + 100) * fl.dt / 1.5, 1.0))
        tau = -m * I.GRAVITY * (l / 2) * math.sin(q)
        D = fl.dt * (tau - c * qd) / (J + fl.dt * c)
        qd += D
        q += fl.dt * qd
        ref.append(q)
    np.testing.assert_allclose(rec["q"][:, 0], ref, atol=1e-12)
    assert abs(ref[-1]) < 0.3  # the swing decays
