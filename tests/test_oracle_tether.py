"""Pins of the oracle's stem coupling (Sec. IV-C, Eqs. 6-7; App. B), CPU only.

Each test derives its expectation independently of the oracle's Schur-complement form:

* the reaction clamp (Eq. 7, "clamped to a maximum", read as F_clamp = 1.2 f_det) scales the
  whole coupled reaction, force and stiffness, by F_clamp / |f_react|, with |f_react| taken
  from the inputs (stem force minus the weight), and is continuous at the threshold;
* on a snapped sub-tree (its own joint or a joint above broken) applied forces are disabled
  (App. B): the tree moves exactly as the bare tree while the stem still acts on the apple;
* the coupled backward-Euler step of tree and apple, written as one unreduced linear system
  in the hinge increment and the apple's new velocity and solved densely, matches the
  oracle's trajectory step for step.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2607_06337_b300 import inputs as I
from tests.test_oracle_pins import _closed_form_hinge

pytestmark = pytest.mark.usefixtures("oracle_lib")

G = I.GRAVITY


def _hinge_with_apple(l=0.2, d=0.02, k=50.0, kd=0.05, ma=0.2, k_s=1000.0, c_s=None, f_det=1e9, gravity=True,
                      u0=(0.0, 0.0, 0.0), v0=(0.0, 0.0, 0.0)):
    """One segment on a single hinge about x (along +z at rest), an apple hung at its tip."""
    m, com, inertia = I.cylinder(d, l, 700.0)
    body = dict(parent=-1, ndof=1, mass=m, com=com, inertia=inertia, k=k, kd=kd, length=l, diam=d)
    c_s = 2 * 0.2 * math.sqrt(k_s * ma) if c_s is None else c_s
    apple = dict(body=0, hang_local=(0.0, 0.0, l), attach_local=(0.0, 0.0, l), mass=ma, k_s=k_s, c_s=c_s,
                 f_detach=f_det, x0=u0, v0=v0)
    g = (0.0, 0.0, -G) if gravity else (0.0, 0.0, 0.0)
    f = I.from_bodies([body], apples=[apple], tips=[(0, (0.0, 0.0, l))], gravity=g)
    J = inertia[0] + m * (l / 2) ** 2
    return f, dict(l=l, m=m, J=J, k=k, kd=kd, ma=ma, k_s=k_s, c_s=c_s)


# ------------------------------------------------------------------------------------------
# Reaction clamp (Sec. IV-C, Eq. 7)
# ------------------------------------------------------------------------------------------
def _loads(f, fl, theta, thetad, u, v=(0.0, 0.0, 0.0), with_apple=True):
    ax = np.array([u], np.float64) if with_apple else None
    av = np.array([v], np.float64) if with_apple else None
    return O.evaluate(f, fl, 0, [theta], [thetad], ax=ax, av=av, detached=np.zeros(1, np.int32),
                      fext=np.zeros((1, 3)))


@pytest.mark.parametrize("over", [1.5, 4.0])
def test_reaction_clamp_scales_force_and_coupling_alike(over):
    """Stem stretched sideways so that |f_react| = |k_s u - m g| is `over` times F_clamp: the
    transmitted force, the generalised force on the hinge and the coupling stiffness the apple
    adds to H are all the unclamped ones times F_clamp / |f_react|."""
    f_det = 12.0
    f, p = _hinge_with_apple(f_det=f_det)
    f_clamp = 1.2 * f_det
    sag = np.array([0.0, 0.0, -p["ma"] * G / p["k_s"]])
    side = np.array([0.3, 0.8, 0.0]) / math.hypot(0.3, 0.8)
    u = sag + over * f_clamp / p["k_s"] * side          # stem force beyond the weight: over * F_clamp
    f_react = np.linalg.norm(p["k_s"] * u + np.array([0.0, 0.0, p["ma"] * G]))
    assert f_react == pytest.approx(over * f_clamp, rel=1e-12)
    th, thd, v = 0.08, -0.4, (0.05, -0.1, 0.2)
    clamped = _loads(f, I.Flags(), th, thd, u, v)
    free = _loads(f, I.Flags(clamp_factor=1e9), th, thd, u, v)
    bare = _loads(f, I.Flags(), th, thd, u, v, with_apple=False)
    sc = f_clamp / f_react
    np.testing.assert_allclose(clamped["fapp"], sc * free["fapp"], rtol=1e-12, atol=0)
    dM_free, dM_clamped = free["M"] - bare["M"], clamped["M"] - bare["M"]
    assert dM_free[0, 0] > 1e-3 * bare["M"][0, 0]         # the coupling is really there
    np.testing.assert_allclose(dM_clamped, sc * dM_free, rtol=1e-12)
    np.testing.assert_allclose(clamped["c"] - bare["c"], sc * (free["c"] - bare["c"]), rtol=1e-12)


def test_reaction_clamp_leaves_loads_below_the_threshold_alone():
    f_det = 12.0
    f, p = _hinge_with_apple(f_det=f_det)
    sag = np.array([0.0, 0.0, -p["ma"] * G / p["k_s"]])
    u = sag + 0.9 * 1.2 * f_det / p["k_s"] * np.array([0.0, 1.0, 0.0])
    a = _loads(f, I.Flags(), 0.05, 0.1, u)
    b = _loads(f, I.Flags(clamp_factor=1e9), 0.05, 0.1, u)
    np.testing.assert_array_equal(a["fapp"], b["fapp"])
    np.testing.assert_array_equal(a["M"], b["M"])


def test_reaction_clamp_is_continuous_at_the_threshold():
    """Across |f_react| = F_clamp the clamped loads move by the same O(eps) as the input."""
    f_det = 12.0
    f, p = _hinge_with_apple(f_det=f_det)
    f_clamp = 1.2 * f_det
    sag = np.array([0.0, 0.0, -p["ma"] * G / p["k_s"]])
    side = np.array([0.0, 1.0, 0.0])
    eps = 1e-7
    lo = _loads(f, I.Flags(), 0.05, 0.1, sag + (1 - eps) * f_clamp / p["k_s"] * side)
    hi = _loads(f, I.Flags(), 0.05, 0.1, sag + (1 + eps) * f_clamp / p["k_s"] * side)
    scale = np.abs(lo["fapp"]).max()
    assert np.abs(hi["fapp"] - lo["fapp"]).max() < 10 * eps * scale
    assert np.abs(hi["M"] - lo["M"]).max() < 10 * eps * np.abs(lo["M"]).max()
    # while a clamp that scaled the force alone, or by the wrong threshold, would jump here:
    # the force just above the threshold has magnitude F_clamp times its unclamped direction
    free = _loads(f, I.Flags(clamp_factor=1e9), 0.05, 0.1, sag + (1 + eps) * f_clamp / p["k_s"] * side)
    np.testing.assert_allclose(hi["fapp"], free["fapp"] / (1 + eps), rtol=1e-12)


# ------------------------------------------------------------------------------------------
# Snapped sub-trees transmit no applied force (App. B)
# ------------------------------------------------------------------------------------------
def _chain3(apple_body=2, apple=True, gravity=(0.0, 0.0, 0.0), u0=(0.0, 0.004, 0.0), l=0.25, d=0.02):
    """Three vertical segments on x hinges (compliant root), an apple at the tip of one of
    them with its stem stretched sideways."""
    m, com, inertia = I.cylinder(d, l, 700.0)
    k = I.beam_stiffness(8e9, d, l) * 1e-3
    bodies = [dict(parent=i - 1, ndof=1, jpos=(0.0, 0.0, 0.0 if i == 0 else l), mass=m, com=com,
                   inertia=inertia, k=k, kd=0.05 * k, length=l, diam=d) for i in range(3)]
    ma, ks = 0.2, 1000.0
    apples = [dict(body=apple_body, hang_local=(0.0, 0.0, l), attach_local=(0.0, 0.0, l), mass=ma, k_s=ks,
                   c_s=0.8, f_detach=1e9, x0=u0)] if apple else []
    f = I.from_bodies(bodies, apples=apples, tips=[(2, (0.0, 0.0, l))], gravity=gravity)
    return f, ma, ks, 0.8


def _run_steps(f, st, n, fl):
    qs, us = [], []
    for t in range(n):
        st, _ = O.rollout(f, fl, 1, state=st, step0=t, n_threads=1)
        qs.append(st.q.copy())
        if f.n_apples:
            us.append(st.ax[0].copy())
    return st, np.array(qs), np.array(us)


@pytest.mark.parametrize("broken_body,apple_body", [(1, 2), (2, 2), (1, 1)])
def test_snapped_subtree_transmits_no_reaction(broken_body, apple_body):
    """Chain at rest, no gravity, stem stretched sideways. With a joint at or above the
    apple's body broken the tree never moves (q stays exactly 0) and the apple is the implicit
    damped oscillator about its fixed hang point; with nothing broken the same stem pulls the
    chain over."""
    f, ma, ks, cs = _chain3(apple_body=apple_body)
    fl = I.Flags()
    n = 300
    st = O.OracleState.initial(f)
    st.broken[broken_body] = 1
    st.break_step[broken_body] = -1000
    st, qs, us = _run_steps(f, st, n, fl)
    assert np.abs(qs).max() == 0.0 and np.abs(st.qd).max() == 0.0
    ref = _closed_form_hinge(ma, ks, cs, fl.dt, 1, 0.004, 0.0, n)
    np.testing.assert_allclose(us[:, 1], ref, atol=1e-15)
    assert np.abs(us[:, [0, 2]]).max() == 0.0
    # control: nothing broken, the reaction bends the chain
    _, qc, _ = _run_steps(f, None, 50, fl)
    assert np.abs(qc).max() > 1e-5


def test_snapped_subtree_moves_as_the_bare_tree():
    """Swinging under gravity with the middle joint broken: the chain with an apple on its
    snapped tip segment follows the bare chain's trajectory exactly."""
    g = (0.0, 0.0, -G)
    fa, *_ = _chain3(apple=True, gravity=g, u0=(0.003, 0.004, -0.002))
    fb, *_ = _chain3(apple=False, gravity=g)
    for f in (fa, fb):
        f.q0[:] = (0.02, 0.01, -0.015)
    fl = I.Flags()
    sa, sb = O.OracleState.initial(fa), O.OracleState.initial(fb)
    for s in (sa, sb):
        s.broken[1] = 1
        s.break_step[1] = 0
    _, ra = O.rollout(fa, fl, 400, state=sa, record_q=True, n_threads=1)
    _, rb = O.rollout(fb, fl, 400, state=sb, record_q=True, n_threads=1)
    assert np.abs(rb["q"]).max() > 0.01
    np.testing.assert_array_equal(ra["q"], rb["q"])


# ------------------------------------------------------------------------------------------
# Coupled backward-Euler step of the tree and the stem (Sec. IV-C, Eqs. 6-7)
# ------------------------------------------------------------------------------------------
def _unreduced_step(p, dt, gvec, th, thd, u, v):
    """One step of the hinge and its apple as a single linear system in (Delta, v').

    Tree:  (J + dt kd + dt^2 k) Delta = dt (-k (th + dt thd) - kd thd - c(th) + J_h^T f_R')
    Apple: m (v' - v) = dt (-k_s u' - c_s v' + m g)
    with u' = u + dt (v' - J_h (thd + Delta)) the stem elongation at the step's end,
    f_R' = k_s u' - m g its reaction beyond the static weight, J_h = d x_hang / d th at the
    step's start and c(th) = -m_b |g| (l/2) sin(th) the hinge's gravity bias.
    """
    l, J, k, kd = p["l"], p["J"], p["k"], p["kd"]
    ma, ks, cs = p["ma"], p["k_s"], p["c_s"]
    Jh = np.array([0.0, -l * math.cos(th), -l * math.sin(th)])
    bias = p["m"] * gvec[2] * (l / 2) * math.sin(th)     # -m_b |g| (l/2) sin th
    A = np.zeros((4, 4))
    b = np.zeros(4)
    # tree row: move the implicit parts of f_R' (through u') to the left
    A[0, 0] = J + dt * kd + dt * dt * k + dt * dt * ks * (Jh @ Jh)
    A[0, 1:] = -dt * dt * ks * Jh
    b[0] = dt * (-k * (th + dt * thd) - kd * thd - bias + Jh @ (ks * (u - dt * Jh * thd) - ma * gvec))
    # apple rows
    A[1:, 1:] = (ma + dt * cs + dt * dt * ks) * np.eye(3)
    A[1:, 0] = -dt * dt * ks * Jh
    b[1:] = ma * v + dt * (-ks * (u - dt * Jh * thd) + ma * gvec)
    x = np.linalg.solve(A, b)
    thd_n = thd + x[0]
    v_n = x[1:]
    u_n = u + dt * (v_n - Jh * thd_n)
    return th + dt * thd_n, thd_n, u_n, v_n


@pytest.mark.parametrize("gravity", [False, True])
def test_coupled_tether_step_is_the_unreduced_backward_euler_system(gravity):
    """A heavy apple on a light hinge (strong coupling): 400 oracle steps against the
    unreduced system solved densely, from a displaced and moving start."""
    f, p = _hinge_with_apple(gravity=gravity, u0=(0.0, 0.002, -0.001), v0=(0.01, -0.05, 0.02))
    sag = np.array([0.0, 0.0, -p["ma"] * G / p["k_s"]]) if gravity else np.zeros(3)
    f.apple_x0[0] = np.array([0.0, 0.002, -0.001]) + sag
    f.q0[0] = 0.05
    f.qd0[0] = 0.3
    fl = I.Flags()
    gvec = f.gravity[0]
    th, thd, u, v = 0.05, 0.3, f.apple_x0[0].copy(), f.apple_v0[0].copy()
    st = None
    errs, ths = [], []
    for t in range(400):
        st, _ = O.rollout(f, fl, 1, state=st, step0=t, n_threads=1)
        th, thd, u, v = _unreduced_step(p, fl.dt, gvec, th, thd, u, v)
        ths.append(th)
        errs.append(max(abs(st.q[0] - th) / 0.05, abs(st.qd[0] - thd) / 0.3,
                        np.abs(st.ax[0] - u).max() / 0.002, np.abs(st.av[0] - v).max() / 0.05))
    assert max(errs) < 1e-11, max(errs)
    # the apple really drives the hinge: the bare hinge (no apple, no gravity) rings differently
    bare = _closed_form_hinge(p["J"], p["k"], p["kd"], fl.dt, 1, 0.05, 0.3, 400)
    assert np.abs(np.array(ths) - bare).max() > 0.1 * np.abs(bare).max()
