"""Pins of the FP64 oracle against closed forms, brute force and invariants (CPU only).

Each test names the paper passage or the textbook result it checks. Between them they fail on
a dropped term, a wrong sign, a transposed operand or a wrong index anywhere in the oracle's
kinematics, mass matrix, bias forces, solve, apple tether, rupture and detachment logic.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2607_06337_b300 import inputs as I
from tests import _trees as T

pytestmark = pytest.mark.usefixtures("oracle_lib")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------------------------------
# Closed forms printed in or following directly from the paper
# ------------------------------------------------------------------------------------------
def test_paper_parameter_closed_forms():
    """Eq. 4 (k = pi E r^4 / (4 l)) and Eq. 5 (M_max = sigma_r pi r^3 / 4) on the paper's
    printed defaults (Table: E = 7 GPa, sigma_r = 50 MPa, trunk radius 0.035 m)."""
    g = json.load(open(os.path.join(GOLDEN, "paper_params.json")))
    for case in g["cases"]:
        d = 2 * case["r_m"]
        assert I.beam_stiffness(case["E_Pa"], d, case["l_m"]) == pytest.approx(case["k_Nm_per_rad"], rel=1e-4)
        assert I.rupture_moment(case["sigma_r_Pa"], d) == pytest.approx(case["M_max_Nm"], rel=1e-4)
    # generated descriptors obey the same closed forms body by body
    f = I.make_forest(I.PLAIN, worlds=[0, 1])
    wid = np.repeat(np.arange(2), np.diff(f.body_off))
    E = f.meta["E"][wid]
    sig = f.meta["sigma_r"][wid]
    r = f.diam / 2
    nonroot = f.parent >= 0
    np.testing.assert_allclose(f.k[nonroot], (math.pi * E * r ** 4 / (4 * f.length))[nonroot], rtol=1e-14)
    np.testing.assert_allclose(f.m_max, sig * math.pi * r ** 3 / 4, rtol=1e-14)
    # pipe rule with exponent 2: d_parent^2 = sum of children's d^2 (Eq. 2, beta = 2)
    for w in range(2):
        b0, b1 = f.body_off[w], f.body_off[w + 1]
        par = f.parent[b0:b1]
        d2 = f.diam[b0:b1] ** 2
        sums = np.zeros(b1 - b0)
        np.add.at(sums, par[par >= 0], d2[par >= 0])
        inner = sums > 0
        np.testing.assert_allclose(d2[inner], sums[inner], rtol=1e-12)


# ------------------------------------------------------------------------------------------
# Kinematics: rest transform and orthonormal frames
# ------------------------------------------------------------------------------------------
def test_rest_pose_reproduces_skeleton():
    """Sec. IV Eq. 3: at q = 0 the articulation reproduces the generated skeleton exactly."""
    f = I.make_forest(I.PLAIN, worlds=[0, 3])
    fl = I.Flags()
    for w in range(2):
        b0, b1 = f.body_off[w], f.body_off[w + 1]
        nv = int(f.ndof[b0:b1].sum())
        ev = O.evaluate(f, fl, w, np.zeros(nv), np.zeros(nv))
        np.testing.assert_allclose(ev["x"], f.rest_x[b0:b1], atol=1e-12)
        np.testing.assert_allclose(ev["R"], f.rest_R[b0:b1], atol=1e-12)


def test_frames_orthonormal_random_q():
    f = I.make_forest(I.PLAIN, worlds=[1])
    rng = np.random.default_rng(0)
    q = rng.uniform(-1, 1, f.n_dofs)
    ev = O.evaluate(f, I.Flags(), 0, q, np.zeros(f.n_dofs))
    for R in ev["R"]:
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-12)


def test_rest_is_stress_free_without_gravity():
    """No gravity, q = 0, qd = 0: the bias force vanishes (stress-free rest, Sec. IV Eq. 3)."""
    f = I.make_forest(I.PLAIN, worlds=[2])
    f.gravity[:] = 0
    ev = O.evaluate(f, I.Flags(), 0, np.zeros(f.n_dofs), np.zeros(f.n_dofs))
    assert np.abs(ev["c"]).max() == 0.0


# ------------------------------------------------------------------------------------------
# Single hinge: the discrete oscillator in closed form
# ------------------------------------------------------------------------------------------
def _closed_form_hinge(J, k, kd, dt, alpha, q0, qd0, n):
    """q_n of the scalar recurrence (J + dt kd + alpha dt^2 k) D = dt(-k(q + alpha dt qd) - kd qd),
    qd' = qd + D, q' = q + dt qd', by Sylvester's formula A^n = (l1^n (A - l2) - l2^n (A - l1)) / (l1 - l2)."""
    H = J + dt * kd + alpha * dt * dt * k
    a = dt * (alpha * dt * k + kd) / H
    A = np.array([[1 - dt * dt * k / H, dt * (1 - a)], [-dt * k / H, 1 - a]], dtype=complex)
    tr, det = A[0, 0] + A[1, 1], A[0, 0] * A[1, 1] - A[0, 1] * A[1, 0]
    disc = np.sqrt(tr * tr - 4 * det + 0j)
    l1, l2 = (tr + disc) / 2, (tr - disc) / 2
    out = []
    x0 = np.array([q0, qd0], dtype=complex)
    for m in range(1, n + 1):
        An = (l1 ** m * (A - l2 * np.eye(2)) - l2 ** m * (A - l1 * np.eye(2))) / (l1 - l2)
        out.append((An @ x0)[0].real)
    return np.array(out)


@pytest.mark.parametrize("alpha,kd", [(0, 0.0), (1, 0.0), (0, 0.3), (1, 0.3)])
def test_single_hinge_closed_form(alpha, kd):
    """One body on a single hinge, no gravity: the full machinery (FK, M by Jacobians, bias,
    solve) reduces to the scalar recurrence with J = m (3 r^2 + l^2) / 12 + m (l / 2)^2."""
    f, J, m = T.single_hinge(k=50.0, kd=kd)
    f.q0[0] = 0.05
    fl = I.Flags(alpha_implicit_spring=alpha)
    st, rec = O.rollout(f, fl, 400, record_q=True, n_threads=1)
    ref = _closed_form_hinge(J, 50.0, kd, fl.dt, alpha, 0.05, 0.0, 400)
    np.testing.assert_allclose(rec["q"][:, 0], ref, atol=1e-12 * 0.05 * 400)


def test_single_hinge_period_converges_to_sqrt_k_over_J():
    """Undamped explicit-spring hinge: the discrete solution obeys q_(n+1) + q_(n-1) = 2 cos(phi) q_n
    with cos(phi) = 1 - (w dt)^2 / 2, w = sqrt(k / J), so the period 2 pi dt / phi tends to
    2 pi / w with an O(dt^2) error."""
    errs = []
    for dt in (5e-4, 2.5e-4):
        f, J, m = T.single_hinge(k=50.0)
        f.q0[0] = 0.01
        fl = I.Flags(alpha_implicit_spring=0, dt=dt)
        omega = math.sqrt(50.0 / J)
        _, rec = O.rollout(f, fl, 2000, record_q=True, n_threads=1)
        q = np.concatenate([[0.01], rec["q"][:, 0]])
        mid = np.abs(q[1:-1]) > 1e-3
        cosphi = ((q[2:] + q[:-2]) / (2 * q[1:-1]))[mid]
        np.testing.assert_allclose(cosphi, 1 - (omega * dt) ** 2 / 2, rtol=1e-10)
        phi = math.acos(float(np.mean(cosphi)))
        period = 2 * math.pi * dt / phi
        errs.append(abs(period - 2 * math.pi / omega) / (2 * math.pi / omega))
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.01)


# ------------------------------------------------------------------------------------------
# Discrete cantilever: static tip deflection under a tip force (static bends)
# ------------------------------------------------------------------------------------------
def test_cantilever_static_deflection():
    """N equal segments on compliant hinges k = E I / l, tip force F through an apple tether:
    the small-angle static tip deflection is F L^3 N(N+1)(2N+1) / (6 N^3 E I), which tends to
    the Euler-Bernoulli F L^3 / (3 E I) with relative excess 3 / (2N) + 1 / (2N^2)."""
    N, L, d, rho, E = 8, 1.0, 0.01, 700.0, 1e9
    F = 1e-3
    ma = 0.01
    apple = dict(mass=ma, k_s=1000.0, c_s=2 * 1.0 * math.sqrt(1000.0 * ma), f_detach=1e9)
    f, k = T.chain(N, L / N, d, rho, E, kd=0.5, apple=apple)
    f.pull_force[0] = (0.0, F, 0.0)
    f.pull_start[0] = 0
    fl = I.Flags(dt=0.02, alpha_implicit_spring=1)
    st, _ = O.rollout(f, fl, 6000, n_threads=1)
    assert np.abs(st.qd).max() < 1e-12
    ev = O.evaluate(f, fl, 0, st.q, st.qd)
    tip = ev["x"][-1] + ev["R"][-1] @ np.array([0, 0, L / N])
    EI = E * math.pi * (d / 2) ** 4 / 4
    delta = F * L ** 3 * N * (N + 1) * (2 * N + 1) / (6 * N ** 3 * EI)
    assert tip[1] == pytest.approx(delta, rel=1e-5)
    eb = F * L ** 3 / (3 * EI)
    assert delta / eb - 1 == pytest.approx(3 / (2 * N) + 1 / (2 * N * N), rel=1e-12)


# ------------------------------------------------------------------------------------------
# Mass matrix against the kinetic-energy Hessian (finite differences of FK)
# ------------------------------------------------------------------------------------------
def _kinetic(f, fl, q, u, h=1e-6):
    """T(u) = 1/2 sum_b (m |v_c|^2 + w^T I w), velocities from central differences of FK."""
    a = O.evaluate(f, fl, 0, q + h * u, np.zeros_like(q))
    b = O.evaluate(f, fl, 0, q - h * u, np.zeros_like(q))
    c = O.evaluate(f, fl, 0, q, np.zeros_like(q))
    Tk = 0.0
    for i in range(f.n_bodies):
        v = (a["com"][i] - b["com"][i]) / (2 * h)
        Wm = (a["R"][i] - b["R"][i]) / (2 * h) @ c["R"][i].T
        w = 0.5 * np.array([Wm[2, 1] - Wm[1, 2], Wm[0, 2] - Wm[2, 0], Wm[1, 0] - Wm[0, 1]])
        Ic = c["R"][i] @ np.diag(f.inertia[i]) @ c["R"][i].T
        Tk += 0.5 * (f.mass[i] * v @ v + w @ Ic @ w)
    return Tk


def test_mass_matrix_is_kinetic_energy_hessian():
    f = T.small_random_tree(1, n_b=7, depth=3)
    fl = I.Flags()
    rng = np.random.default_rng(1)
    q = rng.uniform(-0.4, 0.4, f.n_dofs)
    M = O.evaluate(f, fl, 0, q, np.zeros_like(q))["M"]
    n = f.n_dofs
    E = np.eye(n)
    Tk = [_kinetic(f, fl, q, E[i]) for i in range(n)]
    Mfd = np.zeros((n, n))
    for i in range(n):
        Mfd[i, i] = 2 * Tk[i]
        for j in range(i):
            Mfd[i, j] = Mfd[j, i] = _kinetic(f, fl, q, E[i] + E[j]) - Tk[i] - Tk[j]
    np.testing.assert_allclose(M, Mfd, atol=1e-8 * np.abs(M).max())
    np.testing.assert_allclose(M, M.T, atol=1e-15 * np.abs(M).max())
    assert np.linalg.eigvalsh(M).min() > 0


# ------------------------------------------------------------------------------------------
# Bias force against the Lagrangian form (Christoffel symbols from dM/dq, gravity from dV/dq)
# ------------------------------------------------------------------------------------------
def test_bias_matches_lagrangian():
    f = T.small_random_tree(2, n_b=7, depth=3)
    fl = I.Flags()
    rng = np.random.default_rng(2)
    n = f.n_dofs
    q = rng.uniform(-0.4, 0.4, n)
    qd = rng.uniform(-2, 2, n)
    c = O.evaluate(f, fl, 0, q, qd)["c"]
    h = 1e-6
    dM = []
    dV = np.zeros(n)
    g = f.gravity[0]
    for k in range(n):
        e = np.zeros(n)
        e[k] = h
        a = O.evaluate(f, fl, 0, q + e, qd)
        b = O.evaluate(f, fl, 0, q - e, qd)
        dM.append((a["M"] - b["M"]) / (2 * h))
        Va = -np.sum(f.mass * (a["com"] @ g))
        Vb = -np.sum(f.mass * (b["com"] @ g))
        dV[k] = (Va - Vb) / (2 * h)
    dM = np.array(dM)  # dM[k] = dM/dq_k
    Mdot = np.einsum("kij,k->ij", dM, qd)
    cl = Mdot @ qd - 0.5 * np.einsum("kij,i,j->k", dM, qd, qd) + dV
    np.testing.assert_allclose(c, cl, atol=1e-6 * np.abs(c).max())


# ------------------------------------------------------------------------------------------
# Brute-force maximal-coordinate Newton-Euler (KKT) on trees of <= 8 bodies
# ------------------------------------------------------------------------------------------
def _skew(v):
    return np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])


def _kkt_qdd(f, q, qd, tau):
    """Joint accelerations from 6 unknowns per body, joint constraints at acceleration level and
    one dense KKT solve; tau are the joint torques along the DOF axes."""
    nb = f.n_bodies
    axes, dof_body, Rb = T.joint_axes(f, q)
    ev = O.evaluate(f, I.Flags(), 0, q, qd)
    x, com = ev["x"], ev["com"]
    g = f.gravity[0]
    # angular velocities and com velocities by a direct forward pass
    w = np.zeros((nb, 3))
    dof0 = np.concatenate([[0], np.cumsum(f.ndof)])[:-1]
    for b in range(nb):
        p = f.parent[b]
        w[b] = 0 if p < 0 else w[p]
        for j in range(f.ndof[b]):
            w[b] = w[b] + axes[dof0[b] + j] * qd[dof0[b] + j]
    nacc = 6 * nb
    rows, rhs = [], []
    for b in range(nb):
        p = f.parent[b]
        rb = x[b] - com[b]
        # joint point acceleration equal from both sides
        Ab = np.zeros((3, nacc))
        Ab[:, 6 * b:6 * b + 3] = np.eye(3)
        Ab[:, 6 * b + 3:6 * b + 6] = -_skew(rb)
        vb = np.cross(w[b], np.cross(w[b], rb))
        if p >= 0:
            rp = x[b] - com[p]
            Ab[:, 6 * p:6 * p + 3] -= np.eye(3)
            Ab[:, 6 * p + 3:6 * p + 6] -= -_skew(rp)
            vb = vb - np.cross(w[p], np.cross(w[p], rp))
        rows.append(Ab)
        rhs.append(-vb)
        # rotational constraints on the locked directions
        wp = np.zeros(3) if p < 0 else w[p]
        i0 = dof0[b]
        if f.ndof[b] == 2:
            e0, e1 = axes[i0], axes[i0 + 1]
            locked = [np.cross(e0, e1)]
            e0d = np.cross(wp, e0)
            e1d = np.cross(wp + e0 * qd[i0], e1)
            locked_d = [np.cross(e0d, e1) + np.cross(e0, e1d)]
        elif f.ndof[b] == 1:
            Rj = (np.eye(3) if p < 0 else Rb[p]) @ I.quat_to_mat(f.qrel[b])
            locked = [Rj[:, 1], Rj[:, 2]]
            locked_d = [np.cross(wp, u) for u in locked]
        else:
            locked = list(np.eye(3))
            locked_d = [np.zeros(3)] * 3
        dw = w[b] - wp
        for u, ud in zip(locked, locked_d):
            r = np.zeros((1, nacc))
            r[0, 6 * b + 3:6 * b + 6] = u
            if p >= 0:
                r[0, 6 * p + 3:6 * p + 6] = -u
            rows.append(r)
            rhs.append(np.array([-ud @ dw]))
    G = np.vstack(rows)
    gam = np.concatenate(rhs)
    Mb = np.zeros((nacc, nacc))
    fb = np.zeros(nacc)
    for b in range(nb):
        Ic = Rb[b] @ np.diag(f.inertia[b]) @ Rb[b].T
        Mb[6 * b:6 * b + 3, 6 * b:6 * b + 3] = f.mass[b] * np.eye(3)
        Mb[6 * b + 3:6 * b + 6, 6 * b + 3:6 * b + 6] = Ic
        fb[6 * b:6 * b + 3] = f.mass[b] * g
        fb[6 * b + 3:6 * b + 6] = -np.cross(w[b], Ic @ w[b])
    # joint torques: +tau e on the child, -tau e on the parent
    for i, b in enumerate(dof_body):
        fb[6 * b + 3:6 * b + 6] += tau[i] * axes[i]
        p = f.parent[b]
        if p >= 0:
            fb[6 * p + 3:6 * p + 6] -= tau[i] * axes[i]
    m = G.shape[0]
    K = np.block([[Mb, G.T], [G, np.zeros((m, m))]])
    sol = np.linalg.solve(K, np.concatenate([fb, gam]))
    acc = sol[:nacc]
    qdd = np.zeros(f.n_dofs)
    for b in range(nb):
        p = f.parent[b]
        i0 = dof0[b]
        if f.ndof[b] == 0:
            continue
        dal = acc[6 * b + 3:6 * b + 6] - (0 if p < 0 else acc[6 * p + 3:6 * p + 6])
        wp = np.zeros(3) if p < 0 else w[p]
        vt = np.cross(wp, axes[i0]) * qd[i0]
        if f.ndof[b] == 2:
            vt = vt + np.cross(wp + axes[i0] * qd[i0], axes[i0 + 1]) * qd[i0 + 1]
        for j in range(f.ndof[b]):
            qdd[i0 + j] = axes[i0 + j] @ (dal - vt)
    return qdd


@pytest.mark.parametrize("seed,nb,ndof,root", [(3, 5, 2, 0), (4, 8, 2, 0), (5, 6, 1, 1), (6, 8, 2, 2)])
def test_joint_accelerations_match_maximal_coordinate_kkt(seed, nb, ndof, root):
    f = T.small_random_tree(seed, n_b=nb, depth=4, ndof=ndof, root_ndof=root)
    rng = np.random.default_rng(seed)
    n = f.n_dofs
    q = rng.uniform(-0.5, 0.5, n)
    qd = rng.uniform(-3, 3, n)
    tau = rng.uniform(-0.1, 0.1, n)
    ev = O.evaluate(f, I.Flags(), 0, q, qd)
    qdd = np.linalg.solve(ev["M"], tau - ev["c"])
    qdd_kkt = _kkt_qdd(f, q, qd, tau)
    np.testing.assert_allclose(qdd, qdd_kkt, rtol=1e-9, atol=1e-9 * np.abs(qdd_kkt).max())


# ------------------------------------------------------------------------------------------
# Solve: tree LTDL against dense elimination and a library solve
# ------------------------------------------------------------------------------------------
def test_tree_ldlt_matches_dense():
    rng = np.random.default_rng(7)
    for trial in range(5):
        n = 40
        lam = np.array([-1] + [int(rng.integers(0, i)) for i in range(1, n)], np.int32)
        # build H = L^T D L with L unit lower, nonzeros only on ancestor pairs
        Lm = np.eye(n)
        for i in range(n):
            j = lam[i]
            while j >= 0:
                Lm[i, j] = rng.uniform(-1, 1)
                j = lam[j]
        D = rng.uniform(0.5, 2.0, n)
        H = Lm.T @ np.diag(D) @ Lm
        r = rng.standard_normal(n)
        x_tree = O.solve(H, lam, r, 1)
        x_dense = O.solve(H, lam, r, 0)
        x_np = np.linalg.solve(H, r)
        np.testing.assert_allclose(x_tree, x_np, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(x_dense, x_np, rtol=1e-10, atol=1e-12)
    # and on a real H of a generated tree
    f = I.make_forest(I.PLAIN, worlds=[0])
    ev = O.evaluate(f, I.Flags(), 0, np.zeros(f.n_dofs), np.zeros(f.n_dofs))
    H = ev["M"] + np.diag(np.repeat(f.kd[f.parent >= 0], 2) * 2e-3)
    dof_par = []
    chain = {}
    i = 0
    for b in range(f.n_bodies):
        prev = chain.get(int(f.parent[b]), -1)
        for j in range(f.ndof[b]):
            dof_par.append(prev)
            prev = i
            i += 1
        chain[b] = prev
    r = np.random.default_rng(0).standard_normal(f.n_dofs)
    np.testing.assert_allclose(O.solve(H, np.array(dof_par, np.int32), r, 1), np.linalg.solve(H, r), rtol=1e-8)
