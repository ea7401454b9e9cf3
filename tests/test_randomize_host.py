"""Pins of inputs.randomize, the host counterpart of the on-device domain-randomisation build
(Sec. IV-D and VII-A: per-world geometric and material transforms of a fixed tree graph), CPU only.

The device build is checked against this function on the GPU, so a mistake shared by the two
would pass there; these tests tie it to what the transforms must do: unit factors give back the
generated trees (with the paper's damping law kd = c_d k, Eq. 4), and each factor scales the
derived quantities by the power its definition fixes (solid cylinder m = rho pi d^2 l / 4,
k = E pi r^4 / (4 l) (Eq. 4), M_max = sigma_r pi r^3 / 4 (Eq. 5)), while every body-frame
point moves with the length factor and the rest pose scales as a whole.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2607_06337_b300 import inputs as I

POINTS = ("jpos", "com")
APPLE_POINTS = ("hang_local", "attach_local")
KEPT = ("parent", "ndof", "qrel", "armature", "apple_body", "apple_mass", "k_s", "c_s", "f_detach", "tip_body",
        "body_off", "apple_off", "tip_off")


@pytest.fixture(scope="module")
def forest():
    return I.make_forest(I.BATCH, worlds=[3, 17, 40])


def _factors(f, **kw):
    fac = np.ones((f.n_worlds, 6))
    fac[:, 5] = kw.pop("c_d", 0.1)
    for i, name in enumerate(I.DR_FACTORS[:5]):
        if name in kw:
            fac[:, i] = kw[name]
    return fac


@pytest.mark.parametrize("capsule", [False, True])
def test_unit_factors_give_back_the_generated_trees(capsule):
    var = I.ModelVariant(capsule=capsule)
    f = I.make_forest(I.BATCH, worlds=[3, 17], variant=var)
    c_d = np.array([0.07, 0.12])
    fac = np.ones((2, 6))
    fac[:, 5] = c_d
    g = I.randomize(f, fac, capsule_links=capsule)
    for name in ("length", "diam", "mass", "inertia", "k", "m_max", "jpos", "com", "hang_local", "attach_local",
                 "tip_local") + KEPT:
        np.testing.assert_array_equal(getattr(g, name), getattr(f, name), err_msg=name)
    wid = np.repeat(np.arange(2), np.diff(f.body_off))
    np.testing.assert_array_equal(g.kd, c_d[wid] * f.k)
    assert (g.kd[f.ndof == 0] == 0).all()


def test_length_factor(forest):
    """s_len = 2: every body-frame point doubles, m and I_zz double, I_xx is the cylinder of the
    doubled length, k halves, the rupture moment is unchanged; at q = 0 every joint origin,
    centre of mass and tip of the rest pose is twice as far from the root."""
    f = forest
    g = I.randomize(f, _factors(f, len=2.0))
    for name in POINTS:
        np.testing.assert_array_equal(getattr(g, name), 2 * getattr(f, name), err_msg=name)
    for name in APPLE_POINTS:
        np.testing.assert_array_equal(getattr(g, name), 2 * getattr(f, name), err_msg=name)
    np.testing.assert_array_equal(g.tip_local, 2 * f.tip_local)
    np.testing.assert_array_equal(g.length, 2 * f.length)
    np.testing.assert_allclose(g.mass, 2 * f.mass, rtol=1e-15)
    np.testing.assert_allclose(g.inertia[:, 2], 2 * f.inertia[:, 2], rtol=1e-15)
    r, l = f.diam / 2, 2 * f.length
    np.testing.assert_allclose(g.inertia[:, 0], g.mass * (3 * r * r + l * l) / 12, rtol=1e-14)
    np.testing.assert_allclose(g.inertia[:, 1], g.inertia[:, 0], rtol=0)
    nd = f.ndof > 0
    np.testing.assert_allclose(g.k[nd], f.k[nd] / 2, rtol=1e-15)
    np.testing.assert_array_equal(g.m_max, f.m_max)
    for name in KEPT:
        np.testing.assert_array_equal(getattr(g, name), getattr(f, name), err_msg=name)
    fl = I.Flags()
    for w in range(f.n_worlds):
        nv = int(f.dof_off[w + 1] - f.dof_off[w])
        a = O.evaluate(f, fl, w, np.zeros(nv), np.zeros(nv))
        b = O.evaluate(g, fl, w, np.zeros(nv), np.zeros(nv))
        np.testing.assert_allclose(b["x"], 2 * a["x"], rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(b["com"], 2 * a["com"], rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(b["R"], a["R"], rtol=0, atol=1e-15)


def test_diameter_factor(forest):
    """s_diam = 2: m x4, I_zz x16, k x16 (r^4), M_max x8 (r^3), lengths and points unchanged."""
    f = forest
    g = I.randomize(f, _factors(f, diam=2.0))
    np.testing.assert_allclose(g.mass, 4 * f.mass, rtol=1e-15)
    np.testing.assert_allclose(g.inertia[:, 2], 16 * f.inertia[:, 2], rtol=1e-15)
    nd = f.ndof > 0
    np.testing.assert_allclose(g.k[nd], 16 * f.k[nd], rtol=1e-15)
    np.testing.assert_allclose(g.m_max, 8 * f.m_max, rtol=1e-15)
    r, l = f.diam, f.length
    np.testing.assert_allclose(g.inertia[:, 0], g.mass * (3 * r * r + l * l) / 12, rtol=1e-14)
    for name in POINTS + APPLE_POINTS + ("tip_local", "length"):
        np.testing.assert_array_equal(getattr(g, name), getattr(f, name), err_msg=name)


def test_material_factors(forest):
    """s_rho scales mass and inertia only; s_E scales k only; s_sigma scales M_max only; c_d
    sets kd = c_d k."""
    f = forest
    g = I.randomize(f, _factors(f, rho=1.5, E=0.75, sigma=1.25, c_d=0.2))
    np.testing.assert_allclose(g.mass, 1.5 * f.mass, rtol=1e-15)
    np.testing.assert_allclose(g.inertia, 1.5 * f.inertia, rtol=1e-15)
    nd = f.ndof > 0
    np.testing.assert_allclose(g.k[nd], 0.75 * f.k[nd], rtol=1e-15)
    np.testing.assert_allclose(g.m_max, 1.25 * f.m_max, rtol=1e-15)
    np.testing.assert_allclose(g.kd, 0.2 * g.k, rtol=0)


def test_each_world_takes_its_own_factors(forest):
    """Per-world factors: world w's records follow its own row only."""
    f = forest
    fac = _factors(f)
    fac[:, 0] = (1.0, 2.0, 0.5)
    g = I.randomize(f, fac)
    for w in range(f.n_worlds):
        b = slice(f.body_off[w], f.body_off[w + 1])
        a = slice(f.apple_off[w], f.apple_off[w + 1])
        t = slice(f.tip_off[w], f.tip_off[w + 1])
        s = fac[w, 0]
        np.testing.assert_array_equal(g.length[b], s * f.length[b])
        np.testing.assert_array_equal(g.jpos[b], s * f.jpos[b])
        np.testing.assert_array_equal(g.hang_local[a], s * f.hang_local[a])
        np.testing.assert_array_equal(g.tip_local[t], s * f.tip_local[t])


def test_geometric_similarity_scales_the_rest_sag():
    """Lengths and diameters both x s (E, rho, sigma_r kept): a similar tree. Under gravity the
    load moment on a joint grows as m g l ~ s^4 and its stiffness as r^4 / l ~ s^3, so the
    static sag angles grow as s, exactly so in the linear regime (weak gravity here; apples
    removed: their stems are not scaled)."""
    f = I.make_forest(I.PLAIN, worlds=[2])
    f.apple_off = np.zeros_like(f.apple_off)
    for name in ("apple_body", "hang_local", "attach_local", "apple_mass", "k_s", "c_s", "f_detach", "apple_x0",
                 "apple_v0", "pull_force", "pull_start", "pull_end"):
        setattr(f, name, getattr(f, name)[:0].copy())
    f.gravity = f.gravity * 1e-3
    fl = I.Flags(dt=0.01)
    s = 1.3
    g = I.randomize(f, np.array([[s, s, 1.0, 1.0, 1.0, 0.3]]))
    f.kd = 0.3 * f.k
    sa, _ = O.rollout(f, fl, 3000, n_threads=1)
    sb, _ = O.rollout(g, fl, 3000, n_threads=1)
    assert np.abs(sa.qd).max() < 1e-12 and np.abs(sb.qd).max() < 1e-12
    big = np.abs(sa.q) > 0.1 * np.abs(sa.q).max()
    np.testing.assert_allclose(sb.q[big], s * sa.q[big], rtol=1e-3)
