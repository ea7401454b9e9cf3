"""Model variants of the generated trees (Sec. III Eq. 2, Sec. IV, Sec. IV-A Eq. 4): each against an
independent statement of what it must produce."""
import math

import numpy as np
import pytest

from paper_2607_06337_b300 import inputs as I


def _children_sums(f, values, power):
    """sum over children of values^power, per body (world 0)."""
    out = np.zeros(f.n_bodies)
    for b in range(1, f.n_bodies):
        out[f.parent[b]] += values[b] ** power
    return out


@pytest.mark.parametrize("beta", [2.0, 2.2, 2.5])
def test_pipe_rule_holds_exactly_for_any_exponent(beta):
    """r_parent^beta = sum_c r_c^beta at every branching body (Eq. 2)."""
    f = I.make_forest(I.BATCH, worlds=[3], variant=I.ModelVariant(pipe_exponent=beta))
    r = 0.5 * f.diam
    s = _children_sums(f, r, beta)
    inner = s > 0
    np.testing.assert_allclose(r[inner] ** beta, s[inner], rtol=1e-12)
    assert abs(f.diam[0] - 0.06) < 1e-15  # the trunk keeps its diameter


def test_larger_exponent_gives_thicker_twigs():
    """With the trunk fixed, a larger beta gives every non-trunk segment a larger diameter
    (d ~ leaves^(1/beta), leaves < leaves(root))."""
    a = I.make_forest(I.BATCH, worlds=[3])
    b = I.make_forest(I.BATCH, worlds=[3], variant=I.ModelVariant(pipe_exponent=2.5))
    sub = a.diam < 0.06
    assert np.all(b.diam[sub] > a.diam[sub])


def test_capsule_inertia_against_quadrature():
    """Mass and inertia of the capsule link against a direct integration over the solid:
    slices along z of a cylinder of length l with a hemisphere on each end."""
    d, l, rho = 0.03, 0.25, 700.0
    m, Ixx, Izz = I.capsule(d, l, rho)
    r = d / 2
    z = np.linspace(-l / 2 - r, l / 2 + r, 400001)
    rad = np.where(np.abs(z) <= l / 2, r, np.sqrt(np.maximum(r * r - (np.abs(z) - l / 2) ** 2, 0.0)))
    dm = rho * math.pi * rad ** 2                       # mass per unit length
    m_q = np.trapezoid(dm, z)
    Izz_q = np.trapezoid(dm * rad ** 2 / 2, z)          # discs about their own axis
    Ixx_q = np.trapezoid(dm * (rad ** 2 / 4 + z ** 2), z)  # discs about a diameter, shifted by z
    np.testing.assert_allclose([m, Ixx, Izz], [m_q, Ixx_q, Izz_q], rtol=1e-8)


def test_capsule_links_in_a_generated_tree():
    a = I.make_forest(I.DIFF, worlds=[0])
    b = I.make_forest(I.DIFF, worlds=[0], variant=I.ModelVariant(capsule=True))
    r = 0.5 * a.diam
    np.testing.assert_allclose(b.mass - a.mass, 700.0 * 4.0 / 3.0 * math.pi * r ** 3, rtol=1e-12)
    assert np.all(b.inertia[:, 0] > a.inertia[:, 0]) and np.all(b.inertia[:, 2] > a.inertia[:, 2])


def test_damping_law_cd():
    """Kd = c_d Kp (Eq. 4) for every compliant joint."""
    f = I.make_forest(I.DIFF, worlds=[0], variant=I.ModelVariant(damping_cd=0.1))
    nz = f.ndof > 0
    np.testing.assert_allclose(f.kd[nz], 0.1 * f.k[nz], rtol=1e-15)


def test_per_level_exponential_stiffness():
    """k = k_0 gamma^(depth - 1): a child's joint is gamma times as stiff as its parent's."""
    f = I.make_forest(I.BATCH, worlds=[1], variant=I.ModelVariant(level_k0=2000.0, level_gamma=0.3))
    for b in range(1, f.n_bodies):
        p = f.parent[b]
        if p > 0:
            assert abs(f.k[b] / f.k[p] - 0.3) < 1e-12
        else:
            assert abs(f.k[b] - 2000.0) < 1e-9
