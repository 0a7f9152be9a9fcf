"""Pins of the oracle's membrane mechanics (Section 2.2.1, Eq. 10-14), observables
(Section 3.1-3.2) and node integrators (Eq. 23-25).
"""
import numpy as np
import pytest

import oracle as o
from paper_1903_03356_gb300 import workloads as W


def _deformed(n=40, seed=0, r=6.0, amp=0.3):
    rng = np.random.default_rng(seed)
    ref = W.circle(n, r, 10.0, 12.0)
    cur = ref + amp * rng.standard_normal(ref.shape) * 0.3
    return ref, cur


@pytest.mark.parametrize("ks,kb,ka", [(0.7, 0, 0), (0, 0.3, 0), (0, 0, 2.0), (0.5, 0.2, 1.0)])
def test_force_is_minus_energy_gradient(ks, kb, ka):
    # F = -dE/dX by central differences (h = 1e-6), E = Eq. 10 + bending (R6) + area
    ref, cur = _deformed()
    L0, th0, A0 = o.membrane_reference(ref)
    F = o.membrane_force(cur, L0, th0, A0, ks, kb, ka).reshape(-1)
    x = cur.reshape(-1).copy()
    h = 1e-6
    G = np.zeros_like(x)
    for m in range(x.size):
        xp = x.copy(); xp[m] += h
        xm = x.copy(); xm[m] -= h
        G[m] = (o.membrane_energy(xp, L0, th0, A0, ks, kb, ka)
                - o.membrane_energy(xm, L0, th0, A0, ks, kb, ka)) / (2 * h)
    assert np.abs(F + G).max() < 1e-7 * np.abs(F).max()


def test_stress_free_shape_has_no_force_under_rigid_motion():
    ref = W.biconcave(64, 8.0, 30.0, 20.0)
    L0, th0, A0 = o.membrane_reference(ref)
    for ang in (0.0, 0.4, 2.5):
        R = np.array([[np.cos(ang), -np.sin(ang)], [np.sin(ang), np.cos(ang)]])
        moved = (ref - ref.mean(0)) @ R.T + np.array([3.7, -1.2]) + ref.mean(0)
        F = o.membrane_force(moved, L0, th0, A0, 0.9, 0.4, 1.0)
        assert np.abs(F).max() < 1e-12


def test_internal_forces_have_zero_sum_and_zero_torque():
    ref, cur = _deformed(seed=3, amp=0.6)
    L0, th0, A0 = o.membrane_reference(ref)
    F = o.membrane_force(cur, L0, th0, A0, 0.8, 0.3, 1.5).reshape(-1, 2)
    np.testing.assert_allclose(F.sum(0), 0.0, atol=1e-13)
    c = cur.reshape(-1, 2)
    torque = np.sum(c[:, 0] * F[:, 1] - c[:, 1] * F[:, 0])
    assert abs(torque) < 1e-12


def test_uniform_stretch_of_regular_polygon_closed_form():
    # Each spring of a regular n-gon scaled by s carries k_s (L - L0); the two springs
    # at a vertex sum to 2 k_s (L - L0) sin(pi/n) pointing to the centre (Eq. 11).
    n, r, s, ks = 24, 5.0, 1.1, 0.6
    ref = W.circle(n, r, 0.0, 0.0)
    L0, th0, A0 = o.membrane_reference(ref)
    F = o.membrane_force(ref * s, L0, th0, A0, ks, 0.0, 0.0).reshape(-1, 2)
    mag = 2 * ks * (L0[0] * s - L0[0]) * np.sin(np.pi / n)
    np.testing.assert_allclose(F, -mag * ref / r, atol=1e-14)


def test_area_penalty_pushes_out_a_compressed_ring():
    # Eq. 14 on a regular n-gon scaled by s < 1: radial outward force of magnitude
    # k_a (1 - s^2) p_ref |dA/dX_v|, with |dA/dX_v| = s r sin(2 pi / n) for the n-gon.
    n, r, s, ka = 30, 4.0, 0.9, 1.0
    ref = W.circle(n, r, 0.0, 0.0)
    L0, th0, A0 = o.membrane_reference(ref)
    F = o.membrane_force(ref * s, L0, th0, A0, 0.0, 0.0, ka).reshape(-1, 2)
    mag = ka * (1 - s * s) / 3.0 * s * r * np.sin(2 * np.pi / n)
    np.testing.assert_allclose(F, mag * ref / r, atol=1e-14)


def test_turning_angles_of_regular_and_general_polygons():
    n = 17
    _, th0, _ = o.membrane_reference(W.circle(n, 3.0, 1.0, 1.0))
    np.testing.assert_allclose(th0, 2 * np.pi / n, atol=1e-14)
    _, th0, _ = o.membrane_reference(W.biconcave(128, 8.0, 0, 0))
    assert abs(th0.sum() - 2 * np.pi) < 1e-12    # turning number of a simple CCW curve


def test_area_and_perimeter_closed_forms():
    sq = np.array([[0, 0], [2, 0], [2, 3], [0, 3]], float)
    assert o.area(sq) == 6.0 and o.perimeter(sq) == 10.0
    assert o.area(sq[::-1].copy()) == -6.0
    n, r = 50, 3.0
    c = W.circle(n, r, 5.0, -2.0)
    assert abs(o.area(c) - 0.5 * n * r * r * np.sin(2 * np.pi / n)) < 1e-12
    assert abs(o.perimeter(c) - 2 * n * r * np.sin(np.pi / n)) < 1e-12


def test_observables_of_a_regular_polygon():
    n, r = 64, 10.0
    ob = o.observables(W.circle(n, r, 50.1, 49.3))
    assert abs(ob[2]) < 1e-12                                   # D = 0
    np.testing.assert_allclose(ob[3:5], [50.1, 49.3], atol=1e-12)
    # swelling ratio of the n-gon: pi cos(pi/n) / (n sin(pi/n))
    assert abs(ob[5] - np.pi * np.cos(np.pi / n) / (n * np.sin(np.pi / n))) < 1e-13


@pytest.mark.parametrize("beta", [0.0, 0.3, -0.7])
def test_taylor_deformation_of_a_rectangle_is_exact(beta):
    # A w x h rectangle has area covariance eigenvalues w^2/12 and h^2/12, so
    # a = w/sqrt 3, b = h/sqrt 3 and D = (w - h)/(w + h), inclined at beta.
    w, h = 6.0, 2.0
    m = 10
    top = [(w / 2 - w * k / m, h / 2) for k in range(m)]
    left = [(-w / 2, h / 2 - h * k / m) for k in range(m)]
    bot = [(-w / 2 + w * k / m, -h / 2) for k in range(m)]
    right = [(w / 2, -h / 2 + h * k / m) for k in range(m)]
    pts = np.array(right + top + left + bot)
    R = np.array([[np.cos(beta), -np.sin(beta)], [np.sin(beta), np.cos(beta)]])
    pts = pts @ R.T + np.array([7.0, -3.0])
    ob = o.observables(pts)
    assert abs(ob[0] - w * h) < 1e-12
    assert abs(ob[2] - (w - h) / (w + h)) < 1e-12
    assert abs(ob[6] - beta) < 1e-12
    assert abs(ob[7] - w * w / 12) < 1e-12


def test_taylor_deformation_of_a_fine_ellipse():
    t = 2 * np.pi * np.arange(20000) / 20000
    a, b = 5.0, 3.0
    ob = o.observables(np.stack([a * np.cos(t) + 2, b * np.sin(t) + 1], 1))
    assert abs(ob[2] - (a - b) / (a + b)) < 1e-7


def test_biconcave_area_and_perimeter_match_curve_quadrature():
    # The polygon's Green's-theorem area and its perimeter converge to the integrals of
    # the Eq. 26 curve evaluated by quadrature of its parametrisation.
    a = 8.0
    t = np.linspace(-0.5 * np.pi, 1.5 * np.pi, 400001)
    s = np.sin(t)
    x = a * s
    y = 0.5 * a * (0.207 + 2.003 * s ** 2 - 1.123 * s ** 4) * np.cos(t)
    dx, dy = np.gradient(x, t), np.gradient(y, t)
    A_curve = abs(np.trapezoid(x * dy - y * dx, t)) * 0.5
    P_curve = np.trapezoid(np.hypot(dx, dy), t)
    ob = o.observables(W.biconcave(4096, a, 0, 0))
    assert abs(ob[0] / A_curve - 1) < 1e-5
    assert abs(ob[1] / P_curve - 1) < 1e-5


def test_kinematic_advance_is_exact_for_quadratic_trajectories():
    # Eq. 25 is the BDF2 formula: exact when x(t) is quadratic and xdot is exact at t+1
    rng = np.random.default_rng(0)
    a, b, c = rng.standard_normal((3, 10))
    x = lambda t: a + b * t + c * t * t
    v = lambda t: b + 2 * c * t
    for n in (1, 5):
        out = o.kinematic_advance(x(n), x(n - 1), v(n + 1), first=False)
        np.testing.assert_allclose(out, x(n + 1), atol=1e-12)
    # first step: forward Euler
    np.testing.assert_allclose(o.kinematic_advance(x(0), x(0), v(0), first=True), x(0) + v(0))


def test_dynamic_advance_closed_forms():
    # Eq. 23: x1 = x0 + v0 + F/(2m); Eq. 24: BDF2 velocity, exact for quadratics
    rng = np.random.default_rng(1)
    a, b, c = rng.standard_normal((3, 8))
    x = lambda t: a + b * t + c * t * t
    m = 2.5
    F = rng.standard_normal(8)
    X1, uv = o.dynamic_advance(x(3), x(2), np.zeros(8), F, m)
    np.testing.assert_allclose(X1, x(3) + F / (2 * m), atol=1e-14)
    # choose the tentative velocity so that X^{n+1} = x(n+1); uv must equal x'(n+1)
    xd0 = x(4) - x(3) - F / (2 * m)
    X1, uv = o.dynamic_advance(x(3), x(2), xd0, F, m)
    np.testing.assert_allclose(X1, x(4), atol=1e-12)
    np.testing.assert_allclose(uv, b + 2 * c * 4, atol=1e-12)
