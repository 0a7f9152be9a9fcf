"""Pins of the oracle's rigid particles (Section 2.3.1, Eq. 17-20; readings R27-R30).

The integrator is pinned by closed-form solutions of its recurrences (constant load from
rest; uniform translation and rotation); the load by the exact pressure force of a
linear density field on a regular polygon and on a rectangle, and its moment by the
change of reference point; the coupled particle by physics: at rest it stays at rest, its
markers stay rigid, and a free disk in simple shear turns at half the shear rate.
"""
import numpy as np
import pytest

import oracle as o


def polygon(n, r, cx, cy, phase=0.137):
    t = 2 * np.pi * (np.arange(n) + phase) / n
    return np.stack([cx + r * np.cos(t), cy + r * np.sin(t)], 1)


def polygon_area_inertia(xy):
    """Area, centroid and polar second moment about the centroid of a polygon."""
    x, y = xy[:, 0], xy[:, 1]
    xn, yn = np.roll(x, -1), np.roll(y, -1)
    cr = x * yn - xn * y
    A = 0.5 * cr.sum()
    cx = ((x + xn) * cr).sum() / (6 * A)
    cy = ((y + yn) * cr).sum() / (6 * A)
    Jxx = ((x * x + x * xn + xn * xn) * cr).sum() / 12.0
    Jyy = ((y * y + y * yn + yn * yn) * cr).sum() / 12.0
    J = Jxx + Jyy - A * (cx * cx + cy * cy)
    return A, cx, cy, J


def test_constant_load_from_rest_follows_the_closed_form():
    # Eq. 19 with constant acceleration a from rest (u^0 = u^-1 = 0) has the solution
    # u^n = a n - a/2 + (a/2) 3^-n (roots 1 and 1/3 of the recurrence); the backward
    # position update then gives c^n - c^0 = (a/2) n^2 - (a/2) n + (3a/4)(1 - 3^-n)
    # - (a/6) n 3^-n. Eq. 20 and the angle likewise.
    m, I = 7.0, 90.0
    load = np.array([0.014, -0.021, 0.45])
    a = np.array([load[0] / m, load[1] / m, load[2] / I])
    body = np.array([3.0, 4.0, 0.25, 0.0, 0.0, 0.0])
    prev = body.copy()
    c0 = body[:3].copy()
    for n in range(1, 41):
        body, prev = o.rigid_advance(body, prev, load, m, I)
        u = a * n - a / 2 + (a / 2) * 3.0 ** -n
        c = c0 + (a / 2) * n * n - (a / 2) * n + (3 * a / 4) * (1 - 3.0 ** -n) - (a / 6) * n * 3.0 ** -n
        np.testing.assert_allclose(body[3:], u, rtol=1e-13, atol=1e-16)
        np.testing.assert_allclose(body[:3], c, rtol=1e-13, atol=1e-14)


def test_uniform_translation_and_rotation_are_exact():
    U = np.array([0.013, -0.007, 0.002])
    body = np.array([10.0, 5.0, 0.3, *U])
    prev = np.array([10.0 - U[0], 5.0 - U[1], 0.3 - U[2], *U])
    start = body.copy()
    for n in range(1, 21):
        body, prev = o.rigid_advance(body, prev, np.zeros(3), 2.0, 3.0)
        np.testing.assert_allclose(body[:3], start[:3] + n * U, rtol=0, atol=1e-13)
        np.testing.assert_allclose(body[3:], U, rtol=0, atol=1e-17)


def linear_density(L, G):
    y, x = np.mgrid[0:L.ny, 0:L.nx].astype(float)
    return o.init_equilibrium(L, 1.0 + G[0] * (x - L.nx / 2) + G[1] * (y - L.ny / 2), None, None)


@pytest.mark.parametrize("n,phase", [(24, 0.137), (57, 0.41)])
def test_pressure_load_of_a_linear_density_on_a_regular_polygon(n, phase):
    # fluid at rest, p = rho/3 linear: the MLS reproduces it exactly and tau = 0, so
    # F = -1/3 sum_l (p0 + G.(c_l + 1.2 n_l)) n_l l_l = -(G/3)(A + 1.2 P/2) for a regular
    # polygon (sum c_l n_l^T l_l = A I, sum n_l n_l^T l_l = P/2 I), M = 0 about its centre
    L = o.lattice(80, 80, 0.8, False)
    G = np.array([2e-4, -1.3e-4])
    f = linear_density(L, G)
    xy = polygon(n, 9.0, 40.2, 39.9, phase)
    A, cx, cy, _ = polygon_area_inertia(xy)
    P = np.linalg.norm(np.roll(xy, -1, 0) - xy, axis=1).sum()
    load, st = o.rigid_load(L, f, None, xy, cx, cy)
    assert st == 0
    np.testing.assert_allclose(load[:2], -(G / 3.0) * (A + 0.6 * P), rtol=1e-11)
    assert abs(load[2]) < 1e-14
    # moment about another point: M' = M - (d x F)
    d = np.array([1.7, -2.2])
    load2, _ = o.rigid_load(L, f, None, xy, cx + d[0], cy + d[1])
    np.testing.assert_allclose(load2[:2], load[:2], rtol=1e-15)
    assert load2[2] == pytest.approx(load[2] - (d[0] * load[1] - d[1] * load[0]), abs=1e-14)


def test_pressure_load_of_a_linear_density_on_a_rectangle():
    # sum_l n_l n_l^T l_l = diag(2h, 2w) for a w x h rectangle, so
    # F = -1/3 (A G + 1.2 (2h G_x, 2w G_y))
    L = o.lattice(80, 80, 0.8, False)
    G = np.array([1.5e-4, 2.5e-4])
    f = linear_density(L, G)
    w, h = 14.0, 6.0
    x0, y0 = 33.07, 37.13
    edges = []
    for (ax, ay), (bx, by) in (((x0, y0), (x0 + w, y0)), ((x0 + w, y0), (x0 + w, y0 + h)),
                               ((x0 + w, y0 + h), (x0, y0 + h)), ((x0, y0 + h), (x0, y0))):
        for t in np.arange(7) / 7.0:
            edges.append((ax + t * (bx - ax), ay + t * (by - ay)))
    xy = np.array(edges)
    load, st = o.rigid_load(L, f, None, xy, x0 + w / 2, y0 + h / 2)
    assert st == 0
    expect = -(1.0 / 3.0) * (w * h * G + 1.2 * np.array([2 * h * G[0], 2 * w * G[1]]))
    np.testing.assert_allclose(load[:2], expect, rtol=1e-11)
    assert abs(load[2]) < 1e-13


def free_disk(L, n=40, r=5.0, cx=32.3, cy=20.07, rho_s=1.0):
    xy = polygon(n, r, cx, cy)
    A, _, _, J = polygon_area_inertia(xy)
    return xy, rho_s * A, rho_s * J


def test_disk_at_rest_stays_at_rest_and_rigid():
    L = o.lattice(64, 40, 0.8, True)
    s = o.Sim(L)
    s.init_fields()
    xy, m, I = free_disk(L)
    k = s.add_rigid(xy, m, I)
    assert s.step(60, o.DYNAMIC) == 0
    b = s.read_rigid(k)
    assert np.abs(b[3:6]).max() < 1e-14
    np.testing.assert_allclose(s.read_capsule(k)[0].reshape(-1, 2), xy, atol=1e-12)


def test_free_disk_in_simple_shear_turns_at_half_the_shear_rate():
    # a neutrally buoyant disk at the centre of a Couette flow turns with the fluid's
    # local rotation rate, omega = -gamma/2 (radius 5, H = 48: about 2 % slower from the
    # confinement), and stays in place; its markers stay rigid
    ny, U = 48, 0.01
    gamma = 2 * U / ny
    L = o.lattice(72, ny, 0.8, True, -U, U)
    s = o.Sim(L)
    y = np.arange(ny) + 0.5
    ux = np.tile((-U + gamma * y)[:, None], (1, 72))
    s.init_fields(None, ux, None)
    xy, m, I = free_disk(L, n=48, r=5.0, cx=36.2, cy=ny / 2 - 0.43)
    k = s.add_rigid(xy, m, I)
    assert s.step(1500, o.DYNAMIC) == 0
    b = s.read_rigid(k)
    print(f"omega / (-gamma/2) = {b[5] / (-gamma / 2):.4f}, u = {b[3]:.2e} {b[4]:.2e}")
    assert b[5] / (-gamma / 2) == pytest.approx(1.0, abs=0.05)
    assert abs(b[3]) < 0.05 * U and abs(b[4]) < 0.05 * U
    X = s.read_capsule(k)[0].reshape(-1, 2)
    d0 = np.linalg.norm(xy[:, None] - xy[None], axis=2)
    d1 = np.linalg.norm(X[:, None] - X[None], axis=2)
    np.testing.assert_allclose(d1, d0, atol=1e-11)
    assert abs(b[2]) > 1e-3          # it has turned


def test_kinematic_scheme_refuses_rigid_particles():
    L = o.lattice(40, 30, 0.8, True)
    s = o.Sim(L)
    s.init_fields()
    xy, m, I = free_disk(L, cx=20.3, cy=15.07)
    s.add_rigid(xy, m, I)
    assert s.step(1, o.KINEMATIC) == 7
    assert s.step_count == 0
