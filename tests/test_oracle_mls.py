"""Pins of the oracle's moving-least-squares transfer (Section 2.2, Eq. 8-9, step 3).

The shape functions are checked against a brute-force minimisation of Eq. 9, exact
reproduction of constant and linear fields, the closed form of the symmetric case with
the printed r_w and alpha, the support geometry of Fig. 1a, and the adjointness of
interpolation and spreading.
"""
import json
import os

import numpy as np
import pytest

import oracle as o
from paper_1903_03356_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
RW = GOLD["mls_support_side_rw"]["value"]
ALPHA = GOLD["mls_alpha"]["value"]


def _points(n, seed, L, margin=2.0):
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(margin, L.nx - 1 - margin, n),
                     rng.uniform(margin, L.ny - 1 - margin, n)], axis=1)


def test_shape_functions_minimise_eq9_brute_force():
    # Eq. 9: phi_k are the weights of the value of the weighted least-squares linear fit
    # at the marker. Solve that fit with numpy's lstsq on sqrt(W)-scaled rows for
    # unit data vectors and compare.
    L = o.lattice(20, 20, 0.8)
    for X, Y in _points(25, 1, L):
        ix, iy, phi, gx, gy, st = o.mls(L, X, Y)
        assert st == 0
        cx, cy = np.floor(X + 0.5), np.floor(Y + 0.5)
        xs = np.array([cx + a for b in (-1, 0, 1) for a in (-1, 0, 1)])
        ys = np.array([cy + b for b in (-1, 0, 1) for a in (-1, 0, 1)])
        r = np.hypot(xs - X, ys - Y) / RW
        w = np.exp(-(r / ALPHA) ** 2)
        P = np.stack([np.ones(9), xs, ys], axis=1)        # paper's basis [1, x, y]
        sw = np.sqrt(w)
        coef = np.linalg.lstsq(P * sw[:, None], np.diag(sw), rcond=None)[0]  # 3 x 9
        np.testing.assert_allclose(phi, np.array([1.0, X, Y]) @ coef, atol=1e-12)
        np.testing.assert_allclose(gx, coef[1], atol=1e-11)
        np.testing.assert_allclose(gy, coef[2], atol=1e-11)


def test_reproduces_constant_and_linear_fields():
    L = o.lattice(30, 24, 0.8)
    xx, yy = np.meshgrid(np.arange(L.nx), np.arange(L.ny))
    for X, Y in _points(40, 2, L):
        ix, iy, phi, gx, gy, st = o.mls(L, X, Y)
        assert abs(phi.sum() - 1) < 1e-14
        xk, yk = xx[iy, ix], yy[iy, ix]
        assert abs(phi @ xk - X) < 1e-13 and abs(phi @ yk - Y) < 1e-13
        assert abs(gx.sum()) < 1e-14 and abs(gy.sum()) < 1e-14
        assert abs(gx @ xk - 1) < 1e-13 and abs(gx @ yk) < 1e-13
        assert abs(gy @ yk - 1) < 1e-13 and abs(gy @ xk) < 1e-13
        v = 0.3 - 0.7 * xx + 1.9 * yy
        val, _ = o.interp_scalar(L, v, X, Y)
        assert abs(val - (0.3 - 0.7 * X + 1.9 * Y)) < 1e-12


def test_symmetric_marker_on_a_node_has_closed_form_weights():
    # Marker on a lattice node: by symmetry the linear coefficients do not couple,
    # so phi_k = W_k / sum W with W = exp(-(d/(r_w alpha))^2), d in {0, 1, sqrt 2}.
    L = o.lattice(10, 10, 0.8)
    ix, iy, phi, gx, gy, st = o.mls(L, 4.0, 5.0)
    w1 = np.exp(-(1 / (RW * ALPHA)) ** 2)
    w2 = np.exp(-(np.sqrt(2) / (RW * ALPHA)) ** 2)
    S = 1 + 4 * w1 + 4 * w2
    expect = np.array([w2, w1, w2, w1, 1.0, w1, w2, w1, w2]) / S
    np.testing.assert_allclose(phi, expect, atol=1e-15)
    # diffuse derivative: gx_k = W_k (x_k - X) / sum W_k (x_k - X)^2
    dx = np.array([-1, 0, 1] * 3, float)
    wk = np.array([w2, w1, w2, w1, 1.0, w1, w2, w1, w2])
    np.testing.assert_allclose(gx, wk * dx / np.sum(wk * dx * dx), atol=1e-15)


def test_support_is_centred_on_the_nearest_node_with_periodic_x():
    L = o.lattice(12, 10, 0.8)
    ix, iy, *_ = o.mls(L, 3.49, 4.51)
    assert sorted(set(ix.tolist())) == [2, 3, 4] and sorted(set(iy.tolist())) == [4, 5, 6]
    ix, iy, *_ = o.mls(L, 11.7, 5.2)       # centre 12 wraps to 0
    assert sorted(set(ix.tolist())) == [0, 1, 11]
    ix, iy, *_ = o.mls(L, -0.7, 5.2)       # unwrapped negative position
    assert sorted(set(ix.tolist())) == [0, 10, 11]


def test_support_outside_the_walls_is_reported():
    L = o.lattice(12, 10, 0.8, walls=True)
    assert o.mls(L, 5.3, 1.2)[-1] == 0
    assert o.mls(L, 5.3, 0.4)[-1] == 5
    assert o.mls(L, 5.3, 8.6)[-1] == 5
    Lp = o.lattice(12, 10, 0.8, walls=False)
    assert o.mls(Lp, 5.3, 0.4)[-1] == 0


def test_interpolation_and_spreading_are_adjoint():
    # <spread(F), v>_grid = <F, c I(v)>_markers for arbitrary F and v.
    L = o.lattice(16, 14, 0.8)
    rng = np.random.default_rng(7)
    pts = _points(30, 8, L, margin=0.0)
    F = rng.standard_normal((30, 2))
    c = rng.uniform(0.2, 1.5, 30)
    v = rng.standard_normal((2, L.ny, L.nx))
    fib = np.zeros((2, L.ny, L.nx))
    for (X, Y), (Fx, Fy), ck in zip(pts, F, c):
        o.spread(L, X, Y, Fx, Fy, ck, fib)
    lhs = np.sum(fib * v)
    rhs = 0.0
    for (X, Y), (Fx, Fy), ck in zip(pts, F, c):
        vx, _ = o.interp_scalar(L, v[0], X, Y)
        vy, _ = o.interp_scalar(L, v[1], X, Y)
        rhs += ck * (Fx * vx + Fy * vy)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_spreading_conserves_total_force():
    # step 3: c_l chosen so that the total force on the fluid is conserved; sum phi = 1
    L = o.lattice(16, 14, 0.8)
    fib = np.zeros((2, L.ny, L.nx))
    o.spread(L, 7.3, 6.8, 0.5, -0.25, 0.7, fib)
    np.testing.assert_allclose(fib.sum(axis=(1, 2)), [0.35, -0.175], atol=1e-15)


def test_interp_uses_eq7_velocity_and_pressure():
    # uniform state with force: U = (sum f e + F/2)/rho everywhere, p = rho/3, grad 0
    L = o.lattice(10, 9, 0.8, gx=1e-4)
    rho = np.full((9, 10), 1.05); ux = np.full((9, 10), 0.02); uy = np.full((9, 10), -0.01)
    f = o.init_equilibrium(L, rho, ux, uy)
    fib = np.zeros((2, 9, 10)); fib[1] = 2e-4
    out, st = o.interp(L, f, fib, 4.3, 4.7)
    np.testing.assert_allclose(out[:4], [0.02 + 0.5e-4 / 1.05, -0.01 + 1e-4 / 1.05, 1.05, 0.35],
                               atol=1e-15)
    np.testing.assert_allclose(out[4:], 0.0, atol=1e-15)


def test_velocity_gradient_of_a_linear_flow_is_exact():
    L = o.lattice(20, 20, 0.8)
    yy, xx = np.mgrid[0:20, 0:20].astype(float)
    ux = 0.001 * (xx - 10) + 0.002 * (yy - 10)
    uy = -0.0015 * (xx - 10) + 0.0005 * (yy - 10)
    f = o.init_equilibrium(L, None, ux, uy)
    for X, Y in _points(10, 3, L, margin=3):
        out, _ = o.interp(L, f, None, X, Y)
        np.testing.assert_allclose(out[4:], [0.001, 0.002, -0.0015, 0.0005], atol=1e-14)


def _ring_normals(xy):
    d = np.roll(xy, -1, axis=0) - xy
    ln = np.hypot(d[:, 0], d[:, 1])
    return np.stack([d[:, 1], -d[:, 0]], 1) / ln[:, None], ln


def test_pressure_traction_of_a_linear_density_field_closed_form():
    # rho = 1 + a x at rest: p = rho/3 is linear, so the MLS probes are exact and
    # Eq. 15 gives F_l = -(a/3)(2 * 1.2 n_x) n l on every element, grad u = 0 (Eq. 16).
    L = o.lattice(40, 40, 0.8)
    a = 1e-3
    yy, xx = np.mgrid[0:40, 0:40].astype(float)
    f = o.init_equilibrium(L, 1 + a * xx, None, None)
    xy = W.circle(30, 8.0, 20.2, 19.9)
    Fext, st = o.tractions(L, f, None, xy)
    assert st == 0
    n, ln = _ring_normals(xy)
    Fl = -(a / 3) * (2 * 1.2 * n[:, [0]]) * n * ln[:, None]
    expect = 0.5 * (Fl + np.roll(Fl, 1, axis=0))
    np.testing.assert_allclose(Fext, expect, atol=1e-15)


def test_tractions_vanish_in_a_linear_flow_at_uniform_density():
    # uniform rho and a linear u: p+ = p- and tau+ = tau- on every element
    L = o.lattice(40, 40, 0.8)
    yy, xx = np.mgrid[0:40, 0:40].astype(float)
    f = o.init_equilibrium(L, None, 1e-3 * (yy - 20) + 2e-4 * (xx - 20), -5e-4 * (xx - 20))
    Fext, st = o.tractions(L, f, None, W.circle(30, 8.0, 20.2, 19.9))
    assert np.abs(Fext).max() < 1e-13      # a sign slip would give ~1e-4
