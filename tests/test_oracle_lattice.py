"""Pins of the oracle's lattice Boltzmann update (Section 2.1-2.2, Eq. 1-7).

Each test checks the oracle against something the paper or the mathematics fixes:
the paper's printed lattice constants, moment identities of the D2Q9 equilibrium,
closed-form steady states of the lattice, conservation laws and the viscosity law.
"""
import json
import os

import numpy as np
import pytest

import oracle as o

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
E = np.array(GOLD["d2q9_velocities"]["value"], dtype=float)
Wt = np.array(GOLD["d2q9_weights"]["value"])


def test_rest_equilibrium_is_the_printed_weights():
    # Eq. 2 at rho = 1, u = 0 is w_i (weights printed after Eq. 3)
    np.testing.assert_allclose(o.feq(1.0, 0.0, 0.0), Wt, rtol=0, atol=1e-16)


@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.03, -0.02), (0.97, -0.05, 0.01), (1.2, 0.0, 0.08)])
def test_equilibrium_moments(rho, ux, uy):
    # With the printed velocities (Eq. 3): sum feq = rho, sum feq e = rho u,
    # sum feq e e = rho u u + rho c_s^2 I (second-order Hermite equilibrium).
    f = o.feq(rho, ux, uy)
    u = np.array([ux, uy])
    assert abs(f.sum() - rho) < 1e-15
    np.testing.assert_allclose(E.T @ f, rho * u, atol=1e-16)
    P = np.einsum("i,ia,ib->ab", f, E, E)
    np.testing.assert_allclose(P, rho * np.outer(u, u) + rho / 3.0 * np.eye(2), atol=1e-15)


def _random_state(L, seed, amp=0.02):
    rng = np.random.default_rng(seed)
    rho = 1.0 + amp * rng.standard_normal((L.ny, L.nx))
    ux = amp * rng.standard_normal((L.ny, L.nx))
    uy = amp * rng.standard_normal((L.ny, L.nx))
    f = o.init_equilibrium(L, rho, ux, uy)
    f += 1e-3 * rng.standard_normal(f.shape) * Wt[:, None, None]
    return f


def test_uniform_state_is_a_fixed_point():
    L = o.lattice(7, 5, 0.73)
    rho = np.full((5, 7), 1.07); ux = np.full((5, 7), 0.04); uy = np.full((5, 7), -0.03)
    f = o.init_equilibrium(L, rho, ux, uy)
    g = f
    for _ in range(20):
        g = o.collide_stream(L, g)
    np.testing.assert_allclose(g, f, atol=1e-15)


def test_streaming_moves_each_population_along_its_velocity():
    # tau = 1 makes the post-collision state the equilibrium; a delta of momentum at
    # one node must travel to x + e_i in population i only.
    L = o.lattice(9, 8, 1.0)
    rng = np.random.default_rng(3)
    f = _random_state(L, 3)
    # collision at tau = 1 replaces f by feq(rho, u) node by node
    rho, ux, uy = o.macros(L, f)
    post = o.init_equilibrium(L, rho, ux, uy)
    out = o.collide_stream(L, f)
    for i in range(9):
        np.testing.assert_allclose(out[i], np.roll(np.roll(post[i], int(E[i, 0]), axis=1),
                                                   int(E[i, 1]), axis=0), atol=1e-16)


@pytest.mark.parametrize("tau", [0.55, 0.8, 1.7])
def test_couette_linear_profile_is_exact_steady_state(tau):
    # Walls at y = -1/2 and H - 1/2 moving at -u_w and +u_w: the linear profile
    # u_x = u_w (2 (y + 1/2)/H - 1) is reproduced exactly for any tau.
    ny, uw = 8, 0.01
    L = o.lattice(3, ny, tau, walls=True, u_bottom=-uw, u_top=uw)
    y = np.arange(ny)[:, None] * np.ones((1, 3))
    uex = uw * (2 * (y + 0.5) / ny - 1)
    f = o.init_equilibrium(L, None, uex, None)
    nu = (tau - 0.5) / 3
    for _ in range(int(40 * ny * ny / nu / 3) + 200):
        f = o.collide_stream(L, f)
    rho, ux, uy = o.macros(L, f)
    assert np.abs(ux - uex).max() < 1e-13
    assert np.abs(uy).max() < 1e-13


@pytest.mark.parametrize("tau", [0.6, 0.7, 0.5 + np.sqrt(3) / 4, 1.2])
def test_poiseuille_closed_form_with_bounce_back_slip(tau):
    # Body-force channel with half-way bounce-back: the steady discrete profile is the
    # parabola plus the known BGK slip, u = g/(2 nu) [(y+1/2)(H-y-1/2) + (16 L - 3)/12],
    # L = (tau - 1/2)^2 (zero slip at L = 3/16), and its second difference is -g/nu.
    ny, g = 12, 1e-6
    nu = (tau - 0.5) / 3
    lam = (tau - 0.5) ** 2
    L = o.lattice(3, ny, tau, walls=True, gx=g)
    y = np.arange(ny)
    ex = g / (2 * nu) * ((y + 0.5) * (ny - y - 0.5) + (16 * lam - 3) / 12)
    # start on the expected profile to reach the steady state quickly
    f = o.init_equilibrium(L, None, np.repeat(ex[:, None], 3, axis=1), None)
    for _ in range(int(30 * ny * ny / nu / 3)):
        f = o.collide_stream(L, f)
    rho, ux, uy = o.macros(L, f)
    prof = ux[:, 0]
    assert np.abs(prof - ex).max() / ex.max() < 1e-9
    d2 = prof[2:] - 2 * prof[1:-1] + prof[:-2]
    np.testing.assert_allclose(d2, -g / nu, rtol=1e-8)


def test_mass_is_conserved_with_moving_walls_and_forcing():
    L = o.lattice(10, 9, 0.66, walls=True, u_bottom=0.03, u_top=-0.02, gx=1e-4, gy=-2e-5)
    f = _random_state(L, 11)
    rng = np.random.default_rng(12)
    fib = 1e-3 * rng.standard_normal((2, L.ny, L.nx))
    m0 = f.sum()
    for _ in range(50):
        f = o.collide_stream(L, f, fib)
    assert abs(f.sum() - m0) < 1e-12 * m0


def test_momentum_changes_by_total_force_in_periodic_box():
    # Guo forcing: sum_i F_i e_i = (1 - 1/2tau) F and the collision moves (1/2tau) F,
    # so the total momentum grows by exactly sum_x (g + f_ib) per step.
    L = o.lattice(8, 6, 0.81, gx=3e-5, gy=-1e-5)
    f = _random_state(L, 5)
    rng = np.random.default_rng(6)
    fib = 1e-3 * rng.standard_normal((2, L.ny, L.nx))
    for _ in range(5):
        p0 = np.einsum("iyx,ia->a", f, E)
        f2 = o.collide_stream(L, f, fib)
        p1 = np.einsum("iyx,ia->a", f2, E)
        total = fib.sum(axis=(1, 2)) + np.array([L.gx, L.gy]) * L.N
        np.testing.assert_allclose(p1 - p0, total, atol=1e-14)
        f = f2


@pytest.mark.parametrize("tau", [0.6, 0.9])
def test_shear_wave_decays_with_the_printed_viscosity(tau):
    # nu = c_s^2 (tau - 1/2) (Section 2.1): a transverse wave u_x = U sin(k y) decays
    # as exp(-nu k^2 t) up to O(k^2) lattice corrections.
    ny = 64
    k = 2 * np.pi / ny
    L = o.lattice(4, ny, tau)
    y = np.arange(ny)[:, None] * np.ones((1, 4))
    U0 = 1e-4
    f = o.init_equilibrium(L, None, U0 * np.sin(k * y), None)
    amps = []
    for _ in range(2):  # decay measured between t = 100 and t = 400 (past the start-up)
        for _ in range(100 if not amps else 300):
            f = o.collide_stream(L, f)
        _, ux, _ = o.macros(L, f)
        amps.append(2.0 / ny * np.sum(ux[:, 0] * np.sin(k * np.arange(ny))))
    nu_meas = -np.log(amps[1] / amps[0]) / (k * k * 300)
    assert abs(nu_meas / ((tau - 0.5) / 3) - 1) < 2e-3


def test_macros_recover_equilibrium_fields_and_half_force():
    L = o.lattice(6, 5, 0.9, gx=2e-4, gy=1e-4)
    rng = np.random.default_rng(1)
    rho = 1 + 0.01 * rng.standard_normal((5, 6))
    ux = 0.02 * rng.standard_normal((5, 6)); uy = 0.02 * rng.standard_normal((5, 6))
    f = o.init_equilibrium(L, rho, ux, uy)
    fib = 1e-3 * rng.standard_normal((2, 5, 6))
    r2, u2, v2 = o.macros(L, f, fib)
    np.testing.assert_allclose(r2, rho, atol=1e-15)
    np.testing.assert_allclose(u2, ux + 0.5 * (L.gx + fib[0]) / rho, atol=1e-15)
    np.testing.assert_allclose(v2, uy + 0.5 * (L.gy + fib[1]) / rho, atol=1e-15)


def test_wall_correction_sign_moves_fluid_with_the_wall():
    # Fluid at rest between a resting bottom wall and a top wall moving at +u: after
    # one step only the top row gains x-momentum, 6 (w_5 + w_6) u = u/3 per node, from
    # the two diagonal populations reflected by the wall.
    nx, ny, u = 5, 4, 0.01
    L = o.lattice(nx, ny, 0.8, walls=True, u_top=u)
    f = o.init_equilibrium(L)
    f2 = o.collide_stream(L, f)
    mom_top = np.einsum("iyx,i->yx", f2, E[:, 0])[ny - 1]
    # e_5 and e_6 leave through the top and return as 7 and 8, corrected by
    # -6 w_i (e_i . u_w): -u/6 on direction 7 (e_x = -1), +u/6 on direction 8 (e_x = +1)
    np.testing.assert_allclose(mom_top, 2 * u / 6, atol=1e-16)
    assert abs(np.einsum("iyx,i->yx", f2, E[:, 0])[: ny - 1].max()) < 1e-16
