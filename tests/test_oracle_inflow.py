"""Pins of the oracle's open channel: Zou-He known-velocity inlet and known-density outlet
(Section 2.1 boundaries, Section 3.2 inlet profile and outlet pressure; reading R26).

The closure is pinned by what it must achieve (the prescribed velocity or density, to
rounding, on any state), by exact states it must leave alone (uniform flow; the exact
BGK Couette state, whose non-equilibrium part is a pure shear), and by the physics of the
pressure-driven channel it builds (column mass flux, parabolic profile, the paper's
pressure drop).
"""
import numpy as np
import pytest

import oracle as o

E = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], float)


def moments(f, gx=0.0, gy=0.0):
    rho = f.sum(0)
    ux = (np.tensordot(E[:, 0], f, 1) + 0.5 * gx) / rho
    uy = (np.tensordot(E[:, 1], f, 1) + 0.5 * gy) / rho
    return rho, ux, uy


def noisy_state(L, seed, amp=0.02):
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.01 * rng.standard_normal((L.ny, L.nx))
    ux = 0.02 * rng.standard_normal((L.ny, L.nx))
    uy = 0.02 * rng.standard_normal((L.ny, L.nx))
    f = o.init_equilibrium(L, rho, ux, uy)
    return f * (1.0 + amp * rng.standard_normal(f.shape))


def paper_profile(ny, u_max):
    """Section 3.2 inlet: u_max (1 - (1 - 2 y/H)^2) with y from the wall, H = ny."""
    y = np.arange(ny) + 0.5
    return -u_max * (np.abs(1.0 - y / (ny / 2.0)) ** 2 - 1.0)


@pytest.mark.parametrize("walls", [True, False])
def test_closure_gives_the_prescribed_velocity_and_density(walls):
    nx, ny = 12, 9
    u_in = 0.03 * np.sin(np.arange(ny) + 1.0)
    gx, gy = 2e-4, -3e-4
    L = o.lattice(nx, ny, 0.8, walls, gx=gx, gy=gy, u_in=u_in, rho_out=1.013)
    f = o.open_boundaries(L, noisy_state(L, 3))
    rho, ux, uy = moments(f, gx, gy)
    np.testing.assert_allclose(ux[:, 0], u_in, rtol=0, atol=1e-15)
    np.testing.assert_allclose(uy[:, 0], 0.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(rho[:, -1], 1.013, rtol=0, atol=1e-15)
    np.testing.assert_allclose(uy[:, -1], 0.0, rtol=0, atol=1e-15)


def test_closure_changes_only_the_entering_populations():
    nx, ny = 10, 7
    L = o.lattice(nx, ny, 0.7, True, u_in=np.full(ny, 0.01))
    f = noisy_state(L, 5)
    g = o.open_boundaries(L, f)
    changed = np.abs(g - f) > 0
    assert not changed[:, :, 1:-1].any()                      # interior columns untouched
    assert set(np.nonzero(changed[:, :, 0].any(1))[0]) <= {1, 5, 8}     # entering at x = 0
    assert set(np.nonzero(changed[:, :, -1].any(1))[0]) <= {3, 6, 7}    # entering at x = nx-1


def test_uniform_flow_is_a_fixed_point():
    nx, ny, U0 = 24, 10, 0.03
    L = o.lattice(nx, ny, 0.8, False, u_in=np.full(ny, U0), rho_out=1.0)
    f = o.init_equilibrium(L, None, np.full((ny, nx), U0), None)
    np.testing.assert_allclose(o.open_boundaries(L, f), f, rtol=0, atol=1e-16)
    g = f
    for _ in range(20):
        g = o.collide_stream(L, g)
    np.testing.assert_allclose(g, f, rtol=0, atol=1e-15)


def test_exact_couette_state_is_a_fixed_point():
    # the steady BGK Couette flow is exact for a linear profile; its non-equilibrium part
    # is a pure shear (e_x e_y), so bouncing back the normal non-equilibrium and sharing
    # the tangential one must leave it unchanged
    nx, ny, tau, U = 6, 8, 1.0, 0.02
    Lp = o.lattice(nx, ny, tau, True, -U, U)
    f = o.init_equilibrium(Lp)
    for _ in range(6000):
        f = o.collide_stream(Lp, f)
    assert np.abs(o.collide_stream(Lp, f) - f).max() < 1e-16
    rho, ux, _ = moments(f)
    y = np.arange(ny) + 0.5
    np.testing.assert_allclose(ux[:, 0], -U + 2 * U * y / ny, atol=1e-14)   # the exact profile
    Lo = o.lattice(nx, ny, tau, True, -U, U, u_in=ux[:, 0].copy(), rho_out=float(rho[0, -1]))
    np.testing.assert_allclose(o.open_boundaries(Lo, f), f, rtol=0, atol=2e-16)
    g = f
    for _ in range(50):
        g = o.collide_stream(Lo, g)
    np.testing.assert_allclose(g, f, rtol=0, atol=1e-15)


def test_fluid_at_rest_stays_at_rest():
    L = o.lattice(16, 8, 0.7, True, u_in=np.zeros(8), rho_out=1.0)
    f = o.init_equilibrium(L)
    g = f
    for _ in range(30):
        g = o.collide_stream(L, g)
    np.testing.assert_allclose(g, f, rtol=0, atol=1e-15)   # rounding of the closure's division


def test_pressure_driven_channel():
    # Section 3.2 set-up: parabolic inlet, constant-density outlet, no body force. From
    # rest the boundaries alone drive the flow to the Poiseuille state: the profile far
    # from both ends is the inlet parabola and the pressure drops linearly by the
    # Poiseuille gradient dp/dx = -8 rho nu u_max / H^2 (the paper's -u_max 2 rho nu 4 /
    # H^2; 1.2 % above it here, the bounce-back walls' slip). A weakly damped
    # checkerboard mode of the impulsive start decays over ~10^5 steps, so the steady
    # mass balance (every column carries the same flux) is checked from a start near the
    # Poiseuille state.
    nx, ny, tau, u_max = 96, 16, 0.8, 0.01
    nu = (tau - 0.5) / 3.0
    dpdx = -8.0 * nu * u_max / ny ** 2
    u_in = paper_profile(ny, u_max)
    L = o.lattice(nx, ny, tau, True, u_in=u_in, rho_out=1.0)
    f = o.init_equilibrium(L)
    for _ in range(12000):
        f = o.collide_stream(L, f)
    rho, ux, uy = moments(f)
    np.testing.assert_allclose(ux[:, nx // 2] / u_max, u_in / u_max, atol=0.02)
    fit = np.polyfit(np.arange(24, 72), rho[ny // 2, 24:72] / 3.0, 1)[0]
    assert fit == pytest.approx(dpdx, rel=0.03)
    flux = (rho * ux).sum(0)
    assert np.ptp(flux) / flux.mean() < 2e-3
    rho0 = 1.0 + 3.0 * dpdx * (np.arange(nx) - (nx - 1))
    f = o.init_equilibrium(L, np.tile(rho0, (ny, 1)), np.tile(u_in[:, None], (1, nx)), None)
    for _ in range(4000):
        f = o.collide_stream(L, f)
    rho, ux, uy = moments(f)
    flux = (rho * ux).sum(0)
    assert np.ptp(flux) / flux.mean() < 1e-5
    np.testing.assert_allclose(rho[:, -1], 1.0, atol=1e-15)
    assert np.abs(uy[:, 24:72]).max() < 1e-5 * u_max


def test_supports_must_stay_off_the_open_columns():
    L = o.lattice(20, 12, 0.8, True, u_in=np.zeros(12))
    assert o.mls(L, 2.2, 6.3)[-1] == 0          # support columns 1..3
    assert o.mls(L, 1.3, 6.3)[-1] == 5          # support column 0: the inlet
    assert o.mls(L, 18.4, 6.3)[-1] == 5         # support column 19: the outlet
    Lp = o.lattice(20, 12, 0.8, True)
    assert o.mls(Lp, 1.3, 6.3)[-1] == 0         # periodic: no restriction


def test_simulation_holds_the_open_columns_from_the_start():
    # the fields read before any step already carry the prescribed inlet velocity and
    # outlet density; a capsule in the channel and both schemes keep them every step
    nx, ny = 48, 20
    u_in = paper_profile(ny, 0.01)
    L = o.lattice(nx, ny, 0.8, True, u_in=u_in, rho_out=1.0)
    for scheme in (o.KINEMATIC, o.DYNAMIC):
        s = o.Sim(L)
        s.init_fields()
        rho, ux, uy = s.read_fields()
        np.testing.assert_allclose(ux[:, 0], u_in, rtol=0, atol=1e-16)
        np.testing.assert_allclose(rho[:, -1], 1.0, rtol=0, atol=1e-16)
        t = 2 * np.pi * (np.arange(24) + 0.137) / 24
        s.add_capsule(np.stack([20.3 + 4 * np.cos(t), 10.07 + 4 * np.sin(t)], 1), 0.01, 0.001, 0.0, 1.0)
        assert s.step(30, scheme) == 0
        rho, ux, uy = s.read_fields()
        np.testing.assert_allclose(ux[:, 0], u_in, rtol=0, atol=1e-15)
        np.testing.assert_allclose(uy[:, 0], 0.0, rtol=0, atol=1e-15)
        np.testing.assert_allclose(rho[:, -1], 1.0, rtol=0, atol=1e-15)
