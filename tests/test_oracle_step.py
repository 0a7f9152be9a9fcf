"""Pins of the oracle's coupled LBM-IB step: the Kinematic scheme (Section 2.4, steps
i-viii) and the Dynamic scheme (Section 2.3.2, steps 1-8).

Invariants that hold at any size: Galilean translation of a stress-free capsule in a
uniform flow, conservation of mass, momentum balance against the spread force, the
start-up rules, and the support check near walls.
"""
import numpy as np
import pytest

import oracle as o
from paper_1903_03356_gb300 import workloads as W

E = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], float)


def _sim(L, caps):
    s = o.Sim(L)
    for xy, ks, kb, ka, m in caps:
        s.add_capsule(xy, ks, kb, ka, m)
    return s


@pytest.mark.parametrize("scheme", [o.KINEMATIC, o.DYNAMIC])
def test_stress_free_capsule_translates_with_uniform_flow(scheme):
    # MLS reproduces constants, so U = U0 at every node; internal forces vanish; the
    # Dynamic forcing u_v - U vanishes; Eq. 23-25 then move every node by U0 per step.
    L = o.lattice(40, 36, 0.8)
    U0 = np.array([0.011, -0.004])
    ref = W.circle(32, 6.0, 20.13, 18.07)
    s = _sim(L, [(ref, 0.5, 0.1, 1.0, 2.0)])
    s.init_fields(None, np.full((36, 40), U0[0]), np.full((36, 40), U0[1]))
    f0 = s.populations()
    s.step(25, scheme)
    xy, vel, fint, fext = s.read_capsule(0)
    np.testing.assert_allclose(xy.reshape(-1, 2), ref + 25 * U0, atol=1e-12)
    np.testing.assert_allclose(vel.reshape(-1, 2), np.broadcast_to(U0, ref.shape), atol=1e-13)
    np.testing.assert_allclose(s.populations(), f0, atol=1e-15)
    assert np.abs(s.force_field()).max() < 1e-13   # zero up to round-off of X


def _deformed(ref, centre, sx=1.12, sy=0.9):
    return (ref - centre) * np.array([sx, sy]) + centre


def test_kinematic_conserves_mass_and_momentum_in_a_periodic_box():
    # sum f_ib = sum F^int = 0 (pairwise stretch, torque-free bending, closed ring), so
    # the fluid momentum stays exactly at its initial value while the ring relaxes.
    L = o.lattice(48, 40, 0.75)
    centre = np.array([24.1, 20.03])
    ref = W.circle(40, 7.0, *centre)
    s = _sim(L, [(ref, 0.05, 0.01, 0.5, 3.0)])
    s.set_positions(0, _deformed(ref, centre))
    f = s.populations()
    m0, p0 = f.sum(), np.einsum("iyx,ia->a", f, E)
    for _ in range(10):
        s.step(10, o.KINEMATIC)
        f = s.populations()
        assert abs(f.sum() - m0) < 1e-13 * m0
        # round-off of a sum over 9 N populations is ~1e-16 * 9 N * max f
        np.testing.assert_allclose(np.einsum("iyx,ia->a", f, E), p0, atol=2e-12)
    # and the ring did move: the relaxation is real
    assert np.abs(s.read_capsule(0)[0].reshape(-1, 2) - _deformed(ref, centre)).max() > 1e-4


def test_kinematic_spread_field_is_the_spread_internal_force():
    L = o.lattice(48, 40, 0.75)
    centre = np.array([24.1, 20.03])
    ref = W.circle(40, 7.0, *centre)
    cur = _deformed(ref, centre)
    s = _sim(L, [(ref, 0.05, 0.02, 0.5, 3.0)])
    s.set_positions(0, cur)
    s.step(1, o.KINEMATIC)
    L0, th0, A0 = o.membrane_reference(ref)
    Fint = o.membrane_force(cur, L0, th0, A0, 0.05, 0.02, 0.5).reshape(-1, 2)
    fib = s.force_field()
    np.testing.assert_allclose(fib.sum(axis=(1, 2)), Fint.sum(0), atol=1e-15)
    # each node's force lands on its 3x3 support: the field's first moment is
    # sum_v F_v X_v (MLS reproduces linear functions)
    yy, xx = np.mgrid[0:40, 0:48].astype(float)
    np.testing.assert_allclose(np.sum(fib[0] * xx), np.sum(Fint[:, 0] * cur[:, 0]), atol=1e-12)
    np.testing.assert_allclose(np.sum(fib[1] * yy), np.sum(Fint[:, 1] * cur[:, 1]), atol=1e-12)


def test_dynamic_first_step_applies_no_forcing():
    # start-up: u_v^0 = I(u^0), so F_l = u_v - U = 0 and the first lattice update is
    # the plain update with the uniform body force only.
    L = o.lattice(40, 30, 0.7, walls=True, gx=1e-6)
    c = W.circle(24, 5.0, 20.2, 14.1)
    s = _sim(L, [(c, 0.2, 0.01, 0.0, 3.0)])
    rho, ux, uy = W.parabola(40, 30, 1e-6, 0.7)
    s.init_fields(rho, ux, uy)
    f0 = s.populations()
    s.step(1, o.DYNAMIC)
    np.testing.assert_allclose(s.populations(), o.collide_stream(L, f0, None), atol=1e-16)
    assert np.abs(s.force_field()).max() == 0.0


def test_dynamic_step_momentum_balance_equals_spread_force():
    # periodic box, no body force: the fluid momentum changes by exactly the total
    # spread force sum_l c_l F_l of each step (Guo moment identity).
    L = o.lattice(40, 36, 0.8)
    ref = W.circle(32, 6.0, 20.13, 18.07)
    rng = np.random.default_rng(4)
    s = _sim(L, [(ref, 0.3, 0.05, 0.5, 1.5)])
    ux = 0.01 * np.sin(2 * np.pi * np.arange(36) / 36)[:, None] * np.ones((1, 40))
    s.init_fields(None, ux, None)
    for _ in range(6):
        p0 = np.einsum("iyx,ia->a", s.populations(), E)
        s.step(1, o.DYNAMIC)
        p1 = np.einsum("iyx,ia->a", s.populations(), E)
        np.testing.assert_allclose(p1 - p0, s.force_field().sum(axis=(1, 2)), atol=2e-12)
    assert np.abs(s.force_field().sum(axis=(1, 2))).max() > 1e-7   # forcing is active


@pytest.mark.parametrize("scheme", [o.KINEMATIC, o.DYNAMIC])
def test_mass_is_conserved_in_a_channel_with_capsules(scheme):
    case = W.poiseuille_capsule(nx=80, ny=40, radius=6.0, n=32, ca=1e-2, scheme=scheme)
    L = o.lattice(case.nx, case.ny, case.tau, True, gx=case.gx)
    c = case.capsules[0]
    s = _sim(L, [(c.xy, c.ks, c.kb, c.ka, c.mass)])
    s.init_fields(*case.fields())
    m0 = s.populations().sum()
    assert s.step(100, scheme) == 0
    assert abs(s.populations().sum() - m0) < 1e-11 * m0


def test_support_touching_a_wall_is_reported():
    L = o.lattice(40, 30, 0.7, walls=True)
    c = W.circle(24, 5.0, 20.2, 5.3)     # lowest node at y = 0.3: support row -1
    s = _sim(L, [(c, 0.2, 0.01, 0.0, 3.0)])
    assert s.step(1, o.KINEMATIC) == 5


def test_kinematic_step_follows_steps_i_to_viii():
    # one step composed from the primitives in the order of Section 2.4
    L = o.lattice(36, 32, 0.8, walls=True, u_bottom=-0.004, u_top=0.004)
    ref = W.circle(28, 5.0, 18.2, 15.9)
    s = _sim(L, [(ref, 0.1, 0.02, 0.3, 2.0)])
    rho, ux, uy = W.linear_shear(36, 32, 0.004)
    s.init_fields(rho, ux, uy)
    s.step(3, o.KINEMATIC)
    f = s.populations()
    X, _, _, _ = s.read_capsule(0)
    X = X.reshape(-1, 2)
    s2 = _sim(L, [(ref, 0.1, 0.02, 0.3, 2.0)])
    s2.init_fields(rho, ux, uy)
    s2.step(2, o.KINEMATIC)
    Xm1 = s2.read_capsule(0)[0].reshape(-1, 2)
    s.step(1, o.KINEMATIC)
    L0, th0, A0 = o.membrane_reference(ref)
    Fint = o.membrane_force(X, L0, th0, A0, 0.1, 0.02, 0.3).reshape(-1, 2)    # i
    fib = np.zeros((2, L.ny, L.nx))
    for (px, py), (fx, fy) in zip(X, Fint):                                  # ii-iii
        o.spread(L, px, py, fx, fy, 1.0, fib)
    f1 = o.collide_stream(L, f, fib)                                         # iv-vi
    xdot = np.array([o.interp(L, f1, fib, px, py)[0][:2] for px, py in X])   # vii
    X1 = o.kinematic_advance(X, Xm1, xdot, first=False)                      # viii
    np.testing.assert_allclose(s.populations(), f1, atol=1e-16)
    np.testing.assert_allclose(s.force_field(), fib, atol=1e-18)
    np.testing.assert_allclose(s.read_capsule(0)[0].reshape(-1, 2), X1, atol=1e-14)


def test_dynamic_step_follows_steps_1_to_8():
    L = o.lattice(36, 32, 0.8, walls=True, gx=2e-6)
    ref = W.circle(28, 5.0, 18.2, 15.9)
    ks, kb, ka, m = 0.1, 0.02, 0.3, 2.0
    rho, ux, uy = W.parabola(36, 32, 2e-6, 0.8)
    s = _sim(L, [(ref, ks, kb, ka, m)])
    s.init_fields(rho, ux, uy)
    s.step(3, o.DYNAMIC)
    f = s.populations()
    X, uv, _, _ = s.read_capsule(0)
    X, uv = X.reshape(-1, 2), uv.reshape(-1, 2)
    s2 = _sim(L, [(ref, ks, kb, ka, m)])
    s2.init_fields(rho, ux, uy)
    s2.step(2, o.DYNAMIC)
    Xm1 = s2.read_capsule(0)[0].reshape(-1, 2)
    s.step(1, o.DYNAMIC)
    n = len(X)
    # Eq. 8 on the populations before any IB force (reading R1d): half of g only
    U = np.array([o.interp(L, f, None, px, py)[0][:2] for px, py in X])
    F = uv - U                                                                # step 1
    fib = np.zeros((2, L.ny, L.nx))
    for v in range(n):                                                        # steps 2-3
        cl = 0.5 * (np.hypot(*(X[v] - X[v - 1])) + np.hypot(*(X[(v + 1) % n] - X[v])))
        o.spread(L, X[v, 0], X[v, 1], F[v, 0], F[v, 1], cl, fib)
    f1 = o.collide_stream(L, f, fib)                                          # steps 4-6
    xd0 = U                      # tentative velocity of Eq. 23: U of step 1 (reading R11)
    nu = (0.8 - 0.5) / 3
    Fext = np.zeros_like(X)                                                   # Eq. 15-16
    for l in range(n):
        a, b = X[l], X[(l + 1) % n]
        d = b - a
        ln = np.hypot(*d)
        npl = np.array([d[1], -d[0]]) / ln
        c = 0.5 * (a + b)
        op = o.interp(L, f1, None, *(c + 1.2 * npl))[0]      # probes: reading R1d
        om = o.interp(L, f1, None, *(c - 1.2 * npl))[0]
        gp = op[4:].reshape(2, 2); gm = om[4:].reshape(2, 2)
        tp = op[2] * nu * (gp + gp.T); tm = om[2] * nu * (gm + gm.T)
        Fl = -(op[3] - om[3]) * npl * ln + (tp - tm) @ npl * ln
        Fext[l] += 0.5 * Fl
        Fext[(l + 1) % n] += 0.5 * Fl
    L0, th0, A0 = o.membrane_reference(ref)
    Fint = o.membrane_force(X, L0, th0, A0, ks, kb, ka).reshape(-1, 2)         # step 7
    X1, uv1 = o.dynamic_advance(X, Xm1, xd0, Fint + Fext, m)                  # step 8
    np.testing.assert_allclose(s.populations(), f1, atol=1e-16)
    got = s.read_capsule(0)
    np.testing.assert_allclose(got[0].reshape(-1, 2), X1, atol=1e-14)
    np.testing.assert_allclose(got[1].reshape(-1, 2), uv1, atol=1e-14)
    np.testing.assert_allclose(got[3].reshape(-1, 2), Fext, atol=1e-16)
