"""Closed-form pins of the viscous part of the hydrodynamic traction (Eq. 16, reading R12:
tau = rho nu (grad u + grad u^T), nu = (tau_BGK - 1/2)/3) and of the outer-probe load of a
rigid particle (Eq. 17).

The flow is a piecewise-linear shear u_x = a+ (y - y0) above the line y = y0 and
a- (y - y0) below it, at uniform density rho != 1, held by equilibrium populations. The
element is tilted by 45 degrees across that line so that each probe (centroid +/- 1.2 n)
has its 3x3 support wholly in one linear piece (the kink row y0 carries u = 0 in both).
MLS reproduces linear fields, so each probe sees the exact gradient, and with the outward
normal n = (n_x, n_y) the element force is

    F = rho nu (a+ - a-) (n_y, n_x) l,   with no pressure part (p = rho/3 uniform).

A scale nu -> tau/3, a dropped rho or a dropped transpose (tau = rho nu grad u) each
change the y-component or the magnitude, so each fails these tests.
"""
import numpy as np
import pytest

import oracle as o


def _shear_fields(nx, ny, y0, a_up, a_dn, rho):
    yy, _ = np.mgrid[0:ny, 0:nx].astype(float)
    ux = np.where(yy >= y0, a_up * (yy - y0), a_dn * (yy - y0))
    return np.full((ny, nx), rho), ux, np.zeros((ny, nx))


def _tilted_element(centre, length, n):
    """Two vertices whose element has outward normal n = (dy, -dx)/l (reading R7)."""
    t = np.array([-n[1], n[0]])          # direction X2 - X1 with (dy, -dx)/l = n
    c = np.asarray(centre, float)
    return np.stack([c - 0.5 * length * t, c + 0.5 * length * t])


CASES = [
    # tau_BGK, rho, a+, a-, normal angle from the y axis
    (0.8, 1.25, 2e-3, -1e-3, 45.0),
    (0.65, 0.9, -1.5e-3, 4e-3, 45.0),
    (0.8, 1.1, 3e-3, 3e-3, 30.0),      # no jump in the gradient: no force
    (1.1, 1.3, 1e-3, -2.5e-3, -40.0),
]


@pytest.mark.parametrize("tau, rho, a_up, a_dn, ang", CASES)
def test_viscous_traction_of_a_piecewise_linear_shear_closed_form(tau, rho, a_up, a_dn, ang):
    nx, ny, y0 = 40, 40, 20
    L = o.lattice(nx, ny, tau)
    f = o.init_equilibrium(L, *_shear_fields(nx, ny, y0, a_up, a_dn, rho))
    th = np.radians(ang)
    n = np.array([np.sin(th), np.cos(th)])
    length = 0.7
    # centroid on the kink line, off the lattice nodes and half-integer lines
    xy = _tilted_element((19.83, y0 + 0.03), length, n)
    for s in (+1.0, -1.0):   # each probe's support lies on one side of y0 (row y0 shared)
        ix, iy, phi, gx, gy, st = o.mls(L, *(xy.mean(axis=0) + s * 1.2 * n))
        assert st == 0
        assert (iy >= y0).all() if s > 0 else (iy <= y0).all()
    # a two-vertex ring: the second element runs back with normal -n, and its probes are
    # the first element's with the roles swapped, so both elements carry the same force
    # and each vertex receives all of it
    Fext, st = o.tractions(L, f, None, xy)
    assert st == 0
    nu = (tau - 0.5) / 3.0
    expect = rho * nu * (a_up - a_dn) * np.array([n[1], n[0]]) * length
    np.testing.assert_allclose(Fext[0], expect, rtol=1e-11, atol=1e-15)
    np.testing.assert_allclose(Fext[1], expect, rtol=1e-11, atol=1e-15)


@pytest.mark.parametrize("tau, rho, a_up, a_dn, ang", CASES)
def test_rigid_load_viscous_part_closed_form(tau, rho, a_up, a_dn, ang):
    # Eq. 17 takes the outer probe of every element. On the same two-vertex ring the
    # outer probe of the returning element is the inner probe of the first, with the
    # normal reversed: the summed load is the same jump, rho nu (a+ - a-)(n_y, n_x) l (the
    # uniform pressure cancels between the two), and the moment about the common
    # centroid vanishes.
    nx, ny, y0 = 40, 40, 20
    L = o.lattice(nx, ny, tau)
    f = o.init_equilibrium(L, *_shear_fields(nx, ny, y0, a_up, a_dn, rho))
    th = np.radians(ang)
    n = np.array([np.sin(th), np.cos(th)])
    length = 0.7
    xy = _tilted_element((19.83, y0 + 0.03), length, n)
    c = xy.mean(axis=0)
    load, st = o.rigid_load(L, f, None, xy, c[0], c[1])
    assert st == 0
    nu = (tau - 0.5) / 3.0
    expect = rho * nu * (a_up - a_dn) * np.array([n[1], n[0]]) * length
    np.testing.assert_allclose(load[:2], expect, rtol=1e-11, atol=1e-15)
    assert abs(load[2]) < 1e-15
