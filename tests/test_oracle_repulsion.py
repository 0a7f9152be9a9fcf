"""Pins of the oracle's capsule-capsule repulsion (Section 3.4, Eq. 27; readings R23, R24).

Eq. 27: the force on vertex 1 from vertex 2 of another capsule at distance d is
1e-4 / (8 sqrt 2) * sqrt(dx / d^5) along the inward normal at vertex 1 (dx = 1).
"""
import numpy as np
import pytest

import oracle as o

C = 1e-4 / (8.0 * np.sqrt(2.0))


def square(cx, cy, h):
    return np.array([[cx - h, cy - h], [cx + h, cy - h], [cx + h, cy + h], [cx - h, cy + h]])


def polygon(n, r, cx, cy):
    t = 2 * np.pi * np.arange(n) / n
    return np.stack([cx + r * np.cos(t), cy + r * np.sin(t)], axis=1)


def test_coefficient_is_the_printed_one():
    assert o.REPULSION_COEFF == pytest.approx(1e-4 / (8 * 2 ** 0.5), rel=1e-15)


def test_vertex_normal_of_a_regular_polygon_is_radial():
    xy = polygon(12, 5.0, 3.0, -2.0)
    for v in range(12):
        radial = (xy[v] - [3.0, -2.0]) / 5.0
        np.testing.assert_allclose(o.vertex_normal(xy, v), radial, atol=1e-14)
    # a square corner: the diagonal
    np.testing.assert_allclose(o.vertex_normal(square(0, 0, 1), 2), [2 ** -0.5, 2 ** -0.5], atol=1e-15)


def test_one_pair_in_range_gives_the_closed_form():
    # A's right corners (x = 12) face B's left corners (x = 13) at distance 1; the
    # diagonal pairs are sqrt(17) apart, beyond the cut-off
    A, B = square(10, 10, 2), square(15, 10, 2)
    FA, FB = o.repulsion([A, B], rc=1.5)
    for v in (1, 2):
        n = o.vertex_normal(A, v)
        np.testing.assert_allclose(FA[v], -C * n, rtol=1e-14, atol=0)
    for v in (0, 3):
        n = o.vertex_normal(B, v)
        np.testing.assert_allclose(FB[v], -C * n, rtol=1e-14, atol=0)
    assert not FA[[0, 3]].any() and not FB[[1, 2]].any()


@pytest.mark.parametrize("d", [0.5, 0.8, 1.3])
def test_magnitude_scales_as_d_to_the_minus_five_halves(d):
    A, B = square(10, 10, 2), square(14 + d, 10, 2)
    FA, _ = o.repulsion([A, B], rc=2.0)
    assert np.linalg.norm(FA[1]) == pytest.approx(C * d ** -2.5, rel=1e-14)


def test_cut_off_and_same_ring_vertices():
    A, B = square(10, 10, 2), square(15, 10, 2)
    FA, FB = o.repulsion([A, B], rc=0.999)   # distance 1 is outside
    assert not FA.any() and not FB.any()
    # one ring alone, vertices 0.3 apart: no self-interaction
    (F,) = o.repulsion([polygon(64, 3.0, 0, 0)], rc=2.0)
    assert not F.any()


def test_forces_from_several_neighbours_add():
    A = square(10, 10, 2)
    B = np.array([[12.5, 8.0], [12.0, 7.4], [14.0, 6.0]])   # clockwise is fine for the source ring
    FA, _ = o.repulsion([A, B], rc=1.0)
    n = o.vertex_normal(A, 1)
    expect = -C * n * (0.5 ** -2.5 + 0.6 ** -2.5)
    np.testing.assert_allclose(FA[1], expect, rtol=1e-14)


def test_periodic_minimum_image():
    # B sits across the periodic x boundary of a 40-wide lattice: A's left corners at
    # x = 1, B's right corners at x = 39 = -1 (mod 40): distance 2
    A, B = square(3, 10, 2), square(37, 10, 2)
    FA, _ = o.repulsion([A, B], rc=2.5, px=40.0)
    n = o.vertex_normal(A, 0)
    np.testing.assert_allclose(FA[0], -C * 2.0 ** -2.5 * n, rtol=1e-14)
    FA0, _ = o.repulsion([A, B], rc=2.5)     # without the period they are 34 apart
    assert not FA0.any()


@pytest.mark.parametrize("scheme", [o.KINEMATIC, o.DYNAMIC])
def test_simulation_uses_the_forces_at_the_step_start(scheme):
    lat = o.lattice(64, 40, 0.8, True)
    A, B = polygon(32, 6.0, 24.3, 20.07), polygon(32, 6.0, 37.1, 20.07)   # closest vertices 0.8 apart
    s = o.Sim(lat)
    for xy in (A, B):
        s.add_capsule(xy, 0.01, 0.001, 0.0, 1.0)
    s.set_repulsion(1.5)
    s.step(1, scheme)
    FA, FB = o.repulsion([A, B], rc=1.5, px=64.0)
    np.testing.assert_array_equal(s.read_repulsion(0), FA.reshape(-1))
    np.testing.assert_array_equal(s.read_repulsion(1), FB.reshape(-1))
    assert np.abs(FA).max() > 0


@pytest.mark.parametrize("scheme", [o.KINEMATIC, o.DYNAMIC])
def test_far_apart_capsules_are_unaffected(scheme):
    lat = o.lattice(96, 40, 0.8, True, u_bottom=-0.002, u_top=0.002)
    A, B = polygon(32, 6.0, 24.3, 20.07), polygon(32, 6.0, 70.1, 20.07)
    runs = []
    for rc in (0.0, 2.0):
        s = o.Sim(lat)
        for xy in (A, B):
            s.add_capsule(xy, 0.01, 0.001, 0.0, 1.0)
        s.set_repulsion(rc)
        s.step(20, scheme)
        runs.append(np.concatenate([s.read_capsule(0)[0], s.read_capsule(1)[0]]))
    np.testing.assert_array_equal(runs[0], runs[1])
