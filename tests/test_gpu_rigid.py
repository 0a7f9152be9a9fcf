"""GPU parity of rigid particles (Section 2.3.1, Eq. 17-20) against the FP64 oracle: a free
disk in simple shear, an ellipse (a turning moment) in a body-force channel with its
ring whole or in arcs, a rigid particle beside a capsule with the repulsion on, and the
calls' refusals and the saved state.
"""
import numpy as np
import pytest

import oracle as o
from paper_1903_03356_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_03356_gb300 import lbmib
    return lbmib


def rigid_of(xy, rho_s=1.0):
    A, _, _, J = W.polygon_inertia(xy)
    return rho_s * A, rho_s * J


def pair(L, case, rigids, storage, arcs=0, rc=0.0):
    """GPU context and oracle for a case plus rigid particles [(xy, mass, inertia)]."""
    ctx = L.from_case(case, storage=storage, extra_nodes=sum(len(r[0]) for r in rigids),
                      extra_capsules=len(rigids))
    lat = o.lattice(case.nx, case.ny, case.tau, case.walls, case.u_bottom, case.u_top, case.gx, case.gy)
    s = o.Sim(lat)
    s.init_fields(*case.fields())
    for c in case.capsules:
        s.add_capsule(c.xy, c.ks, c.kb, c.ka, c.mass)
    ids = []
    for xy, m, I in rigids:
        ids.append(ctx.add_rigid(xy, m, I))
        assert s.add_rigid(xy, m, I) == ids[-1]
    if arcs:
        ctx.set_option(L.OPT_ARCS, arcs)
    if rc:
        ctx.set_repulsion(rc)
        s.set_repulsion(rc)
    return ctx, s, ids


def shear_case(ny=48, U=0.01):
    return W.Case("shear", 72, ny, 0.8, True, -U, U, init="shear")


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_free_disk_in_shear_matches_the_oracle(L, storage):
    case = shear_case()
    xy = W.circle(48, 5.0, 36.2, 23.57)
    m, I = rigid_of(xy)
    ctx, s, (k,) = pair(L, case, [(xy, m, I)], storage)
    ctx.step(400, L.DYNAMIC)
    assert s.step(400, o.DYNAMIC) == 0
    g, r = ctx.read_rigid(k), s.read_rigid(k)
    # relative to each quantity's scale: position 1, angle and velocities by the rotation
    # reached, the load by its largest component
    rel = 1e-9 if storage == "fp64" else 2e-4
    print(f"{storage}: omega gpu {g[5]:.6e} oracle {r[5]:.6e}; body error {np.abs(g[:6] - r[:6]).max():.2e}")
    np.testing.assert_allclose(g[:2], r[:2], rtol=0, atol=rel)
    np.testing.assert_allclose(g[2], r[2], rtol=0, atol=rel * abs(r[2]))
    np.testing.assert_allclose(g[3:6], r[3:6], rtol=0, atol=rel * abs(r[5]) * 10)
    np.testing.assert_allclose(g[6:], r[6:], rtol=0, atol=rel * np.abs(r[6:]).max() * 10)
    np.testing.assert_allclose(ctx.read_capsule(k)[0], s.read_capsule(k)[0], rtol=0, atol=rel * 10)
    assert r[5] < 0 and abs(r[2]) > 1e-4      # it turns clockwise with the shear


@pytest.mark.parametrize("arcs", [1, 4])
@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_ellipse_in_a_channel_matches_the_oracle(L, storage, arcs):
    # an ellipse at an angle in Poiseuille flow: a moment from the pressure and the shear
    ny = 40
    case = W.Case("chan", 96, ny, 0.7, True, gx=W.poiseuille_force(0.7, 0.02, ny), init="parabola")
    xy = W.ellipse(60, 8.0, 3.5, 40.3, 16.07, angle=0.6)
    m, I = rigid_of(xy, 1.5)
    ctx, s, (k,) = pair(L, case, [(xy, m, I)], storage, arcs=arcs)
    ctx.step(300, L.DYNAMIC)
    assert s.step(300, o.DYNAMIC) == 0
    g, r = ctx.read_rigid(k), s.read_rigid(k)
    err = np.abs(ctx.read_capsule(k)[0] - s.read_capsule(k)[0]).max()
    print(f"{storage} arcs {arcs}: marker error {err:.2e}; moved {np.hypot(r[0] - 40.3, r[1] - 16.07):.3f}, "
          f"turned {r[2]:.4f}")
    assert err < (1e-9 if storage == "fp64" else 1e-4)
    np.testing.assert_allclose(g[:6], r[:6], rtol=0, atol=(1e-9 if storage == "fp64" else 1e-4))
    assert abs(r[2]) > 1e-3


def test_rigid_particle_beside_a_capsule_with_repulsion(L):
    # a capsule and a rigid disk 1.3 apart in shear: repulsion between them, both schemes'
    # objects stepped by the Dynamic coupling
    case = shear_case()
    cap = W.circle(40, 6.0, 24.3, 23.57)
    W.check_no_ties(cap)
    case.capsules = [W.Capsule(cap, 0.02, 0.002, 0.0, W.node_mass(1.0, W.signed_area(cap), 40))]
    xy = W.circle(40, 5.0, 36.6, 23.9)
    m, I = rigid_of(xy)
    ctx, s, (k,) = pair(L, case, [(xy, m, I)], "fp64", rc=2.0)
    ctx.step(200, L.DYNAMIC)
    assert s.step(200, o.DYNAMIC) == 0
    for j in (0, k):
        assert np.abs(ctx.read_capsule(j)[0] - s.read_capsule(j)[0]).max() < 1e-9
    np.testing.assert_allclose(ctx.read_rigid(k)[:6], s.read_rigid(k)[:6], rtol=0, atol=1e-10)
    assert np.abs(s.read_repulsion(k)).max() > 0


def test_saved_state_carries_the_body(L):
    case = shear_case()
    xy = W.circle(48, 5.0, 36.2, 23.57)
    m, I = rigid_of(xy)
    a = L.from_case(case, storage="fp64", extra_nodes=48, extra_capsules=1)
    k = a.add_rigid(xy, m, I)
    a.step(50, L.DYNAMIC)
    snap = a.save_state()
    a.step(50, L.DYNAMIC)
    b = L.from_case(case, storage="fp64", extra_nodes=48, extra_capsules=1)
    b.add_rigid(xy, m, I)
    b.load_state(snap)
    b.step(50, L.DYNAMIC)
    np.testing.assert_array_equal(b.read_rigid(k), a.read_rigid(k))
    np.testing.assert_array_equal(b.read_capsule(k)[0], a.read_capsule(k)[0])


def test_rigid_particle_refusals(L):
    case = shear_case()
    xy = W.circle(32, 4.0, 36.2, 23.57)
    m, I = rigid_of(xy)
    ctx = L.from_case(case, storage="fp64", extra_nodes=64, extra_capsules=2)
    k = ctx.add_rigid(xy, m, I)
    with pytest.raises(L.LbmibError) as e:
        ctx.step(1, L.KINEMATIC)
    assert e.value.status == L.ERR_STATE
    with pytest.raises(L.LbmibError) as e:
        ctx.set_capsule_positions(k, xy)
    assert e.value.status == L.ERR_ARG
    with pytest.raises(L.LbmibError) as e:
        ctx.adjoint(5, scheme=L.DYNAMIC)
    assert e.value.status == L.ERR_STATE
    for bad in ((xy, -1.0, I), (xy, m, 0.0), (xy[::-1], m, I)):
        with pytest.raises(L.LbmibError) as e:
            ctx.add_rigid(*bad)
        assert e.value.status == L.ERR_ARG
    c2 = ctx.add_capsule(W.circle(32, 4.0, 12.2, 23.57), 0.02, 0.002, 0.0, 1.0)
    with pytest.raises(L.LbmibError) as e:
        ctx.read_rigid(c2)
    assert e.value.status == L.ERR_ARG
