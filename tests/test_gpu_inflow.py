"""GPU parity of the open channel (Section 2.1 Zou-He boundaries, Section 3.2 parabolic inlet
and constant-pressure outlet) against the FP64 oracle: the lattice alone (with and without
a body force, ragged sizes), the populations read back, a capsule in the channel with both
schemes, the support rule at the open columns, and the call's argument checks.
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


def oracle_of(case):
    lat = o.lattice(case.nx, case.ny, case.tau, case.walls, case.u_bottom, case.u_top, case.gx, case.gy,
                    u_in=case.u_in, rho_out=case.rho_out)
    s = o.Sim(lat)
    s.init_fields(*case.fields())
    for c in case.capsules:
        s.add_capsule(c.xy, c.ks, c.kb, c.ka, c.mass)
    return s


def channel(nx, ny, u_max=0.02, gx=0.0, gy=0.0, walls=True, profile=None, rho_out=1.0):
    u_in = W.inlet_parabola(ny, u_max) if profile is None else profile
    return W.Case("open", nx, ny, 0.7, walls, gx=gx, gy=gy, init="rest", u_in=u_in, rho_out=rho_out)


TOL = {"fp64": 1e-12, "fp32": 2e-5}


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
@pytest.mark.parametrize("nx,ny,gx,gy,walls", [
    (96, 24, 0.0, 0.0, True),          # the paper's channel: inlet and outlet only
    (203, 37, 2e-6, -1e-6, True),      # ragged rows, a body force at the open columns
    (64, 20, 0.0, 1e-6, False),        # periodic in y
])
def test_open_lattice_matches_the_oracle(L, storage, nx, ny, gx, gy, walls):
    profile = None if walls else 0.01 * (1.0 + 0.3 * np.sin(2 * np.pi * (np.arange(ny) + 0.5) / ny))
    case = channel(nx, ny, gx=gx, gy=gy, walls=walls, profile=profile, rho_out=1.002)
    ctx = L.from_case(case, storage=storage)
    s = oracle_of(case)
    ctx.step(400)
    s.step(400, o.KINEMATIC)
    rho_g, ux_g, uy_g = ctx.read_fields()
    rho_o, ux_o, uy_o = s.read_fields()
    scale = np.abs(ux_o).max()
    err = max(np.abs(ux_g - ux_o).max(), np.abs(uy_g - uy_o).max()) / scale
    print(f"{storage} {nx}x{ny}: velocity error / max |u| = {err:.2e}, density {np.abs(rho_g - rho_o).max():.2e}")
    assert err < TOL[storage]
    assert np.abs(rho_g - rho_o).max() < TOL[storage] * 0.1
    # the open columns hold their prescribed state
    atol = 1e-14 if storage == "fp64" else 2e-6
    np.testing.assert_allclose(ux_g[:, 0], case.u_in, rtol=0, atol=atol)
    np.testing.assert_allclose(rho_g[:, -1], 1.002, rtol=0, atol=atol)


def test_populations_read_back_match_the_oracle(L):
    case = channel(48, 16, gx=1e-6)
    ctx = L.from_case(case, storage="fp64")
    s = oracle_of(case)
    ctx.step(50)
    s.step(50, o.KINEMATIC)
    np.testing.assert_allclose(ctx.read_populations(), s.populations(), rtol=0, atol=1e-14)


def test_fp16_storage_in_an_open_channel(L):
    case = channel(128, 32)
    ctx = L.from_case(case, storage="fp16")
    s = oracle_of(case)
    ctx.step(400)
    s.step(400, o.KINEMATIC)
    _, ux_g, _ = ctx.read_fields()
    _, ux_o, _ = s.read_fields()
    err = np.abs(ux_g - ux_o).max() / np.abs(ux_o).max()
    print(f"fp16 open channel: velocity error / max |u| = {err:.2e}")
    assert err < 5e-3
    np.testing.assert_allclose(ux_g[:, 0], case.u_in, atol=1e-4)


def small_section_3_2(scheme):
    # Section 3.2 proportions at a size the oracle runs in seconds: H = 40, L = 3H,
    # capsule diameter 7/15 H, elements 0.5 lattice units, centre at 0.433 H
    return W.open_channel_capsule(ny=40, diameter=18.7, spacing=0.5, y_frac=0.433, u_max=0.02, scheme=scheme)


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
@pytest.mark.parametrize("scheme,T", [(o.KINEMATIC, 400), (o.DYNAMIC, 200)])
def test_capsule_in_the_open_channel_matches_the_oracle(L, storage, scheme, T):
    case = small_section_3_2(scheme)
    ctx = L.from_case(case, storage=storage)
    s = oracle_of(case)
    ctx.step(T, scheme)
    assert s.step(T, scheme) == 0
    err = np.abs(ctx.read_capsule(0)[0] - s.read_capsule(0)[0]).max()
    moved = np.abs(s.read_capsule(0)[0] - case.capsules[0].xy.reshape(-1)).max()
    print(f"{storage} scheme {scheme}: position error {err:.2e} (the capsule moved {moved:.3f})")
    assert err < (1e-9 if storage == "fp64" else 1e-4)
    assert moved > 0.05
    assert abs(ctx.observables(0)[2] - s.observables(0)[2]) < (1e-10 if storage == "fp64" else 1e-4)


def test_capsules_with_repulsion_in_the_open_channel(L):
    # two rings 1.8 apart (inside the cut-off), x distances without the periodic image
    t = 2 * np.pi * (np.arange(40) + 0.137) / 40
    caps = []
    for cx, cy in ((30.3, 14.07), (44.1, 14.57)):
        xy = np.stack([cx + 6.0 * np.cos(t), cy + 6.0 * np.sin(t)], 1)
        W.check_no_ties(xy)
        caps.append(W.Capsule(xy, 0.02, 0.002, 0.0, W.node_mass(1.0, W.signed_area(xy), 40)))
    case = W.Case("pair", 96, 30, 0.8, True, init="rest", capsules=caps, u_in=W.inlet_parabola(30, 0.01))
    ctx = L.from_case(case, storage="fp64")
    ctx.set_repulsion(2.0)
    s = oracle_of(case)
    s.set_repulsion(2.0)
    ctx.step(150, o.DYNAMIC)
    assert s.step(150, o.DYNAMIC) == 0
    for k in range(2):
        assert np.abs(ctx.read_capsule(k)[0] - s.read_capsule(k)[0]).max() < 1e-9


def test_support_on_an_open_column_is_reported(L):
    case = channel(48, 24, u_max=0.01)
    ctx = L.from_case(case, storage="fp32", extra_nodes=24, extra_capsules=1)
    ctx.add_capsule(W.circle(24, 4.0, 5.2, 12.3), 0.02, 0.002, 0.0, 1.0)    # support reaches column 0
    ctx.step(1, o.KINEMATIC)
    with pytest.raises(L.LbmibError) as e:
        ctx.sync()
    assert e.value.status == L.ERR_SUPPORT


def test_graphs_and_direct_launches_agree_and_periodic_x_comes_back(L):
    case = channel(64, 20, gx=1e-6)
    a = L.from_case(case, storage="fp64")
    b = L.from_case(case, storage="fp64")
    b.set_option(L.OPT_GRAPHS, 0)
    a.step(37)
    b.step(37)
    np.testing.assert_array_equal(a.read_populations(), b.read_populations())
    # back to periodic x: the same as a context that never had the open channel
    p = L.from_case(channel(64, 20, gx=1e-6), storage="fp64")
    p.set_inflow(None)
    q = L.from_case(W.Case("per", 64, 20, 0.7, True, gx=1e-6), storage="fp64")
    p.step(20)
    q.step(20)
    np.testing.assert_array_equal(p.read_populations(), q.read_populations())


def test_inflow_arguments_are_checked(L):
    ctx = L.from_case(channel(32, 12), storage="fp64")
    for u, r in ((np.full(12, 0.3), 1.0), (np.full(12, np.nan), 1.0), (np.zeros(12), 0.4), (np.zeros(12), 2.5)):
        with pytest.raises(L.LbmibError) as e:
            ctx.set_inflow(u, r)
        assert e.value.status == L.ERR_ARG
    with pytest.raises(ValueError):
        ctx.set_inflow(np.zeros(11))
    small = L.Context(4, 12, 0.7, True, storage="fp64")
    with pytest.raises(L.LbmibError) as e:
        small.set_inflow(np.zeros(12))
    assert e.value.status == L.ERR_ARG


def test_adjoint_refuses_the_open_channel(L):
    case = small_section_3_2(o.KINEMATIC)
    ctx = L.from_case(case, storage="fp64")
    with pytest.raises(L.LbmibError) as e:
        ctx.adjoint(5, scheme=L.KINEMATIC)
    assert e.value.status == L.ERR_STATE
