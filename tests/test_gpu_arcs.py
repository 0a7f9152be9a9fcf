"""The capsule kernels split over several CTAs per capsule (arcs, one thread-block cluster
per capsule where the enclosed area is needed) give the oracle's results, whatever the
split: both schemes, the area term on (Eq. 14), splits with CTAs that own no vertex, and
the global-memory path of a capsule larger than its tile.
"""
import dataclasses

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


def with_area(case, ka):
    return dataclasses.replace(case, capsules=[dataclasses.replace(c, ka=ka) for c in case.capsules])


def oracle_run(case, scheme, T):
    s = o.Sim(o.lattice(case.nx, case.ny, case.tau, case.walls, case.u_bottom, case.u_top, case.gx, case.gy))
    s.init_fields(*case.fields())
    for c in case.capsules:
        s.add_capsule(c.xy, c.ks, c.kb, c.ka, c.mass)
    assert s.step(T, scheme) == 0
    return s


def gpu_run(L, case, scheme, T, arcs, storage="fp64"):
    ctx = L.from_case(case, storage=storage)
    ctx.set_option(L.OPT_ARCS, arcs)
    ctx.step(T, scheme)
    return ctx


def cases(scheme):
    if scheme == o.KINEMATIC:
        return with_area(W.shear_capsule(nx=100, ny=100, ca=1e-3, scheme=o.KINEMATIC), 0.05), 400
    return with_area(W.poiseuille_capsule(nx=160, ny=64, radius=8.0, n=48, ca=1e-2, y_frac=0.45,
                                          scheme=o.DYNAMIC), 0.05), 200


@pytest.mark.parametrize("arcs", [1, 3, 8])
@pytest.mark.parametrize("scheme", [o.KINEMATIC, o.DYNAMIC])
def test_every_split_matches_the_oracle(L, scheme, arcs):
    case, T = cases(scheme)
    s = oracle_run(case, scheme, T)
    ctx = gpu_run(L, case, scheme, T, arcs)
    xy_g, vel_g, fi_g, fe_g = ctx.read_capsule(0)
    xy_o, vel_o, fi_o, fe_o = s.read_capsule(0)
    err = np.abs(xy_g - xy_o).max()
    print(f"scheme {scheme} arcs {arcs}: position error {err:.2e}")
    assert err < 1e-9
    np.testing.assert_allclose(fi_g, fi_o, atol=1e-12 * max(1.0, np.abs(fi_o).max()))
    _, u_g, v_g = ctx.read_fields()
    _, u_o, v_o = s.read_fields()
    np.testing.assert_allclose(np.stack([u_g, v_g]), np.stack([u_o, v_o]), rtol=0, atol=1e-12)


@pytest.mark.parametrize("scheme", [o.KINEMATIC, o.DYNAMIC])
def test_splits_agree_with_each_other_in_single_precision(L, scheme):
    case, T = cases(scheme)
    ref = gpu_run(L, case, scheme, T, 1, "fp32").read_capsule(0)[0]
    for arcs in (2, 5, 8):
        got = gpu_run(L, case, scheme, T, arcs, "fp32").read_capsule(0)[0]
        assert np.abs(got - ref).max() < 1e-5


@pytest.mark.parametrize("scheme", [o.KINEMATIC, o.DYNAMIC])
def test_arcs_without_vertices(L, scheme):
    # 17 vertices in 8 arcs of 3: the sixth CTA owns 2 vertices, the last two none, and
    # the cluster's area sum still needs them
    xy = W.circle(17, 5.0, 30.2, 20.07)
    W.check_no_ties(xy)
    ks = 0.01
    cap = W.Capsule(xy, ks, 1e-3, 0.05, W.node_mass(1.0, W.signed_area(xy), 17))
    case = W.Case("small", 64, 40, 0.8, True, -0.004, 0.004, init="shear", capsules=[cap], scheme=scheme)
    s = oracle_run(case, scheme, 100)
    for arcs in (6, 8):
        ctx = gpu_run(L, case, scheme, 100, arcs)
        assert np.abs(ctx.read_capsule(0)[0] - s.read_capsule(0)[0]).max() < 1e-9


@pytest.mark.parametrize("scheme", [o.KINEMATIC, o.DYNAMIC])
def test_capsule_larger_than_its_tile_takes_the_global_path(L, scheme):
    # one CTA for a radius-40 ring of 250 vertices: its box (about 88 x 88 nodes) exceeds
    # the tile budget, so the kernels gather and spread through global memory
    case = W.shear_capsule(nx=128, ny=128, radius=40.0, n=250, ca=1e-2, scheme=scheme)
    s = oracle_run(case, scheme, 150)
    ctx = gpu_run(L, case, scheme, 150, 1)
    assert np.abs(ctx.read_capsule(0)[0] - s.read_capsule(0)[0]).max() < 1e-9
    _, u_g, v_g = ctx.read_fields()
    _, u_o, v_o = s.read_fields()
    np.testing.assert_allclose(np.stack([u_g, v_g]), np.stack([u_o, v_o]), rtol=0, atol=1e-12)


def test_several_capsules_in_clusters_match_the_oracle(L):
    case = with_area(W.poiseuille_biconcave(nx=300, ny=96, count=6, n=64, seed=0, scheme=o.DYNAMIC), 0.02)
    s = oracle_run(case, o.DYNAMIC, 100)
    ctx = gpu_run(L, case, o.DYNAMIC, 100, 4)
    for k in range(len(case.capsules)):
        assert np.abs(ctx.read_capsule(k)[0] - s.read_capsule(k)[0]).max() < 1e-9


def test_arcs_option_is_checked(L):
    case, _ = cases(o.KINEMATIC)
    ctx = L.from_case(case, storage="fp64")
    for bad in (-1, 9):
        with pytest.raises(L.LbmibError) as e:
            ctx.set_option(L.OPT_ARCS, bad)
        assert e.value.status == L.ERR_ARG
