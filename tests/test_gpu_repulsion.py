"""GPU parity of the capsule-capsule repulsion (Section 3.4, Eq. 27) against the FP64
oracle, both schemes: capsules closer than the cut-off move as the oracle's do; capsules
farther apart are untouched; pairs across the periodic x boundary interact.
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


def polygon(n, r, cx, cy):
    t = 2 * np.pi * (np.arange(n) + 0.137) / n   # phase keeps vertices off half-integer lines
    return np.stack([cx + r * np.cos(t), cy + r * np.sin(t)], axis=1)


def run_pair(L, case, scheme, rc, storage, T):
    ctx = L.from_case(case, storage=storage)
    ctx.set_repulsion(rc)
    ctx.step(T, scheme)
    s = o.Sim(o.lattice(case.nx, case.ny, case.tau, case.walls, case.u_bottom, case.u_top, case.gx, case.gy))
    s.init_fields(*case.fields())
    for c in case.capsules:
        s.add_capsule(c.xy, c.ks, c.kb, c.ka, c.mass)
    s.set_repulsion(rc)
    assert s.step(T, scheme) == 0
    return ctx, s


def capsules(centres, r=7.0, n=48):
    out = []
    for cx, cy in centres:
        xy = polygon(n, r, cx, cy)
        W.check_no_ties(xy)
        out.append(W.Capsule(xy, 0.02, 0.002, 0.0, W.node_mass(1.0, W.signed_area(xy), n)))
    return out


def close_pair(scheme):
    # two circles whose nearest vertices are about 0.9 apart, in a sheared channel
    caps = capsules([(30.3, 20.07), (45.1, 20.57)])
    return W.Case("pair", 80, 40, 0.8, True, -0.004, 0.004, init="shear", capsules=caps, scheme=scheme)


@pytest.mark.parametrize("scheme,T", [(o.KINEMATIC, 300), (o.DYNAMIC, 150)])
@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_close_capsules_match_the_oracle(L, scheme, T, storage):
    case = close_pair(scheme)
    ctx, s = run_pair(L, case, scheme, 2.0, storage, T)
    tol = 1e-9 if storage == "fp64" else 1e-4
    worst = 0.0
    for k in range(2):
        err = np.abs(ctx.read_capsule(k)[0] - s.read_capsule(k)[0]).max()
        print(f"{storage} scheme {scheme} capsule {k}: position error {err:.2e}")
        assert err < tol
        worst = max(worst, err)
    # the repulsion acted: without it the oracle's rings end elsewhere, by far more than
    # the GPU's distance from the oracle
    s0 = o.Sim(o.lattice(case.nx, case.ny, case.tau, True, case.u_bottom, case.u_top))
    s0.init_fields(*case.fields())
    for c in case.capsules:
        s0.add_capsule(c.xy, c.ks, c.kb, c.ka, c.mass)
    s0.step(T, scheme)
    effect = np.abs(s0.read_capsule(0)[0] - s.read_capsule(0)[0]).max()
    print(f"  displacement due to the repulsion {effect:.2e}")
    assert effect > max(100 * worst, 1e-6)


def test_pairs_across_the_periodic_boundary(L):
    # one circle ends at x = 79.6 of an 80-wide lattice, the other starts at x = 0.4:
    # 0.8 apart through the periodic boundary only
    caps = capsules([(72.6, 20.07), (7.4, 20.37)])
    case = W.Case("seam", 80, 40, 0.8, True, -0.004, 0.004, init="shear", capsules=caps, scheme=o.KINEMATIC)
    ctx, s = run_pair(L, case, o.KINEMATIC, 2.0, "fp64", 200)
    for k in range(2):
        assert np.abs(ctx.read_capsule(k)[0] - s.read_capsule(k)[0]).max() < 1e-9


@pytest.mark.parametrize("scheme", [o.KINEMATIC, o.DYNAMIC])
def test_dense_pack_matches_the_oracle(L, scheme):
    # a 3 x 2 block of circles 1.1 to 1.3 apart in a body-force channel
    centres = [(20.3 + 15.1 * i + 0.1 * j, 12.07 + 15.2 * j) for i in range(3) for j in range(2)]
    case = W.Case("pack", 96, 40, 0.7, True, gx=W.poiseuille_force(0.7, 0.01, 40), init="parabola",
                  capsules=capsules(centres), scheme=scheme)
    ctx, s = run_pair(L, case, scheme, 2.0, "fp64", 100)
    for k in range(len(case.capsules)):
        assert np.abs(ctx.read_capsule(k)[0] - s.read_capsule(k)[0]).max() < 1e-9


@pytest.mark.parametrize("scheme", [o.KINEMATIC, o.DYNAMIC])
def test_far_apart_capsules_are_unchanged_by_the_repulsion(L, scheme):
    A, B = polygon(48, 7.0, 20.3, 20.07), polygon(48, 7.0, 60.1, 20.57)
    caps = [W.Capsule(xy, 0.02, 0.002, 0.0, 1.0) for xy in (A, B)]
    case = W.Case("far", 80, 40, 0.8, True, -0.004, 0.004, init="shear", capsules=caps, scheme=scheme)
    a = L.from_case(case, storage="fp64")
    b = L.from_case(case, storage="fp64")
    b.set_repulsion(2.0)
    a.step(60, scheme)
    b.step(60, scheme)
    for k in range(2):
        np.testing.assert_allclose(b.read_capsule(k)[0], a.read_capsule(k)[0], rtol=0, atol=1e-13)


def test_repulsion_arguments_are_checked(L):
    ctx = L.from_case(close_pair(o.KINEMATIC), storage="fp64")
    for bad in (-1.0, 17.0, float("nan")):
        with pytest.raises(L.LbmibError) as e:
            ctx.set_repulsion(bad)
        assert e.value.status == L.ERR_ARG
    ctx.set_repulsion(2.0)
    with pytest.raises(L.LbmibError) as e:      # the adjoint does not cover the repulsion
        ctx.adjoint(5, scheme=L.KINEMATIC)
    assert e.value.status == L.ERR_STATE
