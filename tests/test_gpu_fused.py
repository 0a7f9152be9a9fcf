"""The node update of a step fused with the force and spread of the next: the Dynamic
scheme (Section 2.3.2 steps 7-8 and 1-3 read the same lattice state) and the Kinematic
one (Section 2.4: the advance of step n, then the membrane forces at X^{n+1} and their
spread). Against the separate kernels, against the oracle, through graphs and direct
launches, across call boundaries, and in the launch count it reports.
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


def suspension():
    return W.poiseuille_biconcave(nx=300, ny=96, count=6, n=64, seed=0, scheme=o.DYNAMIC)


def context(L, case, storage, fuse, graphs=True):
    ctx = L.from_case(case, storage=storage)
    ctx.set_option(L.OPT_ARCS, 1)          # one CTA per capsule: the fusable launch shape
    ctx.set_option(L.OPT_FUSE_IB, 1 if fuse else 0)
    ctx.set_option(L.OPT_GRAPHS, 1 if graphs else 0)
    ctx.set_option(L.OPT_GRAPH_STEPS, 16)   # graph boundaries inside the runs below
    return ctx


def state(ctx, ncaps):
    return ctx.read_populations(), np.concatenate([ctx.read_capsule(k)[0] for k in range(ncaps)])


# the shared-memory force tiles add several markers' shares in an unspecified order, so
# runs agree to rounding, not bit for bit
AGREE = {"fp64": 1e-12, "fp32": 2e-6}


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
@pytest.mark.parametrize("graphs", [True, False])
def test_fused_steps_match_the_separate_kernels(L, storage, graphs):
    case = suspension()
    a = context(L, case, storage, fuse=True, graphs=graphs)
    b = context(L, case, storage, fuse=False, graphs=graphs)
    a.step(70, L.DYNAMIC)        # 4 graphs of 16 steps and 6 direct ones
    b.step(70, L.DYNAMIC)
    pa, xa = state(a, len(case.capsules))
    pb, xb = state(b, len(case.capsules))
    print(f"{storage} graphs={graphs}: populations {np.abs(pa - pb).max():.2e}, positions {np.abs(xa - xb).max():.2e}")
    np.testing.assert_allclose(pa, pb, rtol=0, atol=AGREE[storage])
    np.testing.assert_allclose(xa, xb, rtol=0, atol=AGREE[storage] * 10)


def test_fused_steps_match_the_oracle(L):
    case = suspension()
    ctx = context(L, case, "fp64", fuse=True)
    s = o.Sim(o.lattice(case.nx, case.ny, case.tau, case.walls, case.u_bottom, case.u_top, case.gx, case.gy))
    s.init_fields(*case.fields())
    for c in case.capsules:
        s.add_capsule(c.xy, c.ks, c.kb, c.ka, c.mass)
    ctx.step(100, L.DYNAMIC)
    assert s.step(100, o.DYNAMIC) == 0
    _, u_g, v_g = ctx.read_fields()
    _, u_o, v_o = s.read_fields()
    err = max(np.abs(u_g - u_o).max(), np.abs(v_g - v_o).max()) / np.abs(u_o).max()
    assert err < 1e-10
    for k in range(len(case.capsules)):
        assert np.abs(ctx.read_capsule(k)[0] - s.read_capsule(k)[0]).max() < 1e-9


def test_call_boundaries_leave_no_spread_pending(L):
    # the fusion stays inside a call: 30 steps in one call, in three calls, and with a
    # Kinematic step in between (whose spread would double-count a pending one) agree
    case = suspension()
    a = context(L, case, "fp64", fuse=True)
    b = context(L, case, "fp64", fuse=True)
    a.step(30, L.DYNAMIC)
    for n in (7, 1, 22):
        b.step(n, L.DYNAMIC)
    np.testing.assert_allclose(a.read_populations(), b.read_populations(), rtol=0, atol=1e-12)
    c = context(L, case, "fp64", fuse=True)
    d = context(L, case, "fp64", fuse=False)
    for ctx in (c, d):
        ctx.step(10, L.DYNAMIC)
        ctx.step(1, L.KINEMATIC)
        ctx.step(10, L.DYNAMIC)
    np.testing.assert_allclose(c.read_populations(), d.read_populations(), rtol=0, atol=1e-12)


@pytest.mark.parametrize("graphs", [True, False])
def test_launch_count_of_fused_steps(L, graphs):
    # per step: lattice update, patch and update; the first step of a call adds its force
    # and spread, which the other steps get from the previous update
    case = suspension()
    for fuse in (True, False):
        ctx = context(L, case, "fp32", fuse=fuse, graphs=graphs)
        n0 = ctx.launch_count
        ctx.step(37, L.DYNAMIC)
        ctx.sync()
        if not fuse:
            expect = 4 * 37
        elif graphs:
            expect = 2 * (3 * 16 + 1) + (3 * 5 + 1)   # two graphs of 16 steps, then 5 direct steps
        else:
            expect = 3 * 37 + 1
        assert ctx.launch_count - n0 == expect


def test_fuse_option_is_checked(L):
    ctx = context(L, suspension(), "fp32", fuse=True)
    for bad in (-1, 2):
        with pytest.raises(L.LbmibError) as e:
            ctx.set_option(L.OPT_FUSE_IB, bad)
        assert e.value.status == L.ERR_ARG


def kinematic_suspension():
    return W.poiseuille_biconcave(nx=300, ny=96, count=6, n=64, seed=0, scheme=o.KINEMATIC)


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
@pytest.mark.parametrize("graphs", [True, False])
def test_fused_kinematic_steps_match_the_separate_kernels(L, storage, graphs):
    case = kinematic_suspension()
    a = context(L, case, storage, fuse=True, graphs=graphs)
    b = context(L, case, storage, fuse=False, graphs=graphs)
    a.step(70, L.KINEMATIC)
    b.step(70, L.KINEMATIC)
    pa, xa = state(a, len(case.capsules))
    pb, xb = state(b, len(case.capsules))
    print(f"kinematic {storage} graphs={graphs}: populations {np.abs(pa - pb).max():.2e}, "
          f"positions {np.abs(xa - xb).max():.2e}")
    np.testing.assert_allclose(pa, pb, rtol=0, atol=AGREE[storage])
    np.testing.assert_allclose(xa, xb, rtol=0, atol=AGREE[storage] * 10)


def test_fused_kinematic_steps_match_the_oracle(L):
    case = kinematic_suspension()
    ctx = context(L, case, "fp64", fuse=True)
    s = o.Sim(o.lattice(case.nx, case.ny, case.tau, case.walls, case.u_bottom, case.u_top, case.gx, case.gy))
    s.init_fields(*case.fields())
    for c in case.capsules:
        s.add_capsule(c.xy, c.ks, c.kb, c.ka, c.mass)
    ctx.step(100, L.KINEMATIC)
    assert s.step(100, o.KINEMATIC) == 0
    _, u_g, v_g = ctx.read_fields()
    _, u_o, v_o = s.read_fields()
    err = max(np.abs(u_g - u_o).max(), np.abs(v_g - v_o).max()) / np.abs(u_o).max()
    assert err < 1e-10
    for k in range(len(case.capsules)):
        assert np.abs(ctx.read_capsule(k)[0] - s.read_capsule(k)[0]).max() < 1e-9


def test_fused_kinematic_call_boundaries_and_launch_count(L):
    # one call against three, and against Dynamic steps in between; per fused step the
    # lattice update, the patch and the advance with the next spread
    case = kinematic_suspension()
    a = context(L, case, "fp64", fuse=True)
    b = context(L, case, "fp64", fuse=True)
    a.step(30, L.KINEMATIC)
    for n in (7, 1, 22):
        b.step(n, L.KINEMATIC)
    np.testing.assert_allclose(a.read_populations(), b.read_populations(), rtol=0, atol=1e-12)
    c = context(L, case, "fp64", fuse=True)
    d = context(L, case, "fp64", fuse=False)
    for ctx in (c, d):
        ctx.step(10, L.KINEMATIC)
        ctx.step(1, L.DYNAMIC)
        ctx.step(10, L.KINEMATIC)
    np.testing.assert_allclose(c.read_populations(), d.read_populations(), rtol=0, atol=1e-12)
    e = context(L, case, "fp32", fuse=True, graphs=False)
    n0 = e.launch_count
    e.step(37, L.KINEMATIC)
    e.sync()
    assert e.launch_count - n0 == 3 * 37 + 1
