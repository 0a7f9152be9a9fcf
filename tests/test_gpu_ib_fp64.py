"""Single-precision storage with the immersed-boundary arithmetic in FP64
(LBMIB_OPT_IB_FP64): gathers in storage precision, the MLS solve, membrane and traction
forces and node update in double. Against the FP64 oracle within the FP32 bounds, both
schemes, split rings and the fused one-CTA-per-capsule path, FP16 storage, rigid
particles, and the option's checks.
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
    s = o.Sim(o.lattice(case.nx, case.ny, case.tau, case.walls, case.u_bottom, case.u_top, case.gx, case.gy))
    s.init_fields(*case.fields())
    for c in case.capsules:
        s.add_capsule(c.xy, c.ks, c.kb, c.ka, c.mass)
    return s


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("arcs", [0, 1])   # automatic split, and one CTA per capsule (fused)
def test_dynamic_fp32_storage_with_fp64_ib_matches_the_oracle(L, arcs):
    case = W.poiseuille_biconcave(nx=300, ny=96, count=6, n=64, seed=0, scheme=o.DYNAMIC)
    ctx = L.from_case(case, storage="fp32")
    ctx.set_option(L.OPT_IB_FP64, 1)
    ctx.set_option(L.OPT_ARCS, arcs)
    s = oracle_of(case)
    ctx.step(100, L.DYNAMIC)
    assert s.step(100, o.DYNAMIC) == 0
    _, u_g, v_g = ctx.read_fields()
    _, u_o, v_o = s.read_fields()
    err = rel(np.stack([u_g, v_g]), np.stack([u_o, v_o]))
    print(f"arcs={arcs}: velocity rel err {err:.3e}")
    assert err < 1e-5
    for k in range(len(case.capsules)):
        assert np.abs(ctx.read_capsule(k)[0] - s.read_capsule(k)[0]).max() < 1e-4
        assert abs(ctx.observables(k)[2] - s.observables(k)[2]) < 1e-4


def test_kinematic_fp32_storage_with_fp64_ib_matches_the_oracle(L):
    case = W.shear_capsule(nx=100, ny=100, ca=1e-3, scheme=o.KINEMATIC)
    ctx = L.from_case(case, storage="fp32")
    ctx.set_option(L.OPT_IB_FP64, 1)
    s = oracle_of(case)
    ctx.step(1000, L.KINEMATIC)
    assert s.step(1000, o.KINEMATIC) == 0
    _, u_g, v_g = ctx.read_fields()
    _, u_o, v_o = s.read_fields()
    err = rel(np.stack([u_g, v_g]), np.stack([u_o, v_o]))
    print(f"kinematic: velocity rel err {err:.3e}")
    assert err < 1e-5
    assert abs(ctx.observables(0)[2] - s.observables(0)[2]) < 1e-4


def test_fp16_storage_with_fp64_ib_agrees_with_the_default(L):
    case = W.poiseuille_biconcave(nx=300, ny=96, count=6, n=64, seed=0, scheme=o.DYNAMIC)
    a = L.from_case(case, storage="fp16")
    b = L.from_case(case, storage="fp16")
    b.set_option(L.OPT_IB_FP64, 1)
    a.step(100, L.DYNAMIC)
    b.step(100, L.DYNAMIC)
    for k in range(len(case.capsules)):
        assert np.abs(a.read_capsule(k)[0] - b.read_capsule(k)[0]).max() < 1e-3


def test_rigid_particles_with_fp64_ib(L):
    t = 2 * np.pi * (np.arange(48) + 0.137) / 48
    xy = np.stack([36.2 + 5.0 * np.cos(t), 23.57 + 5.0 * np.sin(t)], 1)
    area = 0.5 * np.abs(np.sum(xy[:, 0] * np.roll(xy[:, 1], -1) - np.roll(xy[:, 0], -1) * xy[:, 1]))
    runs = []
    for wide in (0, 1):
        ctx = L.Context(72, 48, 0.8, True, storage="fp32", u_bottom=-0.01, u_top=0.01, max_nodes=64, max_capsules=2)
        ctx.set_option(L.OPT_IB_FP64, wide)
        ctx.init_fields()
        ctx.add_rigid(xy, area, area * 12.5)
        ctx.step(300, L.DYNAMIC)
        runs.append(ctx.read_rigid(0))
    np.testing.assert_allclose(runs[1], runs[0], rtol=0, atol=1e-6)


def test_fp64_ib_option(L):
    case = W.poiseuille_biconcave(nx=300, ny=96, count=2, n=64, seed=0, scheme=o.DYNAMIC)
    a = L.from_case(case, storage="fp64")
    b = L.from_case(case, storage="fp64")
    b.set_option(L.OPT_IB_FP64, 1)            # no effect with FP64 storage
    a.step(40, L.DYNAMIC)
    b.step(40, L.DYNAMIC)
    np.testing.assert_allclose(a.read_populations(), b.read_populations(), rtol=0, atol=1e-14)
    for bad in (-1, 2):
        with pytest.raises(L.LbmibError) as e:
            b.set_option(L.OPT_IB_FP64, bad)
        assert e.value.status == L.ERR_ARG
