"""Zero-copy device views (lbmib_field_ptr): the population view, pulled by hand, gives the
populations the library reads back; the force view is the oracle's last spread force."""
import numpy as np
import pytest

import oracle as o
from paper_1903_03356_gb300 import workloads as W

pytestmark = pytest.mark.gpu

E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
Wt = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_03356_gb300 import lbmib
    return lbmib


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_population_view_pulls_to_the_read_back(L, storage):
    nx, ny = 53, 24
    rng = np.random.default_rng(4)
    ctx = L.Context(nx, ny, 0.8, False, storage=storage)
    ctx.init_fields(1 + 0.01 * rng.standard_normal((ny, nx)), 0.02 * rng.standard_normal((ny, nx)),
                    0.02 * rng.standard_normal((ny, nx)))
    ctx.step(7)
    v = ctx.field_view(L.FIELD_POPULATIONS).double().cpu().numpy()[:, :, :nx]
    pre = np.stack([np.roll(v[i], shift=(E[i][1], E[i][0]), axis=(0, 1)) + Wt[i] for i in range(9)])
    np.testing.assert_allclose(pre, ctx.read_populations(), rtol=0, atol=1e-15 if storage == "fp64" else 1e-7)


def test_force_view_is_the_last_spread(L):
    case = W.shear_capsule(nx=64, ny=64, radius=8.0, n=48, ca=1e-2, scheme=o.KINEMATIC)
    ctx = L.from_case(case, storage="fp64")
    ctx.step(5, L.KINEMATIC)
    s = o.Sim(o.lattice(case.nx, case.ny, case.tau, True, case.u_bottom, case.u_top))
    s.init_fields(*case.fields())
    c = case.capsules[0]
    s.add_capsule(c.xy, c.ks, c.kb, c.ka, c.mass)
    s.step(5, o.KINEMATIC)
    f = ctx.field_view(L.FIELD_FORCE).cpu().numpy()
    ref = s.force_field()
    assert np.abs(ref).max() > 0
    # the spread forces carry the rounding of five steps of positions (about 1e-10 relative)
    np.testing.assert_allclose(f, ref, rtol=1e-8, atol=1e-12 * np.abs(ref).max())
