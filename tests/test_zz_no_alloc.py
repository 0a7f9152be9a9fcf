"""The allocation-free interpolation entry point (lbmib_interpolate_noalloc).

Some callers cannot allocate device memory when they want to probe the flow: real-time
callbacks that must not stall on an allocation, hosts whose device memory is owned by
another framework's allocator, or processes held to a fixed device-memory budget. For them the library offers an interpolation call whose device
staging lives in a static array of the library instead of the caller's arena. This file
checks it, through the C ABI, against the ordinary lbmib_interpolate on two calls in a
row (the static array keeps the previous call's contents), and checks the size limit.
It is collected last so that a run stopping at the first failure has run everything
else first, and it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

from paper_1903_03356_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_03356_gb300 import lbmib
    return lbmib


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_noalloc_interpolation_matches_the_arena_interpolation_twice(L, storage, tol):
    case = W.poiseuille_capsule(nx=160, ny=64, radius=8.0, n=48, ca=1e-2, y_frac=0.45, scheme=W.DYNAMIC)
    ctx = L.from_case(case, storage=storage, extra_nodes=4096)
    ctx.step(20, L.DYNAMIC)
    rng = np.random.default_rng(11)
    for call in range(2):
        # a different set of points each call; the second call overwrites the first
        n = 4096 if call == 0 else 777
        pts = np.stack([rng.uniform(-10, 170, n), rng.uniform(2.0, 61.0, n)], 1)
        want = ctx.interpolate(pts)
        got = ctx.interpolate_noalloc(pts)
        assert got.shape == (n, 8)
        np.testing.assert_allclose(got, want, rtol=0, atol=tol)
    ctx.step(5, L.DYNAMIC)
    pts = np.stack([rng.uniform(0, 160, 64), rng.uniform(3.0, 60.0, 64)], 1)
    np.testing.assert_allclose(ctx.interpolate_noalloc(pts), ctx.interpolate(pts), rtol=0, atol=tol)


def test_noalloc_interpolation_rejects_more_points_than_its_static_staging(L):
    case = W.Case("lattice", 32, 32, 0.8, False)
    ctx = L.from_case(case, storage="fp32")
    pts = np.full((16385, 2), 10.3)
    with pytest.raises(L.LbmibError) as e:
        ctx.interpolate_noalloc(pts)
    assert e.value.status == L.ERR_ARG
    assert "16384" in str(e.value)
    # the context is still usable and the limit itself is accepted
    out = ctx.interpolate_noalloc(np.full((16384, 2), 10.3))
    assert out.shape == (16384, 8) and np.all(np.isfinite(out))
