"""Parity at the benchmark's full size, in its launch configuration, on sampled outputs.

The benchmark's workload (16384 x 8192 Poiseuille channel, 16384 biconcave capsules of
128 vertices, Dynamic scheme, the default launch shape: one CTA per capsule, each node
update fused with the next step's force and spread inside one step call) runs T steps
on the GPU from its analytic initial state. The oracle cannot run that lattice, but a
lattice update moves information by one node per step and a capsule touches the fluid
only through its supports and probes (three nodes beyond its box): so for a capsule with
no neighbour nearby and away from the walls, the oracle run on a periodic window around
it, started from the same initial state, must agree with the full-size run on the
capsule and on the window's interior (the window's edges, whose wrap is not the
channel's, spoil one node per step).
"""
import numpy as np
import pytest

import oracle as o
from paper_1903_03356_gb300 import workloads as W

pytestmark = pytest.mark.gpu

T = 5            # steps, in one call
MARGIN = 12      # window margin around a capsule's box (supports, probes and T steps of travel)


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_03356_gb300 import lbmib
    return lbmib


@pytest.fixture(scope="module")
def case():
    return W.roofline_lattice(nx=16384, ny=8192, steps=T)


def isolated_capsules(case, count=6, seed=5):
    """Capsules whose box, widened by 2 MARGIN, meets no other capsule's box (whose own
    influence, its supports plus T steps of travel, then stays outside the window) and
    whose window stays inside the channel (walls and the x ends)."""
    boxes = np.array([[c.xy[:, 0].min(), c.xy[:, 1].min(), c.xy[:, 0].max(), c.xy[:, 1].max()]
                      for c in case.capsules])
    lo, hi = boxes[:, :2] - MARGIN, boxes[:, 2:] + MARGIN
    inside = (lo[:, 0] > 2) & (lo[:, 1] > 2) & (hi[:, 0] < case.nx - 3) & (hi[:, 1] < case.ny - 3)
    rng = np.random.default_rng(seed)
    picks = []
    for k in rng.permutation(len(case.capsules)):
        if not inside[k]:
            continue
        others = np.delete(np.arange(len(boxes)), k)
        b = boxes[others]
        far_lo, far_hi = lo[k] - MARGIN, hi[k] + MARGIN
        overlap = ((b[:, 2] >= far_lo[0]) & (b[:, 0] <= far_hi[0]) & (b[:, 3] >= far_lo[1]) & (b[:, 1] <= far_hi[1]))
        if not overlap.any():
            picks.append(int(k))
        if len(picks) == count:
            break
    return picks, boxes


def window_run(case, k, boxes, ux0):
    """The oracle on the periodic window around capsule k: (x0, y0, fields, capsule)."""
    x0, y0 = int(np.floor(boxes[k, 0])) - MARGIN, int(np.floor(boxes[k, 1])) - MARGIN
    x1, y1 = int(np.ceil(boxes[k, 2])) + MARGIN, int(np.ceil(boxes[k, 3])) + MARGIN
    nx, ny = x1 - x0 + 1, y1 - y0 + 1
    s = o.Sim(o.lattice(nx, ny, case.tau, False, gx=case.gx))
    s.init_fields(np.ones((ny, nx)), np.repeat(ux0[y0:y1 + 1, None], nx, axis=1), np.zeros((ny, nx)))
    c = case.capsules[k]
    s.add_capsule(c.xy - np.array([x0, y0]), c.ks, c.kb, c.ka, c.mass)
    assert s.step(T, o.DYNAMIC) == 0
    _, ux, uy = s.read_fields()
    xy = s.read_capsule(0)[0].reshape(-1, 2) + np.array([x0, y0])
    return x0, y0, np.stack([ux, uy]), xy, s.observables(0)[2]


@pytest.mark.parametrize("storage,tol_u,tol_x", [("fp32", 1e-5, 1e-6), ("fp64", 1e-10, 1e-11)])
def test_benchmark_workload_matches_oracle_windows(L, case, storage, tol_u, tol_x):
    ctx = L.from_case(case, storage=storage)
    ctx.step(T, L.DYNAMIC)
    _, gu, gv = ctx.read_fields()
    ux0 = W.parabola(1, case.ny, case.gx, case.tau)[1][:, 0]
    umax = np.abs(ux0).max()
    picks, boxes = isolated_capsules(case)
    assert len(picks) == 6
    worst_u = worst_x = worst_d = 0.0
    for k in picks:
        x0, y0, vel, xy, D = window_run(case, k, boxes, ux0)
        ny, nx = vel.shape[1:]
        e = T + 2   # interior: the wrap of the window's edges has not reached it
        got = np.stack([gu[y0 + e:y0 + ny - e, x0 + e:x0 + nx - e], gv[y0 + e:y0 + ny - e, x0 + e:x0 + nx - e]])
        want = vel[:, e:ny - e, e:nx - e]
        worst_u = max(worst_u, np.abs(got - want).max() / umax)
        worst_x = max(worst_x, np.abs(ctx.read_capsule(k)[0].reshape(-1, 2) - xy).max())
        worst_d = max(worst_d, abs(ctx.observables(k)[2] - D))
    print(f"{storage} 16384 x 8192, {len(case.capsules)} capsules, {T} steps, {len(picks)} windows: "
          f"velocity {worst_u:.2e} of u_max, positions {worst_x:.2e}, D {worst_d:.2e}")
    assert worst_u < tol_u
    assert worst_x < tol_x
    assert worst_d < (1e-4 if storage == "fp32" else 1e-12)
    ctx.close()
