"""Physics pins of the oracle's coupled step (small-deformation behaviour the paper reports):
the two coupling schemes agree on the deformation of a neutrally buoyant capsule in shear
(Section 3.1), and a capsule in Couette flow migrates towards the centre line (Section 3.5).
"""
import numpy as np

import oracle as o
from paper_1903_03356_gb300 import workloads as W


def run(case, scheme, T, every=None):
    s = o.Sim(o.lattice(case.nx, case.ny, case.tau, True, case.u_bottom, case.u_top))
    s.init_fields(*case.fields())
    c = case.capsules[0]
    s.add_capsule(c.xy, c.ks, c.kb, c.ka, c.mass)
    if every is None:
        assert s.step(T, scheme) == 0
        return s.observables(0)
    out = []
    for _ in range(T // every):
        assert s.step(every, scheme) == 0
        out.append(s.observables(0))
    return np.array(out)


def test_kinematic_and_dynamic_deformations_agree_at_density_ratio_one():
    # the 100 x 100 shear case at Ca = 0.01: Taylor D of the two schemes within 3 % after
    # 1000 steps (the paper: within about 1 % at rho_s / rho_f = 1; measured here 1.6 %)
    D = {}
    for scheme in (o.KINEMATIC, o.DYNAMIC):
        case = W.shear_capsule(nx=100, ny=100, ca=0.01, scheme=scheme)
        D[scheme] = run(case, scheme, 1000)[2]
    assert D[o.KINEMATIC] > 0.03
    assert abs(D[o.DYNAMIC] - D[o.KINEMATIC]) / D[o.KINEMATIC] < 0.03


def test_capsule_in_couette_flow_migrates_towards_the_centre_line():
    # started at 0.3 H, the centroid moves steadily towards 0.5 H
    case = W.shear_capsule(nx=80, ny=48, radius=6.0, n=40, ca=0.05, scheme=o.KINEMATIC, centre=(40.1, 14.37),
                           shear_rate=4e-4)
    obs = run(case, o.KINEMATIC, 6000, every=1500)
    yc = obs[:, 4]
    assert np.all(np.diff(yc) > 0)
    assert yc[-1] - 14.37 > 0.5 and yc[-1] < 0.5 * case.ny


def test_dynamic_capsules_in_couette_flow_migrate_towards_the_centre_line():
    # Section 3.5: in a linear (Couette) flow capsules of any membrane mass reach 0.5 H.
    # With the Dynamic scheme, density ratios 1 and 2, started at 0.3 H: the centroid rises
    # steadily over 6000 steps (after the start-up interval) and the heavier capsule lags.
    rise = {}
    for ratio in (1.0, 2.0):
        case = W.shear_capsule(nx=80, ny=48, radius=6.0, n=40, ca=0.05, scheme=o.DYNAMIC, centre=(40.1, 14.37),
                               shear_rate=4e-4, density_ratio=ratio)
        yc = run(case, o.DYNAMIC, 6000, every=1500)[:, 4]
        assert np.all(np.diff(yc) > 0)
        assert yc[-1] < 0.5 * case.ny
        rise[ratio] = yc[-1] - 14.37
    assert rise[1.0] > 0.2 and rise[2.0] > 0.15
    assert rise[2.0] < rise[1.0]
