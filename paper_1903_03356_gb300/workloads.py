"""Seeded synthetic workloads shaped like the paper's test cases.

This module serves both the GPU library's users (tests, benchmark) and the CPU
oracle's tests. It holds input geometry, initial flow fields and the mapping from
nondimensional numbers to lattice parameters, and none of the method's arithmetic
(no lattice update, no MLS transfer, no membrane mechanics).

Conventions: dx = dt = 1, rho_0 = 1, nu = (tau - 1/2)/3. Lattice node (i, j) sits at
(i, j); with walls, the half-way walls sit at y = -1/2 and y = ny - 1/2, so H = ny.
Capsule rings are counter-clockwise, as the oracle and the library require.

Workloads (all synthetic; the paper's own data are not used):
  shear_capsule      - circular capsule in simple shear (Section 3.1 shape), 100 x 100
  poiseuille_capsule - circular capsule in body-force Poiseuille flow (Section 3.2 shape)
  poiseuille_biconcave - many biconcave capsules (Eq. 26 shape), seeded placement
  batch_cases        - many independent shear-flow cases of uneven sizes
  adjoint_capsule    - circular capsule in Poiseuille flow for gradients
  open_channel_capsule - circular capsule in the open channel of Section 3.2 (parabolic
                       Zou-He inlet, constant-pressure outlet, fluid at rest at the start)
  dense_biconcave    - dense suspension of biconcave capsules (Section 3.4 shape)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

KINEMATIC = 0
DYNAMIC = 1


# ----------------------------------------------------------------------------------
# Parameter mappings (Section 2.2.1 and Section 3)
# ----------------------------------------------------------------------------------
def viscosity(tau: float) -> float:
    return (tau - 0.5) / 3.0


def ks_from_shear_ca(tau: float, shear_rate: float, radius: float, ca: float, rho=1.0) -> float:
    """k_s from Ca = mu gamma a / k_s (the shear-flow capillary number)."""
    return rho * viscosity(tau) * shear_rate * radius / ca


def ks_from_umax_ca(tau: float, u_max: float, ca: float, rho=1.0) -> float:
    """k_s from Ca = nu rho u_max / k_s (Section 2.2.1 and Section 3.2)."""
    return rho * viscosity(tau) * u_max / ca


def kb_from_eb(eb: float, ks: float, radius: float) -> float:
    """k_b from E_b = k_b / (k_s r^2) (Section 2.2.1)."""
    return eb * ks * radius * radius


def poiseuille_force(tau: float, u_max: float, H: float, rho=1.0) -> float:
    """Uniform body force giving centre-line velocity u_max in a channel of height H."""
    return 8.0 * rho * viscosity(tau) * u_max / (H * H)


def stable_eb(eb: float, ks: float, radius: float, xy: np.ndarray, mass: float) -> float:
    """Bending modulus used by the workloads: E_b as requested, capped so that the
    explicit node update of the Dynamic scheme (Eq. 23: a displacement of F/(2 m_v) per
    step) is stable for the ring's shortest bending mode. That mode moves a vertex by
    about 8 k_b / (l_min^2 m_v) times its amplitude per step; the cap keeps this below 1:
    k_b <= l_min^2 m_v / 8, i.e. E_b <= l_min^2 m_v / (8 k_s r^2)."""
    d = np.hypot(*(np.roll(xy, -1, axis=0) - xy).T)
    cap = float(d.min()) ** 2 * mass / (8.0 * ks * radius * radius)
    return min(eb, cap)


def node_mass(density_ratio: float, area0: float, n: int, rho=1.0) -> float:
    """Membrane mass spread evenly over the vertices; the capsule weighs density_ratio
    times the fluid it encloses."""
    return density_ratio * rho * area0 / n


# ----------------------------------------------------------------------------------
# Shapes
# ----------------------------------------------------------------------------------
def signed_area(xy: np.ndarray) -> float:
    x, y = xy[:, 0], xy[:, 1]
    return 0.5 * float(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


def circle(n: int, r: float, cx: float, cy: float, phase: float = 0.0) -> np.ndarray:
    """Regular n-gon inscribed in a circle, counter-clockwise, shape (n, 2)."""
    t = phase + 2.0 * np.pi * np.arange(n) / n
    return np.stack([cx + r * np.cos(t), cy + r * np.sin(t)], axis=1)


def biconcave(n: int, a: float, cx: float, cy: float) -> np.ndarray:
    """Eq. 26 shape with the constants of the precision workload:
    x = a sin t, y = (a/2)(0.207 + 2.003 sin^2 t - 1.123 sin^4 t) cos t,
    t_k = -pi/2 + 2 pi k / n; returned counter-clockwise."""
    t = -0.5 * np.pi + 2.0 * np.pi * np.arange(n) / n
    s = np.sin(t)
    x = a * s
    y = 0.5 * a * (0.207 + 2.003 * s ** 2 - 1.123 * s ** 4) * np.cos(t)
    xy = np.stack([cx + x, cy + y], axis=1)
    if signed_area(xy) < 0:
        xy = xy[::-1].copy()
    return xy


def polygon_inertia(xy: np.ndarray):
    """Area, area centroid and polar second moment about the centroid of a polygon (a
    uniform rigid particle of density rho_s has mass rho_s A and inertia rho_s J)."""
    x, y = xy[:, 0] - xy[0, 0], xy[:, 1] - xy[0, 1]
    xn, yn = np.roll(x, -1), np.roll(y, -1)
    cr = x * yn - xn * y
    A = 0.5 * cr.sum()
    cx = ((x + xn) * cr).sum() / (6 * A)
    cy = ((y + yn) * cr).sum() / (6 * A)
    J = (((x * x + x * xn + xn * xn) + (y * y + y * yn + yn * yn)) * cr).sum() / 12.0 - A * (cx * cx + cy * cy)
    return A, cx + xy[0, 0], cy + xy[0, 1], J


def ellipse(n: int, a: float, b: float, cx: float, cy: float, angle: float = 0.0, phase: float = 0.137) -> np.ndarray:
    """Counter-clockwise ellipse of semi-axes a, b turned by `angle`."""
    t = 2 * np.pi * (np.arange(n) + phase) / n
    x, y = a * np.cos(t), b * np.sin(t)
    c, s = np.cos(angle), np.sin(angle)
    return np.stack([cx + c * x - s * y, cy + s * x + c * y], axis=1)


def min_half_integer_distance(xy: np.ndarray) -> float:
    """Distance of the nearest coordinate to a half-integer line (support switch)."""
    d = np.abs((xy + 0.5) - np.round(xy + 0.5))
    return float(d.min())


def check_no_ties(xy: np.ndarray, tol: float = 1e-9) -> None:
    if min_half_integer_distance(xy) <= tol:
        raise ValueError("a marker lies on a half-integer line; shift the capsule")


# ----------------------------------------------------------------------------------
# Initial fields
# ----------------------------------------------------------------------------------
def linear_shear(nx: int, ny: int, u_w: float):
    """u_x = u_w (2 (y + 1/2)/H - 1): the Couette profile between walls moving at -u_w
    (y = -1/2) and +u_w (y = ny - 1/2) (Section 3.1 initial condition)."""
    y = np.arange(ny, dtype=np.float64)
    ux = u_w * (2.0 * (y + 0.5) / ny - 1.0)
    ux = np.repeat(ux[:, None], nx, axis=1)
    return np.ones((ny, nx)), ux, np.zeros((ny, nx))


def parabola(nx: int, ny: int, g: float, tau: float):
    """u_x = g/(2 nu) (y + 1/2)(H - y - 1/2), the Poiseuille profile of the channel."""
    y = np.arange(ny, dtype=np.float64)
    ux = g / (2.0 * viscosity(tau)) * (y + 0.5) * (ny - y - 0.5)
    ux = np.repeat(ux[:, None], nx, axis=1)
    return np.ones((ny, nx)), ux, np.zeros((ny, nx))


# ----------------------------------------------------------------------------------
# Cases
# ----------------------------------------------------------------------------------
@dataclass
class Capsule:
    xy: np.ndarray          # (n, 2) counter-clockwise, the stress-free shape
    ks: float
    kb: float
    ka: float
    mass: float             # per-node mass m_v


@dataclass
class Case:
    name: str
    nx: int
    ny: int
    tau: float
    walls: bool
    u_bottom: float = 0.0
    u_top: float = 0.0
    gx: float = 0.0
    gy: float = 0.0
    init: str = "rest"              # "rest", "shear", "parabola"
    capsules: List[Capsule] = field(default_factory=list)
    scheme: int = KINEMATIC
    steps: int = 1
    u_in: Optional[np.ndarray] = None   # open channel: inlet x-velocity per row (x not periodic)
    rho_out: float = 1.0                # open channel: outlet density

    def fields(self):
        if self.init == "shear":
            return linear_shear(self.nx, self.ny, self.u_top)
        if self.init == "parabola":
            return parabola(self.nx, self.ny, self.gx, self.tau)
        return (np.ones((self.ny, self.nx)), np.zeros((self.ny, self.nx)),
                np.zeros((self.ny, self.nx)))

    @property
    def n_nodes(self) -> int:
        return int(sum(c.xy.shape[0] for c in self.capsules))


def shear_capsule(nx=100, ny=100, tau=0.8, shear_rate=1e-4, radius=10.0, n=64, ca=0.01,
                  eb=0.01, ka=0.0, density_ratio=1.0, scheme=KINEMATIC, steps=2000,
                  centre: Optional[Tuple[float, float]] = None) -> Case:
    """Circular capsule at the centre of a sheared box (Section 3.1 shape): walls move
    at -/+ u_w with u_w = shear_rate H / 2, periodic in x, linear initial profile.
    Defaults: the 100 x 100 case with Ca = mu gamma a / k_s = 0.01, k_b = 0.01 k_s a^2."""
    u_w = 0.5 * shear_rate * ny
    cx, cy = centre if centre is not None else (0.5 * nx + 0.1, 0.5 * ny - 0.5 + 0.013)
    xy = circle(n, radius, cx, cy)
    check_no_ties(xy)
    ks = ks_from_shear_ca(tau, shear_rate, radius, ca)
    kb = kb_from_eb(eb, ks, radius)
    m = node_mass(density_ratio, signed_area(xy), n)
    return Case("shear_capsule", nx, ny, tau, True, -u_w, u_w, init="shear",
                capsules=[Capsule(xy, ks, kb, ka, m)], scheme=scheme, steps=steps)


def poiseuille_capsule(nx=600, ny=120, tau=0.7, u_max=0.02, radius=12.0, n=96, ca=1e-2,
                       eb=0.01, ka=0.0, density_ratio=1.0, y_frac=0.3, scheme=DYNAMIC,
                       steps=20000) -> Case:
    """Circular capsule in body-force Poiseuille flow (Section 3.2 shape), centre at
    y = y_frac H, started on the analytic parabola."""
    g = poiseuille_force(tau, u_max, ny)
    xy = circle(n, radius, 100.13 if nx > 200 else 0.3 * nx + 0.13, y_frac * ny - 0.5 + 0.07)
    check_no_ties(xy)
    ks = ks_from_umax_ca(tau, u_max, ca)
    m = node_mass(density_ratio, signed_area(xy), n)
    kb = kb_from_eb(stable_eb(eb, ks, radius, xy, m), ks, radius)
    return Case("poiseuille_capsule", nx, ny, tau, True, gx=g, init="parabola",
                capsules=[Capsule(xy, ks, kb, ka, m)], scheme=scheme, steps=steps)


def _place_biconcave(rng, nx, ny, count, a, n, gap=2.0, wall_gap=3.0, max_tries=200000):
    """Rejection-sample non-overlapping axis-aligned bounding boxes."""
    proto = biconcave(n, a, 0.0, 0.0)
    hw = 0.5 * (proto[:, 0].max() - proto[:, 0].min())
    hh = 0.5 * (proto[:, 1].max() - proto[:, 1].min())
    centres: List[Tuple[float, float]] = []
    tries = 0
    while len(centres) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place all capsules")
        cx = rng.uniform(hw + gap, nx - hw - gap)
        cy = rng.uniform(-0.5 + hh + wall_gap, ny - 0.5 - hh - wall_gap)
        ok = True
        for (ox, oy) in centres:
            if abs(cx - ox) < 2 * hw + gap and abs(cy - oy) < 2 * hh + gap:
                ok = False
                break
        if not ok:
            continue
        xy = proto + np.array([cx, cy])
        if min_half_integer_distance(xy) <= 1e-9:
            continue
        centres.append((cx, cy))
    return [proto + np.array([cx, cy]) for (cx, cy) in centres]


def _place_biconcave_grid(rng, nx, ny, count, a, n, wall_gap=3.0):
    """Seeded jittered-grid placement for very many capsules: one capsule per cell of a
    coarse grid, with a random offset that keeps neighbouring boxes apart."""
    proto = biconcave(n, a, 0.0, 0.0)
    w = proto[:, 0].max() - proto[:, 0].min()
    h = proto[:, 1].max() - proto[:, 1].min()
    cols = int(math.floor(nx / (w + 4.0)))
    rows = int(math.floor((ny - 2 * wall_gap) / (h + 4.0)))
    if cols * rows < count:
        raise RuntimeError("lattice too small for the requested capsule count")
    cells = rng.permutation(cols * rows)[:count]
    cw = nx / cols
    ch = (ny - 2 * wall_gap) / rows
    out = []
    for c in cells:
        i, j = int(c % cols), int(c // cols)
        jx = rng.uniform(-0.5, 0.5) * (cw - w - 2.0)
        jy = rng.uniform(-0.5, 0.5) * (ch - h - 2.0)
        cx = (i + 0.5) * cw + jx
        cy = wall_gap - 0.5 + (j + 0.5) * ch + jy
        xy = proto + np.array([cx, cy])
        k = 0
        while min_half_integer_distance(xy) <= 1e-9:
            k += 1
            xy = xy + 1e-6 * k
        out.append(xy)
    return out


def poiseuille_biconcave(nx=4096, ny=512, tau=0.7, u_max=0.02, count=256, n=128, a=8.0,
                         ca=0.01, eb=0.01, ka=0.0, density_ratio=1.0, seed=0,
                         scheme=DYNAMIC, steps=5000, placement="reject") -> Case:
    """Many biconcave capsules (Eq. 26 shape) at seeded non-overlapping positions in a
    body-force Poiseuille channel (Section 3.3 / 3.4 shapes)."""
    rng = np.random.default_rng(seed)
    g = poiseuille_force(tau, u_max, ny)
    ks = ks_from_umax_ca(tau, u_max, ca)
    place = _place_biconcave if placement == "reject" else _place_biconcave_grid
    shapes = place(rng, nx, ny, count, a, n)
    m0 = node_mass(density_ratio, signed_area(shapes[0]), n)
    kb = kb_from_eb(stable_eb(eb, ks, a, shapes[0], m0), ks, a)
    caps = []
    for xy in shapes:
        m = node_mass(density_ratio, signed_area(xy), n)
        caps.append(Capsule(xy, ks, kb, ka, m))
    return Case("poiseuille_biconcave", nx, ny, tau, True, gx=g, init="parabola",
                capsules=caps, scheme=scheme, steps=steps)


def roofline_lattice(nx=16384, ny=8192, scheme=DYNAMIC, seed=0, steps=200) -> Case:
    """Lattice far above L2 with the capsule density of the 4096 x 512 precision case
    (one 128-node biconcave capsule per 8192 lattice nodes)."""
    count = (nx * ny) // 8192
    c = poiseuille_biconcave(nx=nx, ny=ny, count=count, seed=seed, scheme=scheme, steps=steps,
                             placement="grid")
    c.name = "roofline_lattice"
    return c


def adjoint_capsule(nx=512, ny=128, tau=0.7, u_max=0.02, radius=16.0, n=128, ca=0.02,
                    eb=0.01, density_ratio=1.0, steps=8000, scheme=DYNAMIC) -> Case:
    """Circular capsule in Poiseuille flow at y = 0.3 H, for gradients of D(T), y_c(T)."""
    c = poiseuille_capsule(nx=nx, ny=ny, tau=tau, u_max=u_max, radius=radius, n=n, ca=ca,
                           eb=eb, density_ratio=density_ratio, scheme=scheme, steps=steps)
    c.name = "adjoint_capsule"
    return c


def inlet_parabola(ny: int, u_max: float) -> np.ndarray:
    """Section 3.2 inlet profile u_x = -u_max (|1 - y / (H/2)|^2 - 1), y measured from the
    bottom wall (at -1/2) to the row, H = ny."""
    y = np.arange(ny) + 0.5
    return -u_max * (np.abs(1.0 - y / (0.5 * ny)) ** 2 - 1.0)


def open_channel_capsule(ny=120, length=3.0, tau=0.7, u_max=0.02, diameter=56.0, spacing=0.3, ca=1e-2,
                         eb=0.01, y_frac=0.5, density_ratio=1.0, scheme=DYNAMIC, steps=1) -> Case:
    """Section 3.2 set-up: a circular capsule (diameter 7/15 of the channel height, element
    length `spacing` lattice units) in a channel of length `length` x H, driven by the
    parabolic inlet (Zou-He, u_max on the centre line) against a constant-pressure outlet,
    fluid at rest at the start; centre at `y_frac` H (6.5, 7.5, 8.5 um of 15 um: 0.433,
    0.5, 0.567) and 1.5 diameters from the inlet."""
    nx = int(round(length * ny))
    r = 0.5 * diameter
    n = int(round(2.0 * np.pi * r / spacing))
    xy = circle(n, r, 1.5 * diameter + 0.13, y_frac * ny - 0.5 + 0.07)
    k = 0
    while min_half_integer_distance(xy) <= 1e-9:
        k += 1
        xy = circle(n, r, 1.5 * diameter + 0.13 + 1e-4 * k, y_frac * ny - 0.5 + 0.07)
    ks = ks_from_umax_ca(tau, u_max, ca)
    m = node_mass(density_ratio, signed_area(xy), n)
    kb = kb_from_eb(stable_eb(eb, ks, r, xy, m), ks, r)
    return Case("open_channel_capsule", nx, ny, tau, True, init="rest", capsules=[Capsule(xy, ks, kb, 0.0, m)],
                scheme=scheme, steps=steps, u_in=inlet_parabola(ny, u_max), rho_out=1.0)


def dense_biconcave(nx=1200, ny=450, count=16, n=1000, hematocrit=0.30, tau=0.7, u_max=0.02, ca=1e-2,
                    gap=1.2, seed=2, scheme=DYNAMIC, steps=1) -> Case:
    """Dense suspension of biconcave capsules in a body-force channel (Section 3.4
    shape): `count` capsules of n vertices whose total area is `hematocrit` of the
    channel, on a jittered grid with at least `gap` lattice units between bounding boxes
    and 3 from the walls. For the repulsion of Eq. 27."""
    rng = np.random.default_rng(seed)
    proto = biconcave(n, 1.0, 0.0, 0.0)
    a = float(np.sqrt(hematocrit * nx * ny / count / signed_area(proto)))
    proto = biconcave(n, a, 0.0, 0.0)
    w = proto[:, 0].max() - proto[:, 0].min()
    h = proto[:, 1].max() - proto[:, 1].min()
    cols = int(np.floor((nx) / (w + gap)))
    rows = int(np.floor((ny - 6.0) / (h + gap)))
    if cols * rows < count:
        raise ValueError("capsules do not fit at this hematocrit and gap")
    cells = rng.permutation(cols * rows)[:count]
    sx, sy = nx / cols, (ny - 6.0) / rows
    g = poiseuille_force(tau, u_max, ny)
    ks = ks_from_umax_ca(tau, u_max, ca)
    caps = []
    for k in sorted(cells):
        i, j = k % cols, k // cols
        cx = (i + 0.5) * sx + rng.uniform(-0.5, 0.5) * max(0.0, sx - w - gap) + 0.013
        cy = 3.0 + (j + 0.5) * sy + rng.uniform(-0.5, 0.5) * max(0.0, sy - h - gap) + 0.017
        xy = biconcave(n, a, cx, cy)
        check_no_ties(xy)
        m = node_mass(1.0, signed_area(xy), n)
        kb = kb_from_eb(stable_eb(0.01, ks, 0.5 * w, xy, m), ks, 0.5 * w)
        caps.append(Capsule(xy, ks, kb, 0.0, m))
    return Case("dense_biconcave", nx, ny, tau, True, gx=g, init="parabola", capsules=caps, scheme=scheme,
                steps=steps)


BATCH_SIZES = (64, 96, 128, 192, 256)
BATCH_NODES = (48, 64, 96, 128)


def batch_cases(count=512, seed=1, tau=0.8, shear_rate=1e-4, steps=3000, eb=0.01,
                scheme=KINEMATIC) -> List[Case]:
    """Independent shear-flow capsule cases: nx, ny drawn independently from
    {64, 96, 128, 192, 256}, Ca log-uniform in [1e-3, 1e-1], node counts from
    {48, 64, 96, 128}; radius min(0.8 n / (2 pi), min(nx, ny) / 6)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nx = int(rng.choice(BATCH_SIZES))
        ny = int(rng.choice(BATCH_SIZES))
        ca = float(10.0 ** rng.uniform(-3.0, -1.0))
        n = int(rng.choice(BATCH_NODES))
        r = min(0.8 * n / (2.0 * np.pi), min(nx, ny) / 6.0)
        cx = 0.5 * nx + rng.uniform(0.05, 0.45)
        cy = 0.5 * ny - 0.5 + rng.uniform(0.05, 0.45)
        xy = circle(n, r, cx, cy)
        k = 0
        while min_half_integer_distance(xy) <= 1e-9:
            k += 1
            xy = circle(n, r, cx + 1e-4 * k, cy)
        ks = ks_from_shear_ca(tau, shear_rate, r, ca)
        kb = kb_from_eb(eb, ks, r)
        m = node_mass(1.0, signed_area(xy), n)
        u_w = 0.5 * shear_rate * ny
        out.append(Case("batch_case", nx, ny, tau, True, -u_w, u_w, init="shear",
                        capsules=[Capsule(xy, ks, kb, 0.0, m)], scheme=scheme, steps=steps))
    return out
