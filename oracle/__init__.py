"""ctypes front-end of the FP64 CPU oracle (``lbmib_oracle.c``).

Test infrastructure only: the test-suite, the smoke check and the CPU-baseline leg
of ``bench.py`` import this module. The GPU library never does, and this module
imports nothing from the GPU package.

Every function states the equation of Coclite et al. (arXiv:1903.03356) that it
evaluates; the C source carries the readings of the paper that the oracle takes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbmib_oracle.c")
_LIB = os.path.join(_HERE, "liblbmib_oracle.so")
_LIB_OMP = os.path.join(_HERE, "liblbmib_oracle_omp.so")

CFLAGS = ["-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE"]

# LBMIB_ORACLE_OPENMP=1 loads the all-core build: the same source compiled with -fopenmp,
# whose lattice loop runs its rows on every host core (identical results). Only the
# timed CPU baseline uses it.
OPENMP = os.environ.get("LBMIB_ORACLE_OPENMP", "0") == "1"


def build_library(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no FMA contraction) if it is stale."""
    out = _LIB_OMP if openmp else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        flags = CFLAGS + (["-fopenmp"] if openmp else [])
        subprocess.check_call(["gcc", *flags, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, out)
    return out


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build_library(openmp=OPENMP))
        _declare(_lib)
    return _lib


class Lattice(C.Structure):
    """Lattice description: size, y-boundary, wall velocities, tau, body force."""

    _fields_ = [
        ("nx", C.c_int),
        ("ny", C.c_int),
        ("walls", C.c_int),
        ("u_bottom", C.c_double),
        ("u_top", C.c_double),
        ("tau", C.c_double),
        ("gx", C.c_double),
        ("gy", C.c_double),
        ("inflow", C.c_int),
        ("rho_out", C.c_double),
        ("u_in", C.POINTER(C.c_double)),
    ]

    @property
    def N(self) -> int:
        return self.nx * self.ny


def lattice(nx, ny, tau, walls=False, u_bottom=0.0, u_top=0.0, gx=0.0, gy=0.0, u_in=None,
            rho_out=1.0) -> Lattice:
    """Lattice description. With u_in (ny inlet x-velocities) x is an open channel: a
    known-velocity inlet at x = 0 and a known-density (rho_out) outlet at x = nx - 1
    (reading R26); otherwise x is periodic."""
    L = Lattice(int(nx), int(ny), int(bool(walls)), float(u_bottom), float(u_top),
                float(tau), float(gx), float(gy), 0, float(rho_out), None)
    if u_in is not None:
        u = np.ascontiguousarray(np.asarray(u_in, dtype=np.float64).reshape(-1))
        if u.size != int(ny):
            raise ValueError("u_in needs one value per row")
        L._u_in = u                      # keeps the profile alive while the lattice is used
        L.inflow = 1
        L.u_in = u.ctypes.data_as(C.POINTER(C.c_double))
    return L


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_LP = C.POINTER(Lattice)


def _declare(L):
    vp = C.c_void_p
    sig = {
        "orc_feq": (None, [C.c_double, C.c_double, C.c_double, _dp]),
        "orc_macros": (None, [_LP, _dp, vp, _dp, _dp, _dp]),
        "orc_collide_stream": (None, [_LP, _dp, vp, _dp]),
        "orc_init_equilibrium": (None, [_LP, vp, vp, vp, _dp]),
        "orc_open_boundaries": (None, [_LP, _dp]),
        "orc_mls": (C.c_int, [_LP, C.c_double, C.c_double, _ip, _ip, _dp, _dp, _dp]),
        "orc_interp": (C.c_int, [_LP, _dp, vp, C.c_double, C.c_double, _dp]),
        "orc_interp_scalar": (C.c_int, [_LP, _dp, C.c_double, C.c_double, _dp]),
        "orc_spread": (C.c_int, [_LP, C.c_double, C.c_double, C.c_double, C.c_double,
                                 C.c_double, _dp]),
        "orc_tractions": (C.c_int, [_LP, _dp, vp, _dp, C.c_int, _dp]),
        "orc_area": (C.c_double, [_dp, C.c_int]),
        "orc_perimeter": (C.c_double, [_dp, C.c_int]),
        "orc_membrane_reference": (None, [_dp, C.c_int, _dp, _dp, _dp]),
        "orc_membrane_energy": (C.c_double, [_dp, C.c_int, _dp, _dp, C.c_double, C.c_double,
                                             C.c_double, C.c_double]),
        "orc_membrane_force": (None, [_dp, C.c_int, _dp, _dp, C.c_double, C.c_double,
                                      C.c_double, C.c_double, _dp]),
        "orc_observables": (None, [_dp, C.c_int, _dp]),
        "orc_kinematic_advance": (None, [C.c_int, _dp, _dp, _dp, C.c_int, _dp]),
        "orc_dynamic_advance": (None, [C.c_int, _dp, _dp, _dp, _dp, C.c_double, _dp, _dp]),
        "orc_sim_create": (vp, [_LP]),
        "orc_sim_destroy": (None, [vp]),
        "orc_sim_init_fields": (None, [vp, vp, vp, vp]),
        "orc_sim_populations": (C.POINTER(C.c_double), [vp]),
        "orc_sim_force_field": (C.POINTER(C.c_double), [vp]),
        "orc_sim_add_capsule": (C.c_int, [vp, _dp, C.c_int, C.c_double, C.c_double, C.c_double,
                                          C.c_double]),
        "orc_sim_step": (C.c_int, [vp, C.c_longlong, C.c_int]),
        "orc_sim_set_capsule_positions": (C.c_int, [vp, C.c_int, _dp]),
        "orc_sim_read_fields": (None, [vp, _dp, _dp, _dp]),
        "orc_sim_read_capsule": (C.c_int, [vp, C.c_int, vp, vp, vp, vp]),
        "orc_sim_observables": (C.c_int, [vp, C.c_int, _dp]),
        "orc_sim_step_count": (C.c_longlong, [vp]),
        "orc_vertex_normal": (None, [_dp, C.c_int, C.c_int, _dp]),
        "orc_repulsion": (None, [C.POINTER(C.POINTER(C.c_double)), _ip, C.c_int, C.c_double, C.c_double,
                                 C.c_double, C.c_double, C.POINTER(C.POINTER(C.c_double))]),
        "orc_sim_set_repulsion": (None, [vp, C.c_double, C.c_double]),
        "orc_sim_read_repulsion": (C.c_int, [vp, C.c_int, _dp]),
        "orc_sim_add_rigid": (C.c_int, [vp, _dp, C.c_int, C.c_double, C.c_double]),
        "orc_sim_read_rigid": (C.c_int, [vp, C.c_int, _dp]),
        "orc_rigid_load": (C.c_int, [_LP, _dp, vp, _dp, C.c_int, C.c_double, C.c_double, _dp, vp]),
        "orc_rigid_advance": (None, [_dp, _dp, _dp, C.c_double, C.c_double]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------------------------
# Lattice Boltzmann (Section 2.1, Eq. 1-7)
# ----------------------------------------------------------------------------------
def feq(rho: float, ux: float, uy: float) -> np.ndarray:
    """Eq. 2 equilibrium populations at one node."""
    out = np.zeros(9)
    lib().orc_feq(rho, ux, uy, out)
    return out


def init_equilibrium(L: Lattice, rho=None, ux=None, uy=None) -> np.ndarray:
    """Populations (9, ny, nx) at the Eq. 2 equilibrium of the given fields."""
    f = np.zeros((9, L.ny, L.nx))
    args = [None if a is None else _f64(a) for a in (rho, ux, uy)]
    lib().orc_init_equilibrium(C.byref(L), *[_ptr(a) for a in args], f)
    return f


def macros(L: Lattice, f: np.ndarray, fib: Optional[np.ndarray] = None):
    """Eq. 6-7: density and velocity with half of the total body force."""
    rho = np.zeros((L.ny, L.nx)); ux = np.zeros_like(rho); uy = np.zeros_like(rho)
    fib = None if fib is None else _f64(fib)
    lib().orc_macros(C.byref(L), _f64(f), _ptr(fib), rho, ux, uy)
    return rho, ux, uy


def collide_stream(L: Lattice, f: np.ndarray, fib: Optional[np.ndarray] = None) -> np.ndarray:
    """Eq. 4-5: one forced BGK collision plus streaming with bounce-back walls."""
    out = np.zeros((9, L.ny, L.nx))
    fib = None if fib is None else _f64(fib)
    lib().orc_collide_stream(C.byref(L), _f64(f), _ptr(fib), out)
    return out


def open_boundaries(L: Lattice, f: np.ndarray) -> np.ndarray:
    """Zou-He closure of the inlet and outlet columns (reading R26) applied to a copy of
    the pre-collision populations f (9, ny, nx); f itself is unchanged."""
    out = _f64(f).copy()
    lib().orc_open_boundaries(C.byref(L), out)
    return out


# ----------------------------------------------------------------------------------
# MLS transfer (Eq. 8-9)
# ----------------------------------------------------------------------------------
def mls(L: Lattice, X: float, Y: float):
    """Shape functions phi_k and gradient weights at (X, Y): (ix, iy, phi, gx, gy, status)."""
    ix = np.zeros(9, np.int32); iy = np.zeros(9, np.int32)
    phi = np.zeros(9); gx = np.zeros(9); gy = np.zeros(9)
    st = lib().orc_mls(C.byref(L), float(X), float(Y), ix, iy, phi, gx, gy)
    return ix, iy, phi, gx, gy, st


def interp(L: Lattice, f: np.ndarray, fib: Optional[np.ndarray], X: float, Y: float):
    """Eq. 8 at (X, Y): (ux, uy, rho, p, dux/dx, dux/dy, duy/dx, duy/dy), status."""
    out = np.zeros(8)
    fib = None if fib is None else _f64(fib)
    st = lib().orc_interp(C.byref(L), _f64(f), _ptr(fib), float(X), float(Y), out)
    return out, st


def interp_scalar(L: Lattice, v: np.ndarray, X: float, Y: float) -> Tuple[float, int]:
    out = np.zeros(1)
    st = lib().orc_interp_scalar(C.byref(L), _f64(v), float(X), float(Y), out)
    return float(out[0]), st


def spread(L: Lattice, X, Y, Fx, Fy, c, fib: np.ndarray) -> int:
    """Step 3 / step iii: fib (2, ny, nx) += c phi_k F at the marker's support."""
    assert fib.dtype == np.float64 and fib.flags.c_contiguous
    return lib().orc_spread(C.byref(L), float(X), float(Y), float(Fx), float(Fy), float(c), fib)


def tractions(L: Lattice, f: np.ndarray, fib: Optional[np.ndarray], xy: np.ndarray):
    """Eq. 15-16 nodal shares of the element tractions of a ring: (Fext (n, 2), status)."""
    xy = _f64(xy).reshape(-1)
    out = np.zeros_like(xy)
    fib = None if fib is None else _f64(fib)
    st = lib().orc_tractions(C.byref(L), _f64(f), _ptr(fib), xy, xy.size // 2, out)
    return out.reshape(-1, 2), st


# ----------------------------------------------------------------------------------
# Membrane (Eq. 10-14) and observables
# ----------------------------------------------------------------------------------
def area(xy: np.ndarray) -> float:
    xy = _f64(xy); return lib().orc_area(xy, xy.size // 2)


def perimeter(xy: np.ndarray) -> float:
    xy = _f64(xy); return lib().orc_perimeter(xy, xy.size // 2)


def membrane_reference(xy: np.ndarray):
    xy = _f64(xy); n = xy.size // 2
    L0 = np.zeros(n); th0 = np.zeros(n); A0 = np.zeros(1)
    lib().orc_membrane_reference(xy, n, L0, th0, A0)
    return L0, th0, float(A0[0])


def membrane_energy(xy, L0, th0, A0, ks, kb, ka) -> float:
    xy = _f64(xy)
    return lib().orc_membrane_energy(xy, xy.size // 2, _f64(L0), _f64(th0), A0, ks, kb, ka)


def membrane_force(xy, L0, th0, A0, ks, kb, ka) -> np.ndarray:
    xy = _f64(xy); F = np.zeros_like(xy)
    lib().orc_membrane_force(xy, xy.size // 2, _f64(L0), _f64(th0), A0, ks, kb, ka, F)
    return F


def observables(xy: np.ndarray) -> np.ndarray:
    """(area, perimeter, D, xc, yc, Sw, inclination, lambda_max)."""
    xy = _f64(xy); out = np.zeros(8)
    lib().orc_observables(xy, xy.size // 2, out)
    return out


def kinematic_advance(X, Xm1, xdot, first: bool) -> np.ndarray:
    """Eq. 25 (forward Euler when first)."""
    X = _f64(X); out = np.zeros_like(X)
    lib().orc_kinematic_advance(X.size, X, _f64(Xm1), _f64(xdot), int(first), out)
    return out


def dynamic_advance(X, Xm1, xdot0, Ftot, m):
    """Eq. 23-24: (X^{n+1}, u_v^{n+1})."""
    X = _f64(X); Xn = np.zeros_like(X); uv = np.zeros_like(X)
    lib().orc_dynamic_advance(X.size, X, _f64(Xm1), _f64(xdot0), _f64(Ftot), float(m), Xn, uv)
    return Xn, uv


def rigid_load(L: Lattice, f: np.ndarray, fib: Optional[np.ndarray], xy, cx: float, cy: float):
    """Eq. 17-18 load on a rigid ring about (cx, cy): ((F_x, F_y, M), status)."""
    xy = _f64(xy).reshape(-1)
    out = np.zeros(3)
    fib = None if fib is None else _f64(fib)
    st = lib().orc_rigid_load(C.byref(L), _f64(f), _ptr(fib), xy, xy.size // 2, float(cx), float(cy), out, None)
    return out, st


def rigid_advance(body, prev, load, mass: float, inertia: float):
    """Eq. 19-20 (reading R29) on body = (c_x, c_y, theta, u_x, u_y, omega) at n and prev at
    n - 1: returns (body at n + 1, body at n)."""
    b = _f64(body).copy(); p = _f64(prev).copy()
    lib().orc_rigid_advance(b, p, _f64(load), float(mass), float(inertia))
    return b, p


# ----------------------------------------------------------------------------------
# Whole simulation
# ----------------------------------------------------------------------------------
KINEMATIC = 0
DYNAMIC = 1


# Eq. 27 coefficient: 1e-4 / (8 sqrt 2) with dx = 1
REPULSION_COEFF = 1e-4 / (8.0 * np.sqrt(2.0))


def vertex_normal(xy: np.ndarray, v: int) -> np.ndarray:
    """Outward unit normal at vertex v of a counter-clockwise ring (reading R24)."""
    xy = _f64(xy); out = np.zeros(2)
    lib().orc_vertex_normal(xy, xy.size // 2, v, out)
    return out


def repulsion(rings, rc: float, coeff: float = REPULSION_COEFF, px: float = 0.0, py: float = 0.0):
    """Eq. 27 forces on every vertex of every ring (list of (n, 2) arrays); periods px,
    py (0: none) for minimum-image distances. Returns a list of (n, 2) arrays."""
    rings = [_f64(r).reshape(-1) for r in rings]
    k = len(rings)
    out = [np.zeros_like(r) for r in rings]
    dpp = C.POINTER(C.c_double)
    Xp = (dpp * k)(*[r.ctypes.data_as(dpp) for r in rings])
    Fp = (dpp * k)(*[f.ctypes.data_as(dpp) for f in out])
    n = np.array([r.size // 2 for r in rings], dtype=np.int32)
    lib().orc_repulsion(Xp, n, k, rc, coeff, px, py, Fp)
    return [f.reshape(-1, 2) for f in out]


class Sim:
    """Lattice plus capsules stepped with the Kinematic (Section 2.4) or Dynamic
    (Section 2.3) scheme."""

    def __init__(self, L: Lattice):
        self.L = L
        self._h = lib().orc_sim_create(C.byref(L))
        self._n = []

    def close(self):
        if self._h:
            lib().orc_sim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_fields(self, rho=None, ux=None, uy=None):
        args = [None if a is None else _f64(a) for a in (rho, ux, uy)]
        self._keep = args
        lib().orc_sim_init_fields(self._h, *[_ptr(a) for a in args])

    def add_capsule(self, xy, ks, kb, ka, mass) -> int:
        xy = _f64(xy).reshape(-1)
        n = xy.size // 2
        cid = lib().orc_sim_add_capsule(self._h, xy, n, ks, kb, ka, mass)
        self._n.append(n)
        return cid

    def set_positions(self, cid: int, xy):
        """Start capsule cid at positions xy (its stress-free shape is unchanged)."""
        lib().orc_sim_set_capsule_positions(self._h, cid, _f64(xy).reshape(-1))

    def step(self, n: int, scheme: int) -> int:
        return lib().orc_sim_step(self._h, int(n), int(scheme))

    @property
    def step_count(self) -> int:
        return lib().orc_sim_step_count(self._h)

    def populations(self) -> np.ndarray:
        p = lib().orc_sim_populations(self._h)
        return np.ctypeslib.as_array(p, shape=(9, self.L.ny, self.L.nx)).copy()

    def set_populations(self, f: np.ndarray):
        p = lib().orc_sim_populations(self._h)
        np.ctypeslib.as_array(p, shape=(9, self.L.ny, self.L.nx))[...] = f

    def force_field(self) -> np.ndarray:
        p = lib().orc_sim_force_field(self._h)
        return np.ctypeslib.as_array(p, shape=(2, self.L.ny, self.L.nx)).copy()

    def read_fields(self):
        rho = np.zeros((self.L.ny, self.L.nx)); ux = np.zeros_like(rho); uy = np.zeros_like(rho)
        lib().orc_sim_read_fields(self._h, rho, ux, uy)
        return rho, ux, uy

    def read_capsule(self, cid: int):
        n = self._n[cid]
        xy = np.zeros(2 * n); vel = np.zeros(2 * n); fi = np.zeros(2 * n); fe = np.zeros(2 * n)
        lib().orc_sim_read_capsule(self._h, cid, _ptr(xy), _ptr(vel), _ptr(fi), _ptr(fe))
        return xy, vel, fi, fe

    def set_repulsion(self, rc: float, coeff: float = REPULSION_COEFF):
        """Capsule-capsule repulsion (Eq. 27) with cut-off rc (0: off)."""
        lib().orc_sim_set_repulsion(self._h, rc, coeff)

    def add_rigid(self, xy, mass, inertia) -> int:
        """Rigid particle (readings R27-R30) with its ring, mass and moment of inertia about
        the area centroid; at rest. Dynamic scheme only."""
        xy = _f64(xy).reshape(-1)
        n = xy.size // 2
        cid = lib().orc_sim_add_rigid(self._h, xy, n, float(mass), float(inertia))
        self._n.append(n)
        return cid

    def read_rigid(self, cid: int) -> np.ndarray:
        """(c_x, c_y, theta, u_x, u_y, omega, F_x, F_y, M) of rigid particle cid."""
        out = np.zeros(9)
        if lib().orc_sim_read_rigid(self._h, cid, out):
            raise ValueError("not a rigid particle")
        return out

    def read_repulsion(self, cid: int) -> np.ndarray:
        out = np.zeros(2 * self._n[cid])
        lib().orc_sim_read_repulsion(self._h, cid, out)
        return out

    def observables(self, cid: int) -> np.ndarray:
        """(area, perimeter, D, xc, yc, Sw, inclination, delta_p)."""
        out = np.zeros(8)
        lib().orc_sim_observables(self._h, cid, out)
        return out
