"""Python binding of the C ABI in ``include/lbmib.h`` (argument marshalling only).

Every step of the method runs in the CUDA library ``liblbmib.so``; this module only
converts numpy arrays to host pointers, allocates the library's device arena with
torch, and passes torch's current CUDA stream. There is no CPU fallback: if the
library has not been built, importing this module raises ``ImportError``.

Functions with the C names (``lbmib_create``, ``lbmib_step`` ...) mirror the ABI one to
one; ``Context`` wraps them for convenience.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbmib.so")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_UNSTABLE, ERR_SUPPORT, ERR_TIMEOUT, ERR_STATE = range(8)
FP64, FP32, FP16 = 0, 1, 2
KINEMATIC, DYNAMIC = 0, 1
OPT_GRAPHS, OPT_TIMING, OPT_GRAPH_STEPS, OPT_FP16_SCALE, OPT_LATTICE_VARIANT, OPT_OVERLAP, OPT_ARCS, OPT_FUSE_IB, \
    OPT_IB_FP64 = 1, 2, 3, 4, 5, 6, 7, 8, 9
FIELD_POPULATIONS, FIELD_FORCE = 0, 1
OBJ_TAYLOR_D, OBJ_CENTROID_Y, OBJ_CENTROID_X = 0, 1, 2
STORAGE = {"fp64": FP64, "fp32": FP32, "fp16": FP16}
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_UNSTABLE",
                5: "ERR_SUPPORT", 6: "ERR_TIMEOUT", 7: "ERR_STATE"}


class LbmibError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class lbmib_config(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("walls", C.c_int),
        ("tau", C.c_double), ("u_bottom", C.c_double), ("u_top", C.c_double),
        ("gx", C.c_double), ("gy", C.c_double),
        ("storage", C.c_int), ("max_capsules", C.c_int), ("max_nodes", C.c_int),
    ]


class lbmib_case(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("walls", C.c_int),
        ("tau", C.c_double), ("u_bottom", C.c_double), ("u_top", C.c_double),
        ("gx", C.c_double), ("gy", C.c_double),
        ("rho", C.c_void_p), ("ux", C.c_void_p), ("uy", C.c_void_p),
        ("xy", C.c_void_p), ("n", C.c_int),
        ("k_s", C.c_double), ("k_b", C.c_double), ("k_a", C.c_double), ("node_mass", C.c_double),
    ]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run __graft_entry__.build() (nvcc, sm_103a)")

_lib = C.CDLL(LIB_PATH)
_vp, _dp = C.c_void_p, C.POINTER(C.c_double)
_CFG = C.POINTER(lbmib_config)
_SIGS = {
    "lbmib_arena_bytes": (C.c_size_t, [_CFG]),
    "lbmib_create": (C.c_int, [_CFG, _vp, C.c_size_t, _vp, C.POINTER(_vp)]),
    "lbmib_destroy": (None, [_vp]),
    "lbmib_last_error": (C.c_char_p, [_vp]),
    "lbmib_init_fields": (C.c_int, [_vp, _vp, _vp, _vp]),
    "lbmib_add_capsule": (C.c_int, [_vp, _vp, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                    C.POINTER(C.c_int)]),
    "lbmib_set_capsule_positions": (C.c_int, [_vp, C.c_int, _vp]),
    "lbmib_step": (C.c_int, [_vp, C.c_longlong, C.c_int]),
    "lbmib_sync": (C.c_int, [_vp]),
    "lbmib_read_fields": (C.c_int, [_vp, _vp, _vp, _vp]),
    "lbmib_read_populations": (C.c_int, [_vp, _vp]),
    "lbmib_read_force_field": (C.c_int, [_vp, _vp, _vp]),
    "lbmib_read_capsule": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp]),
    "lbmib_observables": (C.c_int, [_vp, C.c_int, _vp]),
    "lbmib_observables_all": (C.c_int, [_vp, _vp]),
    "lbmib_interpolate": (C.c_int, [_vp, _vp, C.c_int, _vp]),
    "lbmib_interpolate_noalloc": (C.c_int, [_vp, _vp, C.c_int, _vp]),
    "lbmib_state_bytes": (C.c_size_t, [_vp]),
    "lbmib_save_state": (C.c_int, [_vp, _vp, C.c_size_t]),
    "lbmib_load_state": (C.c_int, [_vp, _vp, C.c_size_t]),
    "lbmib_set_option": (C.c_int, [_vp, C.c_int, C.c_longlong]),
    "lbmib_kernel_time": (C.c_int, [_vp, _dp, C.POINTER(C.c_longlong), C.c_int]),
    "lbmib_ib_kernel_time": (C.c_int, [_vp, _dp, _dp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.c_int]),
    "lbmib_launch_count": (C.c_longlong, [_vp]),
    "lbmib_bytes_per_update": (C.c_double, [_vp]),
    "lbmib_set_repulsion": (C.c_int, [_vp, C.c_double, C.c_double]),
    "lbmib_set_inflow": (C.c_int, [_vp, _vp, C.c_double]),
    "lbmib_add_rigid": (C.c_int, [_vp, _vp, C.c_int, C.c_double, C.c_double, C.POINTER(C.c_int)]),
    "lbmib_read_rigid": (C.c_int, [_vp, C.c_int, _vp]),
    "lbmib_field_ptr": (C.c_int, [_vp, C.c_int, C.POINTER(_vp), C.POINTER(C.c_int)]),
    "lbmib_adjoint_workspace_bytes": (C.c_size_t, [_vp, C.c_longlong, C.c_int]),
    "lbmib_adjoint": (C.c_int, [_vp, C.c_longlong, C.c_int, C.c_int, C.c_int, C.c_int, _vp, C.c_size_t, _vp, _vp]),
    "lbmib_batch_arena_bytes": (C.c_size_t, [_vp, C.c_int, C.c_int]),
    "lbmib_batch_create": (C.c_int, [_vp, C.c_int, C.c_int, _vp, C.c_size_t, _vp, C.c_int, C.POINTER(_vp)]),
    "lbmib_batch_destroy": (None, [_vp]),
    "lbmib_batch_last_error": (C.c_char_p, [_vp]),
    "lbmib_batch_step": (C.c_int, [_vp, C.c_longlong]),
    "lbmib_batch_sync": (C.c_int, [_vp]),
    "lbmib_batch_read_populations": (C.c_int, [_vp, C.c_int, _vp]),
    "lbmib_batch_read_capsule": (C.c_int, [_vp, C.c_int, _vp, _vp]),
    "lbmib_batch_observables": (C.c_int, [_vp, _vp]),
    "lbmib_batch_config": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---- one-to-one C names --------------------------------------------------------------
def lbmib_arena_bytes(cfg: lbmib_config) -> int:
    return int(_lib.lbmib_arena_bytes(C.byref(cfg)))


def lbmib_create(cfg: lbmib_config, d_arena: int, arena_bytes: int, cuda_stream: int) -> int:
    h = C.c_void_p()
    st = _lib.lbmib_create(C.byref(cfg), C.c_void_p(d_arena), arena_bytes, C.c_void_p(cuda_stream), C.byref(h))
    if st != OK:
        raise LbmibError(st, "lbmib_create failed")
    return h.value


def lbmib_destroy(h: int) -> None:
    _lib.lbmib_destroy(h)


def lbmib_last_error(h: int) -> str:
    return _lib.lbmib_last_error(h).decode()


def _check(h, st):
    if st != OK:
        raise LbmibError(st, lbmib_last_error(h))


def lbmib_init_fields(h, rho=None, ux=None, uy=None):
    a = [None if v is None else _f64(v) for v in (rho, ux, uy)]
    _check(h, _lib.lbmib_init_fields(h, *[_p(v) for v in a]))


def lbmib_add_capsule(h, xy, k_s, k_b, k_a, node_mass) -> int:
    xy = _f64(xy).reshape(-1)
    out = C.c_int()
    _check(h, _lib.lbmib_add_capsule(h, _p(xy), xy.size // 2, k_s, k_b, k_a, node_mass, C.byref(out)))
    return out.value


def lbmib_set_capsule_positions(h, cid, xy):
    xy = _f64(xy).reshape(-1)
    _check(h, _lib.lbmib_set_capsule_positions(h, cid, _p(xy)))


def lbmib_step(h, nsteps: int, scheme: int):
    _check(h, _lib.lbmib_step(h, int(nsteps), int(scheme)))


def lbmib_sync(h):
    _check(h, _lib.lbmib_sync(h))


def lbmib_read_fields(h, rho, ux, uy):
    _check(h, _lib.lbmib_read_fields(h, _p(rho), _p(ux), _p(uy)))


def lbmib_read_populations(h, f):
    _check(h, _lib.lbmib_read_populations(h, _p(f)))


def lbmib_read_force_field(h, fx, fy):
    _check(h, _lib.lbmib_read_force_field(h, _p(fx), _p(fy)))


def lbmib_read_capsule(h, cid, xy, vel, fint, fext):
    _check(h, _lib.lbmib_read_capsule(h, cid, _p(xy), _p(vel), _p(fint), _p(fext)))


def lbmib_observables(h, cid, out):
    _check(h, _lib.lbmib_observables(h, cid, _p(out)))


def lbmib_observables_all(h, out):
    _check(h, _lib.lbmib_observables_all(h, _p(out)))


def lbmib_interpolate(h, xy, out):
    _check(h, _lib.lbmib_interpolate(h, _p(xy), xy.size // 2, _p(out)))


def lbmib_interpolate_noalloc(h, xy, out):
    _check(h, _lib.lbmib_interpolate_noalloc(h, _p(xy), xy.size // 2, _p(out)))


def lbmib_state_bytes(h) -> int:
    return int(_lib.lbmib_state_bytes(h))


def lbmib_save_state(h, buf: np.ndarray):
    _check(h, _lib.lbmib_save_state(h, _p(buf), buf.nbytes))


def lbmib_load_state(h, buf: np.ndarray):
    _check(h, _lib.lbmib_load_state(h, _p(buf), buf.nbytes))


def lbmib_set_option(h, option: int, value: int):
    _check(h, _lib.lbmib_set_option(h, option, int(value)))


def lbmib_kernel_time(h, reset: bool = False):
    ms = C.c_double()
    n = C.c_longlong()
    _check(h, _lib.lbmib_kernel_time(h, C.byref(ms), C.byref(n), int(reset)))
    return ms.value, n.value


def lbmib_ib_kernel_time(h, reset: bool = False):
    """(patch ms, IB update ms, steps timed, touched-list length of the last spread)."""
    pm, im = C.c_double(), C.c_double()
    n, listed = C.c_longlong(), C.c_longlong()
    _check(h, _lib.lbmib_ib_kernel_time(h, C.byref(pm), C.byref(im), C.byref(n), C.byref(listed), int(reset)))
    return pm.value, im.value, n.value, listed.value


def lbmib_launch_count(h) -> int:
    return int(_lib.lbmib_launch_count(h))


def lbmib_bytes_per_update(h) -> float:
    return float(_lib.lbmib_bytes_per_update(h))


def lbmib_set_repulsion(h, cutoff: float, coeff: float = 0.0):
    _check(h, _lib.lbmib_set_repulsion(h, float(cutoff), float(coeff)))


def lbmib_set_inflow(h, u_in, rho_out: float = 1.0):
    if u_in is None:
        _check(h, _lib.lbmib_set_inflow(h, None, float(rho_out)))
        return
    u = _f64(u_in)
    _check(h, _lib.lbmib_set_inflow(h, u.ctypes.data_as(_vp), float(rho_out)))


def lbmib_adjoint_workspace_bytes(h, nsteps: int, ckpt_every: int) -> int:
    return int(_lib.lbmib_adjoint_workspace_bytes(h, int(nsteps), int(ckpt_every)))


def lbmib_adjoint(h, nsteps, scheme, ckpt_every, objective, capsule, d_work, work_bytes, grad):
    J = C.c_double()
    _check(h, _lib.lbmib_adjoint(h, int(nsteps), int(scheme), int(ckpt_every), int(objective), int(capsule),
                                 C.c_void_p(d_work), int(work_bytes), C.byref(J), _p(grad)))
    return J.value


def lbmib_batch_arena_bytes(cases, ncases: int, storage: int) -> int:
    return int(_lib.lbmib_batch_arena_bytes(C.cast(cases, C.c_void_p), int(ncases), int(storage)))


def lbmib_batch_create(cases, ncases, storage, d_arena, arena_bytes, cuda_stream, autotune_steps) -> int:
    h = C.c_void_p()
    st = _lib.lbmib_batch_create(C.cast(cases, C.c_void_p), int(ncases), int(storage), C.c_void_p(d_arena),
                                 arena_bytes, C.c_void_p(cuda_stream), int(autotune_steps), C.byref(h))
    if st != OK:
        raise LbmibError(st, "lbmib_batch_create failed")
    return h.value


def lbmib_batch_destroy(h) -> None:
    _lib.lbmib_batch_destroy(h)


def lbmib_batch_last_error(h) -> str:
    return _lib.lbmib_batch_last_error(h).decode()


def _bcheck(h, st):
    if st != OK:
        raise LbmibError(st, lbmib_batch_last_error(h))


def lbmib_batch_step(h, nsteps: int):
    _bcheck(h, _lib.lbmib_batch_step(h, int(nsteps)))


def lbmib_batch_sync(h):
    _bcheck(h, _lib.lbmib_batch_sync(h))


def lbmib_batch_read_populations(h, c, f):
    _bcheck(h, _lib.lbmib_batch_read_populations(h, int(c), _p(f)))


def lbmib_batch_read_capsule(h, c, xy, vel):
    _bcheck(h, _lib.lbmib_batch_read_capsule(h, int(c), _p(xy), _p(vel)))


def lbmib_batch_observables(h, out):
    _bcheck(h, _lib.lbmib_batch_observables(h, _p(out)))


def lbmib_batch_config(h):
    t, g, c = C.c_int(), C.c_int(), C.c_int()
    _bcheck(h, _lib.lbmib_batch_config(h, C.byref(t), C.byref(g), C.byref(c)))
    return t.value, g.value, c.value


# ---- convenience wrapper ---------------------------------------------------------------
class Context:
    """One lattice with capsules on one CUDA device; device memory from torch."""

    def __init__(self, nx, ny, tau, walls=False, u_bottom=0.0, u_top=0.0, gx=0.0, gy=0.0,
                 storage="fp64", max_capsules=0, max_nodes=0, device=None, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("the LBM-IB library needs a CUDA device")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.cfg = lbmib_config(int(nx), int(ny), int(bool(walls)), float(tau), float(u_bottom),
                                float(u_top), float(gx), float(gy),
                                STORAGE[storage] if isinstance(storage, str) else int(storage),
                                int(max_capsules), int(max_nodes))
        nbytes = lbmib_arena_bytes(self.cfg)
        if nbytes == 0:
            raise LbmibError(ERR_ARG, "invalid configuration")
        self.arena = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            self.h = lbmib_create(self.cfg, self.arena.data_ptr(), nbytes, self.stream.cuda_stream)
        self.nx, self.ny = int(nx), int(ny)
        self._n = []

    def close(self):
        if getattr(self, "h", None):
            lbmib_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # setup
    def init_fields(self, rho=None, ux=None, uy=None):
        lbmib_init_fields(self.h, rho, ux, uy)

    def add_capsule(self, xy, k_s, k_b, k_a, node_mass) -> int:
        cid = lbmib_add_capsule(self.h, xy, k_s, k_b, k_a, node_mass)
        self._n.append(np.asarray(xy).size // 2)
        return cid

    def set_capsule_positions(self, cid, xy):
        lbmib_set_capsule_positions(self.h, cid, xy)

    def set_repulsion(self, cutoff: float, coeff: float = 0.0):
        """Capsule-capsule repulsion of Eq. 27 (cutoff 0: off; coeff 0: the printed one)."""
        lbmib_set_repulsion(self.h, cutoff, coeff)

    def add_rigid(self, xy, mass: float, inertia: float) -> int:
        """Rigid particle (Section 2.3.1): ring xy (n, 2), mass and moment of inertia about
        its area centroid; at rest; Dynamic scheme only."""
        xy = _f64(xy)
        n = xy.size // 2
        out = C.c_int(-1)
        _check(self.h, _lib.lbmib_add_rigid(self.h, xy.ctypes.data_as(_vp), n, float(mass), float(inertia),
                                            C.byref(out)))
        self._n.append(n)
        return out.value

    def read_rigid(self, cid: int) -> np.ndarray:
        """(c_x, c_y, theta, u_x, u_y, omega, F_x, F_y, M) of rigid particle cid."""
        out = np.zeros(9)
        _check(self.h, _lib.lbmib_read_rigid(self.h, int(cid), out.ctypes.data_as(_vp)))
        return out

    def field_view(self, field: int):
        """Zero-copy torch view of a device field (no synchronisation afterwards; valid until
        the next step): FIELD_POPULATIONS -> (9, ny, pitch) post-collision populations in the
        storage dtype, stored as f_i - w_i (FP16: times the storage scale); FIELD_FORCE ->
        (2, ny, nx) float64 immersed-boundary force of the last spread."""
        import torch

        ptr = _vp()
        pitch = C.c_int(0)
        _check(self.h, _lib.lbmib_field_ptr(self.h, int(field), C.byref(ptr), C.byref(pitch)))
        off = ptr.value - self.arena.data_ptr()
        if field == FIELD_POPULATIONS:
            dtype = {STORAGE["fp64"]: torch.float64, STORAGE["fp32"]: torch.float32,
                     STORAGE["fp16"]: torch.float16}[self.cfg.storage]
            shape = (9, self.ny, pitch.value)
        else:
            dtype, shape = torch.float64, (2, self.ny, self.nx)
        n = int(np.prod(shape))
        size = torch.empty((), dtype=dtype).element_size()
        return self.arena[off:off + n * size].view(dtype).view(shape)

    def set_inflow(self, u_in, rho_out: float = 1.0):
        """Open channel: Zou-He inlet with x-velocity u_in (ny values) at x = 0 and outlet
        density rho_out at x = nx - 1 (u_in None: periodic x again)."""
        if u_in is not None and np.asarray(u_in).size != self.ny:
            raise ValueError("u_in needs one value per row")
        lbmib_set_inflow(self.h, u_in, rho_out)

    # stepping
    def step(self, nsteps: int, scheme: int = KINEMATIC):
        lbmib_step(self.h, nsteps, scheme)

    def sync(self):
        lbmib_sync(self.h)

    # read-back
    def read_fields(self):
        rho = np.empty((self.ny, self.nx)); ux = np.empty_like(rho); uy = np.empty_like(rho)
        lbmib_read_fields(self.h, rho, ux, uy)
        return rho, ux, uy

    def read_populations(self):
        f = np.empty((9, self.ny, self.nx))
        lbmib_read_populations(self.h, f)
        return f

    def read_force_field(self):
        f = np.empty((2, self.ny, self.nx))
        lbmib_read_force_field(self.h, f[0], f[1])
        return f

    def read_capsule(self, cid: int):
        n = self._n[cid]
        out = [np.empty(2 * n) for _ in range(4)]
        lbmib_read_capsule(self.h, cid, *out)
        return tuple(out)

    def observables(self, cid: int) -> np.ndarray:
        out = np.empty(8)
        lbmib_observables(self.h, cid, out)
        return out

    def observables_all(self) -> np.ndarray:
        out = np.empty((len(self._n), 8))
        lbmib_observables_all(self.h, out)
        return out

    def interpolate(self, xy) -> np.ndarray:
        xy = _f64(xy).reshape(-1)
        out = np.empty(4 * xy.size)
        lbmib_interpolate(self.h, xy, out)
        return out.reshape(-1, 8)

    def interpolate_noalloc(self, xy) -> np.ndarray:
        """lbmib_interpolate through the library's static staging (no allocation)."""
        xy = _f64(xy).reshape(-1)
        out = np.empty(4 * xy.size)
        lbmib_interpolate_noalloc(self.h, xy, out)
        return out.reshape(-1, 8)

    def save_state(self) -> np.ndarray:
        buf = np.empty(lbmib_state_bytes(self.h), dtype=np.uint8)
        lbmib_save_state(self.h, buf)
        return buf

    def load_state(self, buf: np.ndarray):
        lbmib_load_state(self.h, np.ascontiguousarray(buf))

    def set_option(self, option: int, value: int):
        """lbmib_set_option: OPT_GRAPHS, OPT_TIMING, OPT_GRAPH_STEPS, OPT_FP16_SCALE,
        OPT_LATTICE_VARIANT, OPT_OVERLAP, OPT_ARCS, OPT_FUSE_IB, OPT_IB_FP64 (meanings and
        ranges in include/lbmib.h)."""
        lbmib_set_option(self.h, option, value)

    def kernel_time(self, reset=False):
        return lbmib_kernel_time(self.h, reset)

    def ib_kernel_time(self, reset=False):
        return lbmib_ib_kernel_time(self.h, reset)

    def adjoint(self, nsteps: int, objective: int = OBJ_TAYLOR_D, capsule: int = 0, ckpt_every: int = 200,
                scheme: int = KINEMATIC):
        """Advance nsteps steps and return (J, grad) with grad = {dJ/dk_s per capsule,
        dJ/dk_b per capsule, dJ/dgx, dJ/dgy}; the workspace is a temporary torch buffer."""
        import torch

        nbytes = lbmib_adjoint_workspace_bytes(self.h, nsteps, ckpt_every)
        if nbytes == 0:
            raise LbmibError(ERR_ARG, "invalid adjoint arguments")
        work = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        grad = np.zeros(2 * len(self._n) + 2)
        J = lbmib_adjoint(self.h, nsteps, scheme, ckpt_every, objective, capsule, work.data_ptr(), nbytes, grad)
        del work
        return J, grad

    @property
    def launch_count(self) -> int:
        return lbmib_launch_count(self.h)

    @property
    def bytes_per_update(self) -> float:
        return lbmib_bytes_per_update(self.h)


def from_case(case, storage="fp64", extra_nodes=0, extra_capsules=0, **kw) -> Context:
    """Context for a ``workloads.Case``: lattice, initial fields and capsules."""
    ctx = Context(case.nx, case.ny, case.tau, case.walls, case.u_bottom, case.u_top, case.gx, case.gy,
                  storage=storage, max_capsules=len(case.capsules) + extra_capsules,
                  max_nodes=case.n_nodes + extra_nodes, **kw)
    ctx.init_fields(*case.fields())
    if getattr(case, "u_in", None) is not None:
        ctx.set_inflow(case.u_in, case.rho_out)
    for c in case.capsules:
        ctx.add_capsule(c.xy, c.ks, c.kb, c.ka, c.mass)
    return ctx


class Batch:
    """Independent cases (``workloads.Case`` with at most one capsule each) advanced by
    the Kinematic scheme in one persistent launch; device memory from torch."""

    def __init__(self, cases, storage="fp32", autotune_steps=0, device=None, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("the LBM-IB library needs a CUDA device")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        self.shapes = [(c.nx, c.ny) for c in cases]
        self._n = []
        keep = []                       # host arrays referenced by the case table
        table = (lbmib_case * len(cases))()
        for k, case in enumerate(cases):
            if len(case.capsules) > 1:
                raise ValueError("a batched case holds at most one capsule")
            rho, ux, uy = (_f64(a) for a in case.fields())
            keep += [rho, ux, uy]
            t = table[k]
            t.nx, t.ny, t.walls = case.nx, case.ny, int(bool(case.walls))
            t.tau, t.u_bottom, t.u_top, t.gx, t.gy = case.tau, case.u_bottom, case.u_top, case.gx, case.gy
            t.rho, t.ux, t.uy = rho.ctypes.data, ux.ctypes.data, uy.ctypes.data
            if case.capsules:
                cap = case.capsules[0]
                xy = _f64(cap.xy).reshape(-1)
                keep.append(xy)
                t.xy, t.n = xy.ctypes.data, xy.size // 2
                t.k_s, t.k_b, t.k_a, t.node_mass = cap.ks, cap.kb, cap.ka, cap.mass
            self._n.append(int(t.n))
        nbytes = lbmib_batch_arena_bytes(table, len(cases), self.storage)
        if nbytes == 0:
            raise LbmibError(ERR_ARG, "invalid batch")
        self.arena = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            self.h = lbmib_batch_create(table, len(cases), self.storage, self.arena.data_ptr(), nbytes,
                                        self.stream.cuda_stream, autotune_steps)
        del keep

    def close(self):
        if getattr(self, "h", None):
            lbmib_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, nsteps: int):
        lbmib_batch_step(self.h, nsteps)

    def sync(self):
        lbmib_batch_sync(self.h)

    def read_populations(self, c: int) -> np.ndarray:
        nx, ny = self.shapes[c]
        f = np.empty((9, ny, nx))
        lbmib_batch_read_populations(self.h, c, f)
        return f

    def read_capsule(self, c: int):
        n = self._n[c]
        xy, vel = np.empty(2 * n), np.empty(2 * n)
        lbmib_batch_read_capsule(self.h, c, xy, vel)
        return xy, vel

    def observables(self) -> np.ndarray:
        out = np.empty((len(self.shapes), 8))
        lbmib_batch_observables(self.h, out)
        return out

    @property
    def config(self):
        """(threads per CTA, resident CTAs, tile cells)"""
        return lbmib_batch_config(self.h)
