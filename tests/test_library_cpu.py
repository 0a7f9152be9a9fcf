"""CPU checks of the CUDA library and the input generator (no GPU needed).

The library is built for sm_103a here (nvcc cross-compiles), loaded with ctypes, and
checked to export every entry point that include/*.h declares. Host-only logic (arena
sizing, argument validation) runs without a device.
"""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

from paper_1903_03356_gb300 import build
from paper_1903_03356_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    path = build.build()
    return C.CDLL(path)


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(lbmib_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbmib_create", "lbmib_add_capsule", "lbmib_step", "lbmib_read_fields",
                     "lbmib_read_capsule", "lbmib_observables", "lbmib_save_state",
                     "lbmib_load_state", "lbmib_last_error", "lbmib_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def header_constants():
    """Every enumerator `LBMIB_NAME = value` that include/*.h declares."""
    out = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for name, value in re.findall(r"\bLBMIB_(\w+)\s*=\s*(\d+)", text):
            out[name] = int(value)
    return out


def test_binding_constants_match_the_header():
    from paper_1903_03356_gb300 import lbmib
    hc = header_constants()
    checked = 0
    for name, value in hc.items():
        if isinstance(getattr(lbmib, name, None), int):
            assert getattr(lbmib, name) == value, name
            checked += 1
    opts = [n for n in hc if n.startswith("OPT_")]
    assert len(opts) >= 9 and all(hasattr(lbmib, n) for n in opts), opts
    assert checked >= len(opts) + 5


def _cfg(lib_mod, **kw):
    base = dict(nx=100, ny=64, walls=1, tau=0.8, u_bottom=0.0, u_top=0.0, gx=0.0, gy=0.0,
                storage=1, max_capsules=4, max_nodes=512)
    base.update(kw)
    return lib_mod.lbmib_config(**base)


def test_arena_sizing_is_host_logic():
    from paper_1903_03356_gb300 import lbmib as L
    fp64 = L.lbmib_arena_bytes(_cfg(L, storage=0))
    fp32 = L.lbmib_arena_bytes(_cfg(L, storage=1))
    fp16 = L.lbmib_arena_bytes(_cfg(L, storage=2))
    assert fp64 > fp32 > fp16 > 0
    # two population buffers of 9 planes with rows padded to 128 bytes
    N = 100 * 64
    assert fp32 >= 2 * 9 * 64 * 128 * 4 + 2 * 2 * N * 8
    big = L.lbmib_arena_bytes(_cfg(L, nx=16384, ny=8192, max_capsules=16384, max_nodes=16384 * 128))
    assert 9.6e9 < big < 40e9          # fits a GB300 with room to spare


@pytest.mark.parametrize("bad", [dict(nx=2), dict(ny=0), dict(tau=0.5), dict(storage=7),
                                 dict(max_nodes=-1)])
def test_invalid_configurations_are_rejected(bad):
    from paper_1903_03356_gb300 import lbmib as L
    assert L.lbmib_arena_bytes(_cfg(L, **bad)) == 0


def test_create_rejects_bad_arguments_without_touching_a_device():
    from paper_1903_03356_gb300 import lbmib as L
    h = C.c_void_p()
    cfg = _cfg(L)
    # NULL arena, misaligned arena and undersized arena are refused before any CUDA call
    assert L._lib.lbmib_create(C.byref(cfg), None, 1 << 30, None, C.byref(h)) == L.ERR_ARG
    assert L._lib.lbmib_create(C.byref(cfg), C.c_void_p(4096 + 8), 1 << 30, None, C.byref(h)) == L.ERR_ARG
    assert L._lib.lbmib_create(C.byref(cfg), C.c_void_p(4096), 16, None, C.byref(h)) == L.ERR_OOM
    assert h.value is None


def test_shapes_are_counter_clockwise_and_tie_free():
    for xy in (W.circle(64, 10, 50.1, 49.513), W.biconcave(128, 8.0, 33.3, 21.7)):
        assert W.signed_area(xy) > 0
        assert W.min_half_integer_distance(xy) > 1e-9
    c = W.poiseuille_biconcave(nx=1024, ny=256, count=32, seed=0, steps=1)
    c2 = W.poiseuille_biconcave(nx=1024, ny=256, count=32, seed=0, steps=1)
    assert all(np.array_equal(a.xy, b.xy) for a, b in zip(c.capsules, c2.capsules))
    boxes = [(cap.xy[:, 0].min(), cap.xy[:, 0].max(), cap.xy[:, 1].min(), cap.xy[:, 1].max())
             for cap in c.capsules]
    for i in range(len(boxes)):
        assert boxes[i][2] > 1.5 and boxes[i][3] < 256 - 2.5      # clear of the walls
        for j in range(i):
            a, b = boxes[i], boxes[j]
            assert a[1] < b[0] or b[1] < a[0] or a[3] < b[2] or b[3] < a[2]


def test_parameter_mappings():
    # shear case: Ca = mu gamma a / k_s = 0.01 with nu = 0.1, gamma = 1e-4, a = 10
    # gives k_s = 0.1 * 1e-4 * 10 / 0.01 = 1e-2 and k_b = 0.01 k_s a^2 = 1e-2 (shear case: no cap)
    case = W.shear_capsule()
    assert abs(case.capsules[0].ks - 1e-2) < 1e-15
    assert abs(case.capsules[0].kb - 1e-2) < 1e-15
    assert abs(case.u_top - 0.005) < 1e-15 and case.u_bottom == -case.u_top
    # Poiseuille: g = 8 rho nu u_max / H^2
    p = W.poiseuille_capsule()
    assert abs(p.gx - 8 * (0.2 / 3) * 0.02 / 120 ** 2) < 1e-20
    assert abs(p.capsules[0].ks - (0.2 / 3) * 0.02 / 1e-2) < 1e-15


def test_batch_cases_follow_their_recipe():
    cases = W.batch_cases(count=64, seed=1, steps=1)
    for c in cases:
        assert c.nx in W.BATCH_SIZES and c.ny in W.BATCH_SIZES
        n = c.capsules[0].xy.shape[0]
        assert n in W.BATCH_NODES
        assert W.signed_area(c.capsules[0].xy) > 0


def _batch_table(L, cases):
    keep, table = [], (L.lbmib_case * len(cases))()
    for k, case in enumerate(cases):
        t = table[k]
        t.nx, t.ny, t.walls, t.tau = case.nx, case.ny, int(case.walls), case.tau
        t.u_bottom, t.u_top = case.u_bottom, case.u_top
        if case.capsules:
            xy = np.ascontiguousarray(case.capsules[0].xy, dtype=np.float64).reshape(-1)
            keep.append(xy)
            t.xy, t.n = xy.ctypes.data, xy.size // 2
            cap = case.capsules[0]
            t.k_s, t.k_b, t.k_a, t.node_mass = cap.ks, cap.kb, cap.ka, cap.mass
    return table, keep


def test_batch_arena_sizing_and_rejection_are_host_logic():
    from paper_1903_03356_gb300 import lbmib as L
    cases = W.batch_cases(count=16, seed=1, steps=1)
    table, keep = _batch_table(L, cases)
    fp32 = L.lbmib_batch_arena_bytes(table, 16, L.FP32)
    fp16 = L.lbmib_batch_arena_bytes(table, 16, L.FP16)
    fp64 = L.lbmib_batch_arena_bytes(table, 16, L.FP64)
    assert fp64 > fp32 > fp16 > 0
    # two population buffers of 9 planes per case, rows padded to 128 bytes
    pops = sum(2 * 9 * c.ny * ((c.nx * 4 + 127) // 128 * 128) for c in cases)
    assert fp32 >= pops
    assert L.lbmib_batch_arena_bytes(table, 16, 5) == 0
    assert L.lbmib_batch_arena_bytes(table, 0, L.FP32) == 0
    table[3].tau = 0.5
    assert L.lbmib_batch_arena_bytes(table, 16, L.FP32) == 0
    table[3].tau = 0.8
    table[5].n = 2
    assert L.lbmib_batch_arena_bytes(table, 16, L.FP32) == 0
    table[5].n = 0                   # a case without a capsule is valid
    assert L.lbmib_batch_arena_bytes(table, 16, L.FP32) > 0
    h = C.c_void_p()
    create = L._lib.lbmib_batch_create
    assert create(C.cast(table, C.c_void_p), 16, L.FP32, None, 1 << 30, None, 0, C.byref(h)) == L.ERR_ARG
    assert create(C.cast(table, C.c_void_p), 16, L.FP32, C.c_void_p(4096 + 16), 1 << 34, None, 0,
                  C.byref(h)) == L.ERR_ARG
    assert create(C.cast(table, C.c_void_p), 16, L.FP32, C.c_void_p(4096), 64, None, 0,
                  C.byref(h)) == L.ERR_OOM
    assert h.value is None
