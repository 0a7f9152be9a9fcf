"""The all-core build of the oracle (the same C compiled with -fopenmp, used only as the
timed all-core CPU baseline) gives bit-identical results to the plain single-thread
build: its lattice loop splits independent rows over threads."""
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import oracle as o
from paper_1903_03356_gb300 import workloads as W
case = W.poiseuille_biconcave(nx=512, ny=128, count=6, n=64, seed=0, scheme=W.DYNAMIC)
s = o.Sim(o.lattice(case.nx, case.ny, case.tau, True, gx=case.gx))
s.init_fields(*case.fields())
for c in case.capsules:
    s.add_capsule(c.xy, c.ks, c.kb, c.ka, c.mass)
assert s.step(30, o.DYNAMIC) == 0
np.savez(sys.argv[2], f=s.populations(), x=s.read_capsule(0)[0], omp=o.OPENMP)
"""


def _run(path, openmp):
    env = dict(os.environ, LBMIB_ORACLE_OPENMP="1" if openmp else "0", OMP_NUM_THREADS="4")
    subprocess.run([sys.executable, "-c", SCRIPT, ROOT, path], check=True, env=env, timeout=300)
    return np.load(path)


def test_all_core_build_is_bit_identical(tmp_path):
    a = _run(str(tmp_path / "plain.npz"), False)
    b = _run(str(tmp_path / "omp.npz"), True)
    assert not bool(a["omp"]) and bool(b["omp"])
    assert np.array_equal(a["f"], b["f"]) and np.array_equal(a["x"], b["x"])
