"""Benchmark of one coupled LBM-IB time step on GB300 (MLUPS and HBM roofline).

A step is one pass of the whole hot path: spread, lattice update (collide-stream),
forced-node patch, interpolation, tractions, membrane forces and node update
(Coclite et al., arXiv:1903.03356, Section 2.3-2.4). Default workload: a 16384 x 8192
Poiseuille channel (1.34e8 lattice nodes, far above L2) holding 16384 biconcave
capsules of 128 vertices (the capsule density of the 4096 x 512 precision workload),
Dynamic IB, FP32 shifted storage.

Prints one JSON line. ``--impl reference`` times the FP64 CPU oracle instead, on a
bounded sample of the same workload (the CPU baseline arm).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1903_03356_gb300 import workloads as W  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
METRIC = "LBM-IB MLUPS (coupled step) and % of HBM roofline"

# DRAM bytes (read + write) per lattice update of k_collide_stream from one ncu capture of
# the current kernel on a lattice whose writes dwarf L2 (profiles/k_collide_stream_*.md);
# scaled to a full launch by the number of updates. None where no such capture exists.
MEASURED_TRAFFIC_PER_UPDATE = {"fp32": (1208041472 + 1165416704) / (8192 * 4096), "fp64": None, "fp16": None}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference", "oracle-sample"],
                   help="oracle-sample: internal, one timed oracle sample printed as JSON (the all-core run)")
    p.add_argument("--nx", type=int, default=16384)
    p.add_argument("--ny", type=int, default=8192)
    p.add_argument("--storage", default="fp32", choices=["fp64", "fp32", "fp16"])
    p.add_argument("--scheme", default="dynamic", choices=["dynamic", "kinematic"])
    p.add_argument("--no-capsules", action="store_true", help="lattice update only")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU baseline sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the batched-launch and adjoint measurements that follow the main line")
    p.add_argument("--batch-steps", type=int, default=3000, help="steps per case of the batched workload")
    p.add_argument("--adjoint-steps", type=int, default=8000, help="horizon T of the adjoint measurement")
    p.add_argument("--batch-autotune", type=int, default=20,
                   help="steps per candidate launch shape of the batch autotuner (0: default shape)")
    p.add_argument("--sample-steps", type=int, default=0, help="oracle-sample: timed steps (0: time-bounded)")
    p.add_argument("--study-out", default="", help="oracle-sample --only study: where the oracle's state goes")
    p.add_argument("--study-steps", type=int, default=5000, help="precision study: steps of the GPU runs")
    p.add_argument("--study-oracle-steps", type=int, default=100,
                   help="precision study: steps of the FP64 oracle run the GPU runs are compared with")
    p.add_argument("--only", default="all",
                   choices=["all", "batched", "adjoint", "precision", "dense", "open", "rigid", "study", "fp64",
                            "poiseuille"],
                   help="batched / adjoint: run only that measurement and print its JSON object")
    return p.parse_args()


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def make_case(a):
    scheme = W.DYNAMIC if a.scheme == "dynamic" else W.KINEMATIC
    if a.no_capsules:
        return W.Case("poiseuille_lattice", a.nx, a.ny, 0.7, True,
                      gx=W.poiseuille_force(0.7, 0.02, a.ny), init="parabola", scheme=scheme)
    return W.roofline_lattice(nx=a.nx, ny=a.ny, scheme=scheme, seed=0)


def workload_name(a, case):
    caps = f"{len(case.capsules)}x{case.capsules[0].xy.shape[0] if case.capsules else 0}"
    return f"poiseuille-biconcave-{a.nx}x{a.ny}-{caps}-{a.scheme}-{a.storage}"


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if len(s) > 5 + k and s[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def dist_setup(n):
    if n <= 1 and "WORLD_SIZE" not in os.environ:
        return 0, 1, None
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(n)))
    backend = "nccl" if os.environ.get("LBMIB_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
    dist.init_process_group(backend)
    return rank, world, dist


def max_over_ranks(value: float, dist, device=None) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, elapsed_ms: float, world: int, dist, device=None):
    """Whole-job rate of N independent replicas (no data-path collective): all ranks'
    units over the slowest rank's time. Returns (units per second, slowest ms)."""
    slowest = max_over_ranks(elapsed_ms, dist, device)
    return world * units_per_rank / (slowest / 1e3), slowest


def host_cpu():
    """Model and logical core count of the host that runs the CPU baseline."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu model")):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return {"cpu_model": model or "unknown", "nproc": os.cpu_count()}


SLAB = (2048, 512)


def slab_case(a):
    """The bounded CPU sample of the workload: a 2048 x 512 slab of the same channel with
    the same capsule density (one 128-vertex biconcave capsule per 8192 nodes)."""
    nx, ny = SLAB
    scheme = W.DYNAMIC if a.scheme == "dynamic" else W.KINEMATIC
    if a.no_capsules:
        return W.Case("slab", nx, ny, 0.7, True, gx=W.poiseuille_force(0.7, 0.02, ny), init="parabola")
    return W.poiseuille_biconcave(nx=nx, ny=ny, count=(nx * ny) // 8192, seed=0, scheme=scheme,
                                  placement="grid")


def slab_name(a, case):
    return (f"poiseuille-biconcave-{case.nx}x{case.ny}-{len(case.capsules)}x128-{a.scheme}-f64 "
            f"(CPU sample of the {a.nx}x{a.ny} workload)")


def oracle_sample(a, steps=0, seconds=12.0, warmup=0):
    """The FP64 CPU oracle, as it stands, on the slab: `warmup` untimed steps after the
    start-up step, then `steps` timed steps (or as many as fit in `seconds` when steps is
    0). Threads: one, or every core in the all-core build (LBMIB_ORACLE_OPENMP=1, set by
    oracle_sample_all_cores for its child process)."""
    import oracle as o
    case = slab_case(a)
    scheme = W.DYNAMIC if a.scheme == "dynamic" else W.KINEMATIC
    L = o.lattice(case.nx, case.ny, 0.7, True, gx=case.gx)
    s = o.Sim(L)
    s.init_fields(*case.fields())
    for c in case.capsules:
        s.add_capsule(c.xy, c.ks, c.kb, c.ka, c.mass)
    s.step(1 + warmup, scheme)  # start-up step and warm-up, untimed
    t0 = time.perf_counter()
    done = 0
    if steps > 0:
        s.step(steps, scheme)
        done = steps
    else:
        while time.perf_counter() - t0 < seconds:
            s.step(1, scheme)
            done += 1
    dt = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)) if o.OPENMP else 1
    nodes = case.nx * case.ny
    return {"value": nodes * done / dt / 1e6, "unit": "MLUPS", "cores": threads, "kind": "oracle",
            "steps": done, "ms_per_step": dt / done * 1e3, "workload": slab_name(a, case),
            "sample": f"{case.nx}x{case.ny} slab, {len(case.capsules)} capsules, {done} steps, FP64, "
                      + (f"lattice loop on {threads} threads (OpenMP build)" if o.OPENMP else "single thread"),
            **host_cpu()}


def oracle_sample_all_cores(a, steps=0, seconds=12.0, warmup=0):
    """oracle_sample in a child process that loads the all-core (OpenMP) build."""
    cmd = [sys.executable, os.path.abspath(__file__), "--impl", "oracle-sample", "--scheme", a.scheme,
           "--nx", str(a.nx), "--ny", str(a.ny), "--sample-steps", str(steps), "--cpu-seconds", str(seconds),
           "--warmup", str(warmup)] + (["--no-capsules"] if a.no_capsules else [])
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=600,
                           env=dict(os.environ, LBMIB_ORACLE_OPENMP="1"))
        return json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:   # the baseline line must not sink the benchmark
        return {"unavailable": f"all-core oracle run failed: {type(e).__name__}: {e}"}


def cpu_baseline(a, seconds: float):
    out = oracle_sample(a, seconds=seconds)
    out["all_cores"] = oracle_sample_all_cores(a, seconds=seconds)
    return out


def run_reference(a):
    """The CPU baseline arm: the FP64 oracle as it stands (single thread), W warm-up and K
    timed steps on the slab sample of the workload (there is no reference code; the paper
    describes a method). The line reports what ran: the slab, its steps and its time per
    step; the all-core (OpenMP) run of the same sample and the time per step extrapolated
    to the full lattice are separate keys. Under torchrun only rank 0 runs it."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    base = oracle_sample(a, steps=a.steps, warmup=a.warmup)
    allc = oracle_sample_all_cores(a, steps=a.steps, warmup=a.warmup)
    full = make_case(a)
    line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": "MLUPS",
            "n_gpus": a.gpus, "steps": base["steps"], "warmup": a.warmup, "ms_per_step": base["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": base["workload"], "nx": SLAB[0], "ny": SLAB[1], "scheme": a.scheme,
                       "sample_of": workload_name(a, full), "sample": base["sample"]},
            "cpu_baseline": base,
            "cpu_baseline_all_cores": allc,
            "extrapolated_full_lattice_ms_per_step": base["ms_per_step"] * (a.nx * a.ny) / (SLAB[0] * SLAB[1]),
            "e2e": {"value": base["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(a):
    import torch

    rank, world, dist = dist_setup(a.gpus)
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    from paper_1903_03356_gb300 import lbmib as L

    case = make_case(a)
    scheme = L.DYNAMIC if a.scheme == "dynamic" else L.KINEMATIC
    N = a.nx * a.ny
    t_setup = time.perf_counter()
    ctx = L.from_case(case, storage=a.storage)
    setup_s = time.perf_counter() - t_setup
    stream = ctx.stream

    # warm-up (graph capture, clocks ramp); inputs are far larger than L2
    ctx.step(a.warmup, scheme)
    ctx.sync()
    launches0 = ctx.launch_count

    # the timed steps: the library's own launch path (steps replayed from CUDA graphs)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(dev) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        start.record(stream)
        ctx.step(a.steps, scheme)
        end.record(stream)
        torch.cuda.synchronize()
    elapsed_ms = start.elapsed_time(end)
    ctx.sync()
    launches = ctx.launch_count - launches0

    # the same steps once more with CUDA events around each kernel (direct launches), for
    # the roofline of the lattice kernel and the times of the IB kernels
    ctx.set_option(L.OPT_TIMING, 1)
    ctx.step(2, scheme)
    ctx.sync()
    ctx.kernel_time(reset=True)
    ctx.ib_kernel_time(reset=True)
    start2, end2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start2.record(stream)
    ctx.step(a.steps, scheme)
    end2.record(stream)
    torch.cuda.synchronize()
    timed_ms = start2.elapsed_time(end2)
    ctx.sync()
    k1_ms, k1_n = ctx.kernel_time(reset=True)
    p_ms, ib_ms, ib_n, listed = ctx.ib_kernel_time(reset=True)
    ctx.set_option(L.OPT_TIMING, 0)
    rate, elapsed_ms = job_throughput(N * a.steps, elapsed_ms, world, dist, torch.device("cuda", dev))
    mlups = rate / 1e6
    hbm, src = peaks()
    bpu = ctx.bytes_per_update
    k1_avg_ms = k1_ms / max(1, k1_n)
    achieved = bpu * N / (k1_avg_ms / 1e3) / 1e9

    line = {
        "metric": METRIC,
        "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": elapsed_ms / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "fp16": "f16-storage/f32"}[a.storage],
        "data": "synthetic",
        "config": {"workload": workload_name(a, case), "nx": a.nx, "ny": a.ny,
                   "capsules": len(case.capsules), "markers": case.n_nodes, "scheme": a.scheme,
                   "storage": a.storage, "tau": case.tau,
                   "l2": "inputs larger than L2 (populations 2 x %.1f GB)" % (9 * N * bpu / 18 / 1e9)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm,
                     "traffic": (MEASURED_TRAFFIC_PER_UPDATE[a.storage] * N
                                 if MEASURED_TRAFFIC_PER_UPDATE[a.storage] else None),
                     "kernel": "k_collide_stream", "bytes_per_update": bpu,
                     "kernel_ms": k1_avg_ms, "kernel_share": k1_ms / timed_ms,
                     "timing_pass_ms_per_step": timed_ms / a.steps,
                     "peak_source": src},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "setup_s": setup_s,
    }
    if ib_n:
        # per listed node the patch reads and writes the node's 9 populations and reads its
        # force, and clears the last step's force and reads both lists' entries and its claim
        p_bytes = listed * (bpu + 16 + 16 + 4 + 4 + 4)
        p_avg = p_ms / ib_n
        line["ib_kernels"] = {
            "steps_timed": ib_n, "listed_nodes": listed,
            "patch_ms": p_avg, "patch_share": p_ms / timed_ms,
            "patch_achieved_GBps": p_bytes / (p_avg / 1e3) / 1e9,
            "patch_frac": p_bytes / (p_avg / 1e3) / 1e9 / hbm,
            "ib_update_ms": ib_ms / ib_n, "ib_update_share": ib_ms / timed_ms,
            "note": ("CUDA events on the context stream around each step's patch (k_patch) and "
                     "immersed-boundary node update (k_dyn_update_spread: the update fused with the "
                     "next step's force and spread, with the list-counter reset before it); the "
                     "patch's algorithmic bytes per listed node are its 9 populations read and "
                     "written, the 16-byte force read, the last force cleared and three 4-byte "
                     "list and claim words"),
        }

    if not a.no_e2e:
        line["e2e"] = e2e_run(a, case, L, scheme, dev)
    if rank == 0 and not a.no_extras:
        ctx.close()
        line["ib_fp64"] = ib_fp64_run(L, a, case, scheme)
        line["fp64_storage"] = fp64_coupled_run(L, a, case, scheme, dev)
        line["precision"] = precision_run(L, dev)
        line["precision_study"] = precision_study(L, a.study_steps, a.study_oracle_steps)
        line["poiseuille_runs"] = poiseuille_runs(L)
        line["dense"] = dense_run(L)
        line["open"] = open_run(L)
        line["rigid"] = rigid_run(L)
        line["batched"] = batched_run(L, a.batch_steps, a.batch_autotune)
        line["adjoint"] = {"dynamic": adjoint_run(L, a.storage, a.adjoint_steps, scheme=1),
                           "kinematic": adjoint_run(L, a.storage, a.adjoint_steps, scheme=0)}
    if rank == 0 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(a, a.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


# FP64 instructions (DADD + DMUL + DFMA, thread level) per lattice update of the FP64
# lattice kernel, from one ncu count (profiles/k_collide_stream_fp64_alu.md); GB300 issues
# 2 such instructions per SM per cycle (ncu peak_sustained of the DFMA counter).
FP64_INSTR_PER_UPDATE = 105.5
FP64_INSTR_PER_SM_CYCLE = 2
SM_COUNT = 152


def precision_run(L, dev, steps=(12, 60)):
    """Lattice update alone on the 16384 x 8192 lattice with FP64 and FP16 storage:
    FP16 against the HBM roofline (36 B per update), FP64 against the FP64 ALU roofline
    (measured instructions per update x updates/s against 2 per SM per cycle at the
    sampled clock)."""
    import torch

    out = {}
    for storage, n in (("fp64", steps[0]), ("fp16", steps[1])):
        case = W.Case("lattice", 16384, 8192, 0.7, True, gx=W.poiseuille_force(0.7, 0.02, 8192), init="parabola")
        ctx = L.from_case(case, storage=storage)
        ctx.set_option(L.OPT_TIMING, 1)
        ctx.step(2)
        ctx.sync()
        ctx.kernel_time(reset=True)
        with Clocks(dev) as clk:
            ctx.step(n)
            ctx.sync()
        ms, launches = ctx.kernel_time(reset=True)
        per = ms / max(1, launches)
        nodes = 16384 * 8192
        gl = nodes / (per / 1e3) / 1e9
        r = {"kernel_ms": per, "glups": gl, "bytes_per_update": ctx.bytes_per_update, "clocks": clk.summary()}
        if storage == "fp16":
            hbm, src = peaks()
            achieved = ctx.bytes_per_update * nodes / (per / 1e3) / 1e9
            r["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                             "frac": achieved / hbm, "peak_source": src}
        else:
            mhz = clk.summary().get("sm_mhz") or 2070.0
            peak = FP64_INSTR_PER_SM_CYCLE * SM_COUNT * mhz * 1e6 / 1e9   # G instr/s
            r["roofline"] = {"bound": "alu", "unit": "G FP64 instr/s", "peak": peak,
                             "peak_source": "2 FP64 instructions per SM per cycle x 152 SMs x sampled SM clock",
                             "achieved": (FP64_INSTR_PER_UPDATE * gl if FP64_INSTR_PER_UPDATE else None)}
            if FP64_INSTR_PER_UPDATE:
                r["roofline"]["frac"] = r["roofline"]["achieved"] / peak
        out[storage] = r
        ctx.close()
    return out


def fp64_coupled_run(L, a, case, scheme, dev, steps=20, warmup=3):
    """The main workload (same lattice, capsules and scheme) with FP64 storage: the whole
    coupled step, and its lattice kernel against the FP64 ALU roofline."""
    import torch

    ctx = L.from_case(case, storage="fp64")
    ctx.set_option(L.OPT_TIMING, 1)
    ctx.step(warmup, scheme)
    ctx.sync()
    ctx.kernel_time(reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(dev) as clk:
        torch.cuda.synchronize()
        e0.record(ctx.stream)
        ctx.step(steps, scheme)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ctx.sync()
    kms, kn = ctx.kernel_time(reset=True)
    per = kms / max(1, kn)
    nodes = a.nx * a.ny
    gl = nodes / (per / 1e3) / 1e9
    mhz = clk.summary().get("sm_mhz") or 2070.0
    peak = FP64_INSTR_PER_SM_CYCLE * SM_COUNT * mhz * 1e6 / 1e9
    ctx.close()
    return {"workload": workload_name(a, case).replace(f"-{a.storage}", "-fp64"), "steps": steps,
            "ms_per_step": ms, "mlups": nodes / ms / 1e3, "lattice_kernel_ms": per, "lattice_share": per / ms,
            "roofline": {"bound": "alu", "unit": "G FP64 instr/s", "peak": peak,
                         "achieved": FP64_INSTR_PER_UPDATE * gl, "frac": FP64_INSTR_PER_UPDATE * gl / peak,
                         "peak_source": "2 FP64 instructions per SM per cycle x 152 SMs x sampled SM clock"},
            "clocks": clk.summary()}


def poiseuille_runs(L, steps=20000, every=2000):
    """Dynamic against Kinematic IB for an inertial circular capsule in plane Poiseuille
    flow: 600 x 120 channel, tau 0.7, body force for a centre-line velocity of 0.02,
    radius 12 with 96 vertices starting at y = 0.3 H, density ratio 1 and 5 (Kinematic:
    1 only), Ca 1e-3, 1e-2, 1e-1, FP64 and FP32 storage, `steps` steps: the centroid
    trajectory and Taylor D every `every` steps, and each FP32 run's largest departure
    from its FP64 run."""
    import torch

    out = {"workload": "600x120 Poiseuille channel, circular capsule r 12 (96 vertices) at 0.3 H, tau 0.7, "
                       "u_max 0.02", "steps": steps, "every": every, "runs": []}
    t0 = time.perf_counter()
    for scheme, ratios in ((L.DYNAMIC, (1.0, 5.0)), (L.KINEMATIC, (1.0,))):
        for ratio in ratios:
            for ca in (1e-3, 1e-2, 1e-1):
                case = W.poiseuille_capsule(ca=ca, density_ratio=ratio, scheme=scheme, steps=steps)
                traj = {}
                for storage in ("fp64", "fp32"):
                    ctx = L.from_case(case, storage=storage)
                    rows = []
                    for _ in range(steps // every):
                        ctx.step(every, scheme)
                        o = ctx.observables(0)
                        rows.append([float(o[3]), float(o[4]), float(o[2])])   # x_c, y_c, D
                    ctx.close()
                    traj[storage] = np.array(rows)
                d64, d32 = traj["fp64"], traj["fp32"]
                out["runs"].append({
                    "scheme": "dynamic" if scheme == L.DYNAMIC else "kinematic", "density_ratio": ratio, "ca": ca,
                    "k_s": case.capsules[0].ks, "k_b": case.capsules[0].kb,
                    "fp64": {"x_c": d64[:, 0].round(4).tolist(), "y_c": d64[:, 1].round(5).tolist(),
                             "D": d64[:, 2].round(6).tolist()},
                    "fp32_max_dev": {"y_c": float(np.abs(d32[:, 1] - d64[:, 1]).max()),
                                     "D": float(np.abs(d32[:, 2] - d64[:, 2]).max())}})
    torch.cuda.synchronize()
    out["wall_s"] = time.perf_counter() - t0
    return out


def _study_case():
    # 4096 x 512 channel, 256 biconcave capsules of 128 vertices (a = 8) at non-overlapping
    # random positions from seed 0, Ca = 0.01, Dynamic
    return W.poiseuille_biconcave(nx=4096, ny=512, count=256, n=128, seed=0, scheme=W.DYNAMIC)


def _study_state(fields, obs):
    _, ux, uy = fields
    return np.stack([ux, uy]), np.asarray(obs)[:, 2]


def precision_study(L, steps=5000, oracle_steps=100):
    """Precision study: FP64, FP32 and FP16 population storage on the 4096 x 512 channel
    with 256 biconcave capsules, each run's velocity field and capsule Taylor deformations
    against FP64 references: (1) the FP64 CPU oracle after `oracle_steps` steps (the
    all-core build, a child process); (2) the GPU's FP64-storage run (itself held to the
    oracle at 1e-10 over 1000 steps by the parity tests) after the full `steps`."""
    import tempfile

    case = _study_case()
    out = {"workload": "4096x512 channel, 256 biconcave capsules x 128 vertices (seed 0), Ca 0.01, Dynamic",
           "steps": steps, "oracle_steps": oracle_steps}
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "oracle.npz")
        cmd = [sys.executable, os.path.abspath(__file__), "--impl", "oracle-sample", "--only", "study",
               "--study-oracle-steps", str(oracle_steps), "--study-out", path]
        t0 = time.perf_counter()
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=1800,
                           env=dict(os.environ, LBMIB_ORACLE_OPENMP="1"))
        if r.returncode != 0 or not os.path.exists(path):
            out["vs_oracle"] = {"unavailable": (r.stderr or r.stdout).strip()[-300:]}
            ref = None
        else:
            z = np.load(path)
            ref = (z["vel"], z["D"])
            out["oracle_s"] = time.perf_counter() - t0
    runs = {}
    for storage in ("fp64", "fp32", "fp16"):
        ctx = L.from_case(case, storage=storage)
        ctx.step(oracle_steps, L.DYNAMIC)
        early = _study_state(ctx.read_fields(), ctx.observables_all())
        ctx.step(steps - oracle_steps, L.DYNAMIC)
        late = _study_state(ctx.read_fields(), ctx.observables_all())
        runs[storage] = (early, late)
        ctx.close()

    def err(a, b):
        return {"velocity_rel_max": float(np.abs(a[0] - b[0]).max() / np.abs(b[0]).max()),
                "max_abs_dD": float(np.abs(a[1] - b[1]).max())}

    if ref is not None:
        out["vs_oracle"] = {k: err(v[0], ref) for k, v in runs.items()}
    out["vs_gpu_fp64"] = {k: err(runs[k][1], runs["fp64"][1]) for k in ("fp32", "fp16")}
    out["D_mean_end"] = float(runs["fp64"][1][1].mean())
    return out


def study_oracle(oracle_steps, path):
    """Child process of precision_study: the oracle's state after oracle_steps steps."""
    import oracle as o
    case = _study_case()
    s = o.Sim(o.lattice(case.nx, case.ny, case.tau, True, gx=case.gx))
    s.init_fields(*case.fields())
    for c in case.capsules:
        s.add_capsule(c.xy, c.ks, c.kb, c.ka, c.mass)
    assert s.step(oracle_steps, o.DYNAMIC) == 0
    vel, D = _study_state(s.read_fields(), [s.observables(k) for k in range(len(case.capsules))])
    np.savez(path, vel=vel, D=D)


def ib_fp64_run(L, a, case, scheme, steps=100, warmup=10):
    """The main workload with the immersed-boundary arithmetic in FP64 over the same
    storage (LBMIB_OPT_IB_FP64: gathers in storage precision; MLS solve, membrane and
    traction forces and node update in double)."""
    import torch

    ctx = L.from_case(case, storage=a.storage)
    ctx.set_option(L.OPT_IB_FP64, 1)
    ctx.step(warmup, scheme)
    ctx.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(ctx.stream)
    ctx.step(steps, scheme)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ctx.close()
    return {"workload": workload_name(a, case) + "-ib-fp64", "steps": steps, "ms_per_step": ms,
            "mlups": a.nx * a.ny / ms / 1e3}


def dense_run(L, steps=200, warmup=20, rc=2.0):
    """Section 3.4 suspension: 16 biconcave capsules of 1000 vertices at 30% hematocrit in a
    1200 x 450 channel (540 000 lattice nodes, 16 000 markers), Dynamic IB, FP32, with the
    capsule-capsule repulsion of Eq. 27 (cut-off rc) and without it."""
    import torch

    case = W.dense_biconcave()
    out = {"workload": "1200x450 channel, 16 biconcave capsules x 1000 vertices, 30% hematocrit, Dynamic, FP32",
           "steps": steps, "cutoff": rc}
    for key, cut in (("with_repulsion", rc), ("without", 0.0)):
        ctx = L.from_case(case, storage="fp32")
        ctx.set_repulsion(cut)
        ctx.step(warmup, L.DYNAMIC)
        ctx.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(ctx.stream)
        ctx.step(steps, L.DYNAMIC)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ctx.sync()
        out[key] = {"ms_per_step": ms / steps, "mlups": case.nx * case.ny * steps / ms / 1e3}
        ctx.close()
    return out


def open_run(L, steps=500, warmup=50):
    """Section 3.2 open channel (Zou-He parabolic inlet, constant-pressure outlet): the
    capsule case at H = 120 (3H x H = 360 x 120, diameter 56 = 7/15 H, 586 vertices at 0.3
    lattice units), both schemes, FP32; and the 16384 x 8192 lattice with open ends and no
    capsules, against the same lattice periodic in x (the cost of the open columns)."""
    import torch

    def timed(ctx, n, scheme):
        ctx.step(warmup, scheme)
        ctx.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(ctx.stream)
        ctx.step(n, scheme)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        ctx.sync()
        return e0.elapsed_time(e1) / n

    out = {"workload": "Section 3.2 open channel: parabolic Zou-He inlet (u_max 0.02), outlet density 1, FP32"}
    for name, scheme in (("dynamic", L.DYNAMIC), ("kinematic", L.KINEMATIC)):
        case = W.open_channel_capsule(scheme=scheme)
        ctx = L.from_case(case, storage="fp32")
        ms = timed(ctx, steps, scheme)
        out[f"capsule_{name}"] = {"lattice": f"{case.nx}x{case.ny}", "vertices": len(case.capsules[0].xy),
                                  "ms_per_step": ms, "mlups": case.nx * case.ny / ms / 1e3}
        ctx.close()
    nx, ny = 16384, 8192
    big = {}
    for key, u_in in (("open", W.inlet_parabola(ny, 0.02)), ("periodic", None)):
        case = W.Case("lattice", nx, ny, 0.7, True, init="rest", u_in=u_in)
        ctx = L.from_case(case, storage="fp32")
        ms = timed(ctx, 100, L.KINEMATIC)
        big[key] = {"ms_per_step": ms, "glups": nx * ny / ms / 1e6}
        ctx.close()
    big["open_cost"] = big["open"]["ms_per_step"] / big["periodic"]["ms_per_step"] - 1.0
    out["lattice_16384x8192"] = big
    return out


def rigid_run(L, steps=200, warmup=20):
    """Rigid particles (Section 2.3.1, Eq. 17-20): the 256 biconcave shapes of the 4096 x 512
    precision workload (seed 0, jittered grid, 128 vertices) as rigid particles of the
    fluid's density, Dynamic, FP32, against the same shapes as deformable capsules."""
    import dataclasses
    import torch

    case = W.poiseuille_biconcave(nx=4096, ny=512, count=256, n=128, seed=0, placement="grid", steps=steps)

    def timed(ctx):
        ctx.step(warmup, L.DYNAMIC)
        ctx.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(ctx.stream)
        ctx.step(steps, L.DYNAMIC)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        ctx.sync()
        return e0.elapsed_time(e1) / steps

    out = {"workload": "4096x512 channel, 256 biconcave shapes x 128 vertices (seed 0), Dynamic, FP32",
           "steps": steps}
    ctx = L.from_case(case, storage="fp32")
    ms = timed(ctx)
    out["deformable"] = {"ms_per_step": ms, "mlups": case.nx * case.ny / ms / 1e3}
    ctx.close()
    ctx = L.from_case(dataclasses.replace(case, capsules=[]), storage="fp32", extra_nodes=case.n_nodes,
                      extra_capsules=len(case.capsules))
    for c in case.capsules:
        A, _, _, J = W.polygon_inertia(c.xy)
        ctx.add_rigid(c.xy, A, J)
    ms = timed(ctx)
    b = ctx.read_rigid(0)
    out["rigid"] = {"ms_per_step": ms, "mlups": case.nx * case.ny / ms / 1e3,
                    "particle0_after": {"c": [b[0], b[1]], "theta": b[2], "u": [b[3], b[4]], "omega": b[5]}}
    ctx.close()
    return out


def batched_run(L, steps, autotune=20):
    """512 independent shear-flow capsule cases (seed 1, uneven sizes and capillary
    numbers) in one persistent launch, FP32, `steps` steps each; against the same cases
    run one after another through single-case contexts (a sample of 32 cases, 300 steps
    each, scaled by lattice updates)."""
    import torch

    cases = W.batch_cases(count=512, seed=1, steps=steps)
    lu = sum(c.nx * c.ny for c in cases)
    b = L.Batch(cases, storage="fp32", autotune_steps=autotune)
    threads, grid, cells = b.config
    s = b.stream
    b.step(steps)          # graph capture at the timed length, warm-up
    b.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    b.step(steps)          # one persistent launch
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    b.sync()
    launches = 1
    b.close()
    seq_ms, seq_lu = 0.0, 0
    for k in range(0, 512, 16):
        c = cases[k]
        ctx = L.from_case(c, storage="fp32")
        ctx.step(300, L.KINEMATIC)
        ctx.sync()
        torch.cuda.synchronize()
        e0.record(ctx.stream)
        ctx.step(300, L.KINEMATIC)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        seq_ms += e0.elapsed_time(e1)
        seq_lu += c.nx * c.ny * 300
        ctx.close()
    mlups = lu * steps / ms / 1e3
    seq_mlups = seq_lu / seq_ms / 1e3
    return {"workload": "512 shear cases, sizes {64..256}^2, Ca in [1e-3, 1e-1], 48-128 vertices, seed 1, "
                        "Kinematic, FP32",
            "steps": steps, "ms": ms, "cases_per_s": 512 / (ms / 1e3), "mlups": mlups,
            "sequential_mlups": seq_mlups, "speedup_vs_sequential": mlups / seq_mlups,
            "launch": {"threads": threads, "ctas": grid, "tile_cells": cells}, "gpu_launches": launches,
            "sequential_sample": "32 cases x 300 steps through single-case contexts (CUDA graphs)"}


def adjoint_run(L, storage, T=800, scheme=1):
    """Gradient of D(T) with respect to (k_s, k_b, g_x) on the 512 x 128 channel capsule
    (radius 16, 128 vertices, Ca = 0.02), Dynamic (1) or Kinematic (0), T steps with a
    checkpoint every 200, against T forward steps of the same context (cost ratio)."""
    import torch

    case = W.adjoint_capsule(scheme=scheme, steps=T)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx = L.from_case(case, storage=storage)
    ctx.step(T, scheme)           # warm-up and graph capture
    ctx.sync()
    torch.cuda.synchronize()
    e0.record(ctx.stream)
    ctx.step(T, scheme)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1)
    ctx.close()
    ctx = L.from_case(case, storage=storage)
    nbytes = L.lbmib_adjoint_workspace_bytes(ctx.h, T, 200)
    work = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    grad = np.zeros(4)
    L.lbmib_adjoint(ctx.h, T, scheme, 200, 0, 0, work.data_ptr(), nbytes, grad)   # warm-up
    ctx.close()
    ctx = L.from_case(case, storage=storage)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J = L.lbmib_adjoint(ctx.h, T, scheme, 200, 0, 0, work.data_ptr(), nbytes, grad)
    adj_ms = (time.perf_counter() - t0) * 1e3
    ctx.close()
    # the same gradient with the whole horizon taped (no segment recompute): the tape of
    # T + 1 population buffers fits easily in HBM at this size
    del work
    ctx = L.from_case(case, storage=storage)
    tbytes = L.lbmib_adjoint_workspace_bytes(ctx.h, T, T)
    work = torch.empty(tbytes, dtype=torch.uint8, device="cuda")
    g2 = np.zeros(4)
    L.lbmib_adjoint(ctx.h, T, scheme, T, 0, 0, work.data_ptr(), tbytes, g2)   # warm-up
    ctx.close()
    ctx = L.from_case(case, storage=storage)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L.lbmib_adjoint(ctx.h, T, scheme, T, 0, 0, work.data_ptr(), tbytes, g2)
    taped_ms = (time.perf_counter() - t0) * 1e3
    ctx.close()
    del work
    return {"workload": "512x128 channel, radius-16 capsule of 128 vertices, Ca 0.02, "
                        + ("Dynamic" if scheme == 1 else "Kinematic") + ", " + storage,
            "steps": T, "ckpt_every": 200, "forward_ms": fwd_ms, "adjoint_ms": adj_ms,
            "cost_ratio": adj_ms / fwd_ms, "J": J,
            "taped": {"adjoint_ms": taped_ms, "cost_ratio": taped_ms / fwd_ms, "workspace_bytes": tbytes,
                      "note": "checkpoint interval = T: the forward writes the tape, no segment recompute"},
            "grad": {"k_s": grad[0], "k_b": grad[1], "g_x": grad[2]},
            "workspace_bytes": nbytes,
            "note": "adjoint_ms: host clock around lbmib_adjoint (forward with checkpoints, recompute, reverse)"}


def e2e_run(a, case, L, scheme, dev):
    """Same metric through the public API with host buffers. Timed: the fields copied
    in from pinned host memory (lbmib_init_fields), the steps (lbmib_step), and the
    fields plus every capsule's observables read back into pinned host memory."""
    import torch

    N = a.nx * a.ny
    rho, ux, uy = case.fields()
    pin = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in (rho, ux, uy)]
    out = [torch.empty((a.ny, a.nx), dtype=torch.float64).pin_memory() for _ in range(3)]
    ncap = len(case.capsules)
    obs = torch.empty((max(ncap, 1), 8), dtype=torch.float64).pin_memory()
    ctx = L.from_case(case, storage=a.storage)

    def once():
        torch.cuda.synchronize()
        t = [time.perf_counter()]
        L.lbmib_init_fields(ctx.h, *[p.numpy() for p in pin])
        t.append(time.perf_counter())
        L.lbmib_step(ctx.h, a.steps, scheme)
        L.lbmib_sync(ctx.h)
        t.append(time.perf_counter())
        L.lbmib_read_fields(ctx.h, *[o.numpy() for o in out])
        if ncap:
            L.lbmib_observables_all(ctx.h, obs.numpy())
        L.lbmib_sync(ctx.h)
        t.append(time.perf_counter())
        return t

    once()   # untimed pass: the step graphs are captured on the first call of a context
    t = once()
    dt = t[-1] - t[0]
    ctx.close()
    h2d = 3 * N * 8
    d2h = 3 * N * 8 + 8 * 8 * ncap
    return {"value": N * a.steps / dt / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": h2d / a.steps, "d2h_bytes_per_step": d2h / a.steps,
            "ms": {"init_fields": 1e3 * (t[1] - t[0]), "steps": 1e3 * (t[2] - t[1]),
                   "read_back": 1e3 * (t[3] - t[2])},
            "note": ("init_fields + step + read_fields + observables_all, host-pinned buffers; the "
                     "second of two passes on one context (the first captures the step graphs)")}


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.impl == "oracle-sample":
        if a.only == "study":
            study_oracle(a.study_oracle_steps, a.study_out)
        else:
            print(json.dumps(oracle_sample(a, steps=a.sample_steps, seconds=a.cpu_seconds, warmup=a.warmup)),
                  flush=True)
    elif a.only != "all":
        import torch

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        from paper_1903_03356_gb300 import lbmib as L

        out = (batched_run(L, a.batch_steps, a.batch_autotune) if a.only == "batched"
               else precision_run(L, int(os.environ.get("LOCAL_RANK", "0"))) if a.only == "precision"
               else dense_run(L) if a.only == "dense"
               else open_run(L) if a.only == "open"
               else rigid_run(L) if a.only == "rigid"
               else precision_study(L, a.study_steps, a.study_oracle_steps) if a.only == "study"
               else poiseuille_runs(L) if a.only == "poiseuille"
               else fp64_coupled_run(L, a, make_case(a), L.DYNAMIC if a.scheme == "dynamic" else L.KINEMATIC,
                                     int(os.environ.get("LOCAL_RANK", "0"))) if a.only == "fp64"
               else {"dynamic": adjoint_run(L, a.storage, a.adjoint_steps, scheme=1),
                     "kinematic": adjoint_run(L, a.storage, a.adjoint_steps, scheme=0)})
        print(json.dumps(out), flush=True)
    else:
        run_gpu(a)


if __name__ == "__main__":
    main()
