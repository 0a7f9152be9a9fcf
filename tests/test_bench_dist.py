"""Host logic of bench.py's multi-GPU replicas, run as two gloo ranks on the CPU.

With N GPUs the benchmark runs N independent replicas (the lattice is not split; there
is no data-path collective): the job rate is all ranks' units over the slowest rank's
time, taken with an all-reduce MAX.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed = [120.0, 150.0][rank]        # the second rank is slower
    rate, slowest = bench.job_throughput(1e6, elapsed, world, dist, torch.device("cpu"))
    q.put((rank, rate, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_uses_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, rate, slowest in res:
        assert slowest == 150.0
        assert abs(rate - 2 * 1e6 / 0.150) < 1e-6


def test_single_process_needs_no_process_group():
    import bench
    rate, slowest = bench.job_throughput(5e5, 250.0, 1, None)
    assert slowest == 250.0 and abs(rate - 2e6) < 1e-9


def test_reference_arm_prints_the_contract_line():
    # the reference arm is the FP64 oracle on the host: it runs here, without a GPU
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                          "--cpu-seconds", "1"], cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "MLUPS"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    # the line names what ran: the slab sample, its own steps and time per step
    assert line["config"]["workload"].startswith("poiseuille-biconcave-2048x512")
    assert line["config"]["sample_of"].startswith("poiseuille-biconcave-16384x8192")
    assert line["steps"] == 1 and line["cpu_baseline"]["steps"] == 1
    assert abs(line["ms_per_step"] - 2048 * 512 / (line["value"] * 1e6) * 1e3) < 1e-6 * line["ms_per_step"]
    assert line["cpu_baseline"]["nproc"] >= 1 and line["cpu_baseline"]["cpu_model"]
    allc = line["cpu_baseline_all_cores"]
    assert allc["kind"] == "oracle" and allc["cores"] >= 1 and allc["value"] > 0
