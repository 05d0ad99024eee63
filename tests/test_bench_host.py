"""CPU checks of bench.py's host-side logic: the replica time reduction over
two gloo ranks, the reference arm's JSON line, and its silent exit on ranks
other than 0."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, values, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out[rank] = bench.max_over_ranks(values[rank], torch.device("cpu"))
    dist.destroy_process_group()


def test_replica_time_is_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    values = [3.5, 7.25]
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, values, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 7.25


def test_reference_arm_prints_one_line_with_the_contract_keys():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--cpu-moves", "200", "--cpu-workers", "2"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "moves/s"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 2


def test_reference_arm_is_silent_on_other_ranks():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--cpu-moves", "200"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_kernel_traffic_follows_the_sources():
    """The captured DRAM bytes of the --kernels-only calls are reported only
    while the kernels' sources hash to the captured prefix."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench._kernel_traffic("nothing") is None
    for name in ("cell_build_mixture_1m", "trial_energy_mixture_1m", "total_energy_mixture_1m",
                 "energy_grad_262k"):
        assert bench._kernel_traffic(name) > 0, name
    saved = dict(bench.KERNEL_TRAFFIC["cells"])
    try:
        bench.KERNEL_TRAFFIC["cells"]["sha256_prefix"] = "0" * 16
        assert bench._kernel_traffic("cell_build_mixture_1m") is None
    finally:
        bench.KERNEL_TRAFFIC["cells"].update(saved)
