#!/usr/bin/env python
"""GCMC moves/s on GB300 -- the benchmark line.

Workload (default): the single-species Lennard-Jones fluid with N = 131,072,
rho* = 0.6 (L = 60.226), rc = 3.0, T* = 1.5, moves 1/3 displace / insert /
delete, max displacement 0.3, 10^6 moves per step, FP32 pair terms with FP64
sums (the FP32-vs-FP64 workload); uniform random start (seeded), synthetic.

One step = the whole hot path once: bin the input into cells, full-system
cell-list energy (the chain's starting energy), 10^6 GCMC moves on the
device, and the full-system gradient (virial) of the final configuration.
value = moves per second of device time over the K timed steps (inputs
resident in HBM; L2 flushed between steps by writing a 256 MiB buffer).
e2e = the same through the public API with the inputs copied from pinned host
memory and the result read back every step.

--impl reference runs the CPU oracle (plain FP64 C) on the host cores as the
reference arm.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GCMC moves/sec at 1 GB300 (FP32+batched vs plain FP64) at ΔE rel err ≤1e-5"
UNIT = "moves/s"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--moves", type=int, default=1_000_000, help="moves per step")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64 comparison run")
    ap.add_argument("--cpu-moves", type=int, default=1_000_000)
    return ap.parse_args()


# ---------------------------------------------------------------- clocks ---

class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- helpers ---

def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def _cpu_baseline(w, n_moves):
    """The oracle as it stands, on one host core, on a bounded sample."""
    import oracle as O
    s = O.System(w.L, w.rc, w.eps, w.sigma)
    s.build(w.positions(), w.types())
    s.set_energy(s.total_energy())
    t0 = time.perf_counter()
    s.run_moves(w.seed, 0, n_moves, w.p_disp, w.p_ins, w.p_del, w.max_disp, w.beta, w.log_z, trace=False)
    dt = time.perf_counter() - t0
    return n_moves / dt, dt


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def run_reference(a):
    """Reference arm: the CPU oracle timed on the host, same workload/metric."""
    ws, rank = _dist()
    if rank != 0:
        return 0
    from paper_1408_3764_gb300 import workloads as W
    import oracle as O
    w = W.c2_fp32_vs_fp64()
    per_step = 200_000
    s = O.System(w.L, w.rc, w.eps, w.sigma)
    s.build(w.positions(), w.types())
    s.set_energy(s.total_energy())
    for k in range(a.warmup):
        s.run_moves(w.seed, k * per_step, per_step, w.p_disp, w.p_ins, w.p_del, w.max_disp, w.beta, w.log_z,
                    trace=False)
    t0 = time.perf_counter()
    for k in range(a.steps):
        s.run_moves(w.seed, (a.warmup + k) * per_step, per_step, w.p_disp, w.p_ins, w.p_del, w.max_disp,
                    w.beta, w.log_z, trace=False)
    dt = time.perf_counter() - t0
    v = a.steps * per_step / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt * 1e3 / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w.name, "n": w.n, "rho": w.rho, "rc": w.rc, "T": w.temperature,
                       "moves_per_step": per_step, "l2": "host"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d moves per step of the %s chain (continuing chain)" % (per_step, w.name)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    a = _args()
    if a.impl == "reference":
        return run_reference(a)
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1408_3764_gb300 import _lib, workloads as W
    from paper_1408_3764_gb300.gcmc import Box, Mix

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    w = W.c2_fp32_vs_fp64()
    M = a.moves
    mix = Mix(w.p_disp, w.p_ins, w.p_del, w.max_disp, w.beta, w.log_z)
    pos_h = torch.from_numpy(w.positions()).pin_memory()
    typ_h = torch.from_numpy(w.types()).pin_memory()
    pos_d = pos_h.to(dev)
    typ_d = typ_h.to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def make_box(precision):
        return Box(w.L, w.rc, w.eps, w.sigma, precision=precision, device=dev)

    box = make_box(a.precision)
    seed = w.seed + 7919 * rank  # replicas: independent chains per rank

    def step(b, k, pos, typ, timers=None):
        b.build_cells(pos, typ)
        b.total_energy()
        if timers is not None:
            timers[0].record(stream)
        st = b.run_moves(seed, k * M, M, mix)
        if timers is not None:
            timers[1].record(stream)
        g = b.energy_grad(want_pos=True)
        return st, g

    # warm-up
    for k in range(a.warmup):
        step(box, k, pos_d, typ_d)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    launches0 = box.launches()
    times, chain_times = [], []
    last = None
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(a.steps):
            flush.fill_(k & 0xFF)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            c = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            e0.record(stream)
            last = step(box, a.warmup + k, pos_d, typ_d, timers=c)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            chain_times.append(c[0].elapsed_time(c[1]))
        torch.cuda.synchronize()
    launches = box.launches() - launches0
    counters = box.chain_counters()
    total_ms = sum(times)
    if ws > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = ws * a.steps * M / (total_ms / 1e3)

    # end to end through the public API: host inputs, result read back
    e2e_box = make_box(a.precision)
    for k in range(1):
        step(e2e_box, k, pos_h.to(dev, non_blocking=True), typ_h.to(dev, non_blocking=True))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2d = d2h = 0
    for k in range(a.steps):
        pd = pos_h.to(dev, non_blocking=True)
        td = typ_h.to(dev, non_blocking=True)
        h2d += pd.numel() * 8 + td.numel() * 4
        st, g = step(e2e_box, a.warmup + k, pd, td)
        res = torch.tensor([st["energy"], g["virial"]]).numpy()  # stats arrive on the host
        d2h += 8 * 2 + 8 * 13
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": a.steps * M / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d // a.steps,
           "d2h_bytes_per_step": d2h // a.steps}

    # latency floor of one chain (roofline of the dominant kernel)
    probe = _lib.ProbeResult()
    import ctypes as C
    st_ws = 8 << 20
    rc = _lib.load().gcmc_probe_latency(C.c_void_p(stream.cuda_stream), st_ws, C.byref(probe))
    chain_ms = sum(chain_times) / len(chain_times)
    achieved = M / (chain_ms / 1e3)
    peak = 1e9 / probe.floor_ns if rc == 0 and probe.floor_ns > 0 else None
    roofline = {"bound": "latency", "achieved": achieved, "peak": peak, "unit": UNIT,
                "frac": (achieved / peak) if peak else None, "traffic": None,
                "kernel": "k_chain", "floor_ns": probe.floor_ns,
                "floor_parts_ns": {"l2_hop": probe.l2_hop_ns, "sync_round": probe.sync_round_ns,
                                   "philox": probe.philox_ns, "log": probe.log_ns},
                "peak_source": "measured by gcmc_probe_latency in this run (2 dependent L2 hops + "
                               "CTA reduction/broadcast + Philox + FP64 log)"}

    compare = {}
    if not a.no_compare and rank == 0:
        other = "fp64" if a.precision == "fp32" else "fp32"
        b2 = make_box(other)
        step(b2, 0, pos_d, typ_d)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        c = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        flush.fill_(1)
        e0.record(stream)
        st2, _ = step(b2, 1, pos_d, typ_d, timers=c)
        e1.record(stream)
        e1.synchronize()
        compare = {"%s_moves_per_s" % other: M / (e0.elapsed_time(e1) / 1e3),
                   "%s_chain_moves_per_s" % other: M / (c[0].elapsed_time(c[1]) / 1e3)}

    cpu = None
    if rank == 0 and not a.no_cpu_baseline:
        v, dt = _cpu_baseline(w, a.cpu_moves)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "first %d moves of the %s chain, FP64 oracle, 1 core (%.1f s)" % (a.cpu_moves, w.name, dt)}

    if rank == 0:
        st = last[0]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if a.precision == "fp32" else "f64",
                "data": "synthetic",
                "config": {"workload": w.name, "n": w.n, "rho": w.rho, "L": w.L, "rc": w.rc, "T": w.temperature,
                           "moves_per_step": M, "mix": [w.p_disp, w.p_ins, w.p_del], "max_disp": w.max_disp,
                           "precision": a.precision, "l2": "flushed (256 MiB write) between steps",
                           "parallelism": "replicas" if ws > 1 else "single chain"},
                "chain_moves_per_s": achieved,
                "acceptance": [st["accepted"][i] / max(1, st["attempted"][i]) for i in range(3)],
                "final_n": st["n"], "flagged": st["flagged"], "chain_counters_last_step": counters,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk.summary(), "compare": compare}
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
