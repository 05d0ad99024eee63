#!/usr/bin/env python
"""GCMC moves/s on GB300 -- the benchmark line.

Workload (default, ``--workload isotherm``): the batched isotherm -- 64
independent single-species Lennard-Jones chains, N0 log-uniform in
[500, 20000], rho* 0.1 .. 0.7, ln z interpolated along the isotherm, rc 2.5,
T* 1.2, moves 1/3 displace / insert / delete, max displacement 0.3; FP32 pair
terms (compensated) with FP64 sums and FP64 Metropolis decisions; 10^5 moves
per chain per step, all chains in one graph-replayed launch with the team
shape picked by the online tuner.  The first step starts from seeded uniform
random positions (synthetic); every later step starts from the configuration
the previous step left (exported and binned again), so the timed steps run
chains that have relaxed for the warm-up steps' moves.

One step = the whole hot path once over every chain: bin the configuration
into cells and take the full-system cell-list energy (the chain's starting
energy) for all boxes in one batched call, 10^5 GCMC moves per chain on the
device, the full-system gradient (forces, virial) of every final
configuration in one batched call, and the export of the configuration for
the next step.  value = moves of all chains per second of device time over
the K timed steps (inputs resident in HBM; L2 flushed between steps by
writing a 256 MiB buffer).  e2e = the same through the public API with each
step's configuration copied in from pinned host memory and its forces and
final configuration read back every step.

Also reported: the precision of the FP32 chain against the FP64 oracle
(computed from the CPU baseline's sample: every move of 64 chains x 20,000
moves from the initial configurations, the 2,048-particle chain, 10^6 moves
of the 131,072-particle chain with its energy drift, and the FP32
full-system energies of the 131,072-particle and million-particle boxes),
the plain FP64 single chain (the 2,048-particle workload), the
131,072-particle chain in FP32 and FP64, the batched isotherm in FP64 and
with the running virial, the same single chains over the microcell list
(Sec. 3.3), the throughput kernels (trial energies, full-system energy,
gradient, cell build) of the million-particle mixture and the
262,144-particle gradient workload against measured pipe peaks, and the
cutoff sweep (one 87,296-particle chain per cutoff, rc 2.5 .. 4.25, FP32,
FP64 and microcells).  --kernels-only and --micro-only print just those
figures; --no-compare / --no-kernels / --no-sweep / --no-cpu-baseline /
--no-precision skip parts of the default run.

--impl reference runs the CPU oracle (plain FP64 C) on the host cores as the
reference arm, on the same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import math
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
FLUSH_BYTES = 256 << 20
# DRAM bytes (read + write) of one full-size chain launch (64 chains x 10^5
# moves) from an ncu capture (profiles/k_chain_isotherm_fp32.md), valid for
# the chain kernel source with this sha256 prefix only (captured with the
# source 19137a71284994a4, which differs from this one in comments only)
CHAIN_TRAFFIC = {"sha256_prefix": "fb1ab48a525325ae", "bytes": 19.05e6, "moves": 6.4e6}
# DRAM bytes (read + write, summed over the call's launches) of the timed calls
# of --kernels-only from one ncu capture (profiles/cell_build_mixture_1m.md),
# valid for the sources whose joint sha256 has this prefix
KERNEL_TRAFFIC = {
    "cells": {"sources": ("gcmc_cells.cu", "gcmc_device.cuh"), "sha256_prefix": "820ee9a4c2fb519e",
              "bytes": {"cell_build_mixture_1m": 115.4e6}},
    "energy": {"sources": ("gcmc_energy.cu", "gcmc_stage.cuh", "gcmc_device.cuh"),
               "sha256_prefix": "13f89e1759c1ac26",
               "bytes": {"trial_energy_mixture_1m": 151.6e6, "total_energy_mixture_1m": 17.97e6,
                         "energy_grad_262k": 6.39e6}},
}
DEFAULT_MOVES = {"isotherm": 100_000, "c2": 1_000_000, "c1": 10_000}
DEFAULT_CPU_MOVES = {"isotherm": 20_000, "c2": 1_000_000, "c1": 10_000}


def _kernel_traffic(name):
    """The captured DRAM bytes of a --kernels-only call, or None when its
    sources changed since the capture."""
    import hashlib
    for ref in KERNEL_TRAFFIC.values():
        if name not in ref["bytes"]:
            continue
        h = hashlib.sha256()
        try:
            for f in ref["sources"]:
                with open(os.path.join(ROOT, "paper_1408_3764_gb300", "csrc", f), "rb") as fh:
                    h.update(fh.read())
        except OSError:
            return None
        return ref["bytes"][name] if h.hexdigest().startswith(ref["sha256_prefix"]) else None
    return None


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="isotherm", choices=["isotherm", "c2", "c1"])
    ap.add_argument("--moves", type=int, default=0, help="moves per chain per step (0: the workload's)")
    ap.add_argument("--precision", default="", choices=["", "fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision", action="store_true", help="skip the precision figures against the oracle")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-kernels", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="skip the cutoff sweep figures")
    ap.add_argument("--micro-only", action="store_true",
                    help="only the microcell chain's single-chain rates (moves per chain: --moves, default 10^5)")
    ap.add_argument("--sweep-moves", type=int, default=100_000, help="moves per cutoff and precision")
    ap.add_argument("--kernels-only", action="store_true",
                    help="only the throughput kernels (trial energies, total energy, gradient, cell build)")
    ap.add_argument("--cpu-moves", type=int, default=0, help="oracle moves per chain in the CPU sample")
    ap.add_argument("--cpu-workers", type=int, default=0)
    a = ap.parse_args()
    if not a.moves:
        a.moves = DEFAULT_MOVES[a.workload]
    if not a.cpu_moves:
        a.cpu_moves = DEFAULT_CPU_MOVES[a.workload]
    if not a.precision:
        a.precision = "fp64" if a.workload == "c1" else "fp32"
    return a


def _chains(name):
    from paper_1408_3764_gb300 import workloads as W
    if name == "isotherm":
        return W.isotherm_chains()
    if name == "c2":
        return [W.c2_fp32_vs_fp64()]
    return [W.c1_plain_fp64()]


def _workload_config(name, chains, M, precision):
    ns = [w.n for w in chains]
    cfg = {"workload": {"isotherm": "batched isotherm: 64 LJ chains, N0 500-20000, rho 0.1-0.7",
                        "c2": "single-species LJ, N=131072, rho 0.6, rc 3.0, T 1.5",
                        "c1": "plain single-species LJ, N=2048, rho 0.5, rc 2.5, T 1.2"}[name],
           "chains": len(chains), "n0_total": int(sum(ns)), "n0_min": int(min(ns)), "n0_max": int(max(ns)),
           "rho": [round(chains[0].rho, 4), round(chains[-1].rho, 4)], "rc": chains[0].rc,
           "T": chains[0].temperature, "moves_per_chain_per_step": M,
           "mix": [chains[0].p_disp, chains[0].p_ins, chains[0].p_del], "max_disp": chains[0].max_disp,
           "precision": precision, "l2": "flushed (256 MiB write) between steps"}
    return cfg


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


# ------------------------------------------------------------ CPU oracle ---

def _oracle_chain_step(k_chain, workload, first, n_moves, want_trace=False):
    """One step of the hot path for chain k on the CPU oracle: bin, total
    energy, n_moves moves, gradient.  Returns (moves, seconds, trace, sum|u|):
    the per-move records and sums of |u_j| when asked (the CPU baseline's
    sample doubles as the reference of the precision figures)."""
    import oracle as O
    w = _chains(workload)[k_chain]
    t0 = time.perf_counter()
    s = O.System(w.L, w.rc, w.eps, w.sigma)
    s.build(w.positions(), w.types())
    s.set_energy(s.total_energy())
    res = s.run_moves(w.seed, first, n_moves, w.p_disp, w.p_ins, w.p_del, w.max_disp, w.beta, w.log_z,
                      chain=k_chain if workload == "isotherm" else 0, trace=want_trace, with_sabs=want_trace)
    s.energy_grad()
    dt = time.perf_counter() - t0
    if want_trace:
        return n_moves, dt, res[0], res[2]
    return n_moves, dt, None, None


def _oracle_chain_trace(wl_name, n_moves, relax=0):
    """The oracle's trace of a single chain (the 2,048- or the 131,072-particle
    workload): `relax` moves first, then the running energy is reset to the
    full-system energy and n_moves moves are recorded.  Returns (trace,
    sum|u|, starting energy, running energy after, full-system energy of
    the final configuration, particle count after)."""
    import oracle as O
    from paper_1408_3764_gb300 import workloads as W
    w = W.c1_plain_fp64() if wl_name == "c1" else W.c2_fp32_vs_fp64()
    s = O.System(w.L, w.rc, w.eps, w.sigma)
    s.build(w.positions(), w.types())
    s.set_energy(s.total_energy())
    args = (w.p_disp, w.p_ins, w.p_del, w.max_disp, w.beta, w.log_z)
    if relax:
        s.run_moves(w.seed, 0, relax, *args, tol=1e-5, trace=False)
        s.set_energy(s.total_energy())
    e0 = s.energy()
    tr, st, sabs = s.run_moves(w.seed, relax, n_moves, *args, tol=1e-5, with_sabs=True)
    return tr, sabs, e0, st.energy, s.total_energy(), int(sum(st.n[:1]))


def _oracle_total_energy(wl_name):
    """The oracle's full-system energy of a workload's initial configuration."""
    import oracle as O
    from paper_1408_3764_gb300 import workloads as W
    w = W.c2_fp32_vs_fp64() if wl_name == "c2" else W.c3_mixture_1m()
    s = O.System(w.L, w.rc, w.eps, w.sigma)
    s.build(w.positions(), w.types())
    return s.total_energy()


class OraclePool:
    """The oracle's chains spread over host processes (spawned, so that no
    worker inherits a CUDA context)."""

    def __init__(self, workload, workers):
        import concurrent.futures as cf
        import multiprocessing as mp
        self.workload = workload
        self.n_chains = len(_chains(workload))
        self.workers = max(1, workers)
        self.ex = cf.ProcessPoolExecutor(self.workers, mp_context=mp.get_context("spawn"))
        # start the workers (imports, oracle load) outside any timed region
        list(self.ex.map(_oracle_chain_step, [0] * self.workers, [workload] * self.workers,
                         [0] * self.workers, [1] * self.workers))

    def step(self, first, n_moves, want_trace=False):
        """One bounded sample of the workload's step on the host cores:
        (moves, seconds, per-chain traces and sums of |u_j| or None)."""
        t0 = time.perf_counter()
        ks = list(range(self.n_chains))
        # largest chains first for a balanced finish
        ns = [w.n for w in _chains(self.workload)]
        ks.sort(key=lambda k: -ns[k])
        futs = {k: self.ex.submit(_oracle_chain_step, k, self.workload, first, n_moves, want_trace) for k in ks}
        res = {k: f.result() for k, f in futs.items()}
        dt = time.perf_counter() - t0
        traces = [(res[k][2], res[k][3]) for k in range(self.n_chains)] if want_trace else None
        return sum(r[0] for r in res.values()), dt, traces

    def submit(self, fn, *args):
        return self.ex.submit(fn, *args)

    def close(self):
        self.ex.shutdown()


def _cpu_workers(a):
    if a.cpu_workers:
        return a.cpu_workers
    try:
        n = len(os.sched_getaffinity(0))
    except Exception:
        n = os.cpu_count() or 1
    return max(1, min(16, n))


def max_over_ranks(x: float, device) -> float:
    """The largest of x over the ranks of the default process group (the
    job's time is its slowest replica's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def run_reference(a):
    """Reference arm: the CPU oracle timed on the host cores, same workload
    and metric; each step is a bounded sample of the workload's step."""
    ws, rank = _dist()
    if rank != 0:
        return 0
    chains = _chains(a.workload)
    pool = OraclePool(a.workload, min(_cpu_workers(a), len(chains)))
    M = a.cpu_moves
    for k in range(a.warmup):
        pool.step(k * M, M)
    tot_moves, tot_s = 0, 0.0
    for k in range(a.steps):
        m, dt, _ = pool.step((a.warmup + k) * M, M)
        tot_moves += m
        tot_s += dt
    pool.close()
    v = tot_moves / tot_s
    sample = ("%d chain(s) x %d moves per step (bin + total energy + moves + gradient per chain), "
              "FP64 oracle, %d worker process(es)" % (len(chains), M, pool.workers))
    cfg = _workload_config(a.workload, chains, M, "fp64")
    cfg["l2"] = "host"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": tot_s * 1e3 / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded uniform random positions)", "config": cfg,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": pool.workers, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------- GPU side ---

class Runner:
    """The chains of one workload on the GPU, and one step of the hot path.

    Every box has its own CUDA stream.  A step bins each chain's current
    configuration and takes its energy (one batched call for all boxes), runs
    the moves (one launch), takes the gradient (one batched call) and exports
    the final configuration as the next step's input.  host_inputs: each
    step's configuration comes from pinned host memory and the forces and
    the final configuration go back there (the end-to-end measurement)."""

    def __init__(self, chains, precision, dev, rank, host_inputs=False, virial=False):
        import torch
        from paper_1408_3764_gb300.gcmc import Batch, Box, Mix
        self.torch = torch
        self.chains = chains
        self.dev = dev
        self.stream = torch.cuda.current_stream(dev)
        self.box_streams = [torch.cuda.Stream(device=dev) for _ in chains]
        self.boxes = [Box(w.L, w.rc, w.eps, w.sigma, precision=precision, device=dev, stream=s)
                      for w, s in zip(chains, self.box_streams)]
        self.mixes = [Mix(w.p_disp, w.p_ins, w.p_del, w.max_disp, w.beta, w.log_z, virial=virial) for w in chains]
        self.seeds = [w.seed + 7919 * rank for w in chains]  # replicas: independent chains per rank
        self.batch = Batch(self.boxes)
        self.host_inputs = host_inputs
        self.pos, self.typ, self.dpos, self.pos_h, self.typ_h, self.dpos_h = [], [], [], [], [], []
        for w in chains:
            self._alloc(2 * w.n + 1024)
        self.reset()
        self.chain_ms = 0.0
        self.h2d_bytes = 0
        self.d2h_bytes = 0

    def _alloc(self, cap, k=None):
        torch = self.torch
        bufs = (torch.empty((cap, 3), dtype=torch.float64, device=self.dev),
                torch.empty(cap, dtype=torch.int32, device=self.dev),
                torch.empty((cap, 3), dtype=torch.float32, device=self.dev))
        hb = (None, None, None)
        if self.host_inputs:
            hb = (torch.empty((cap, 3), dtype=torch.float64).pin_memory(),
                  torch.empty(cap, dtype=torch.int32).pin_memory(),
                  torch.empty((cap, 3), dtype=torch.float32).pin_memory())
        if k is None:
            for lst, v in zip((self.pos, self.typ, self.dpos, self.pos_h, self.typ_h, self.dpos_h), bufs + hb):
                lst.append(v)
        else:
            for lst, v in zip((self.pos, self.typ, self.dpos, self.pos_h, self.typ_h, self.dpos_h), bufs + hb):
                old = lst[k]
                if old is not None:
                    v[: old.shape[0]].copy_(old)
                lst[k] = v

    def reset(self):
        """Back to the workload's initial (seeded uniform random) configurations."""
        torch = self.torch
        self.n = []
        for k, w in enumerate(self.chains):
            p = torch.from_numpy(w.positions())
            t = torch.from_numpy(w.types())
            self.pos[k][: w.n].copy_(p)
            self.typ[k][: w.n].copy_(t)
            if self.host_inputs:
                self.pos_h[k][: w.n].copy_(p)
                self.typ_h[k][: w.n].copy_(t)
            self.n.append(w.n)
        torch.cuda.synchronize(self.dev)

    def launches(self):
        return sum(b.launches() for b in self.boxes) + self.batch.launches()

    def step(self, k, M):
        torch = self.torch
        K = len(self.boxes)
        if self.host_inputs:
            for i in range(K):
                with torch.cuda.stream(self.box_streams[i]):
                    n = self.n[i]
                    self.pos[i][:n].copy_(self.pos_h[i][:n], non_blocking=True)
                    self.typ[i][:n].copy_(self.typ_h[i][:n], non_blocking=True)
                    self.h2d_bytes += n * (3 * 8 + 4)
        energies = self.batch.prepare([self.pos[i][: self.n[i]] for i in range(K)],
                                      [self.typ[i][: self.n[i]] for i in range(K)])
        stats = self.batch.run_moves(self.seeds, k * M, M, self.mixes)
        self.chain_ms = self.batch.device_ms()
        N = [int(sum(st["n"])) for st in stats]
        for i in range(K):
            if N[i] > self.pos[i].shape[0]:  # rare: a chain grew past its buffers
                self._alloc(2 * N[i] + 1024, i)
        eg, wg = self.batch.energy_grad([self.dpos[i][: N[i]] for i in range(K)])
        self.batch.export_positions(self.pos, self.typ)
        self.n = list(N)
        if self.host_inputs:
            for i in range(K):
                with torch.cuda.stream(self.box_streams[i]):
                    n = N[i]
                    self.pos_h[i][:n].copy_(self.pos[i][:n], non_blocking=True)
                    self.typ_h[i][:n].copy_(self.typ[i][:n], non_blocking=True)
                    self.dpos_h[i][:n].copy_(self.dpos[i][:n], non_blocking=True)
                    self.d2h_bytes += n * (3 * 8 + 4 + 3 * 4)
            for st_ in self.box_streams:
                st_.synchronize()
        else:
            for st_ in self.box_streams:
                self.stream.wait_stream(st_)
        return stats, (eg, wg), energies

    def close(self):
        self.batch.close()


def _time_steps(runner, first_step, steps, M, flush):
    torch = runner.torch
    times, chain = [], []
    last = None
    for k in range(steps):
        flush.fill_(k & 0xFF)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(runner.stream)
        runner.stream.synchronize()  # the flush is done before any box stream starts
        last = runner.step(first_step + k, M)
        e1.record(runner.stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        chain.append(runner.chain_ms)
    return times, chain, last


def _single_chain_rate(w, precision, M, dev, flush):
    """Moves/s of one chain (device time of the chain kernel) after a warm-up step."""
    r = Runner([w], precision, dev, 0)
    r.step(0, min(M, 20_000))
    times, chain, _ = _time_steps(r, 1, 1, M, flush)
    r.close()
    return {"moves_per_s": M / (chain[0] / 1e3), "step_moves_per_s": M / (times[0] / 1e3), "moves": M,
            "precision": precision, "n": w.n}


def _micro_chain_rate(w, precision, M, dev, flush):
    """Moves/s of one chain evaluated over the microcell list (Sec. 3.3; device
    time of the chain launch) after a warm-up run of 20,000 moves."""
    import torch
    from paper_1408_3764_gb300.gcmc import Box, Mix
    b = Box(w.L, w.rc, w.eps, w.sigma, precision=precision, device=dev)
    mix = Mix(w.p_disp, w.p_ins, w.p_del, w.max_disp, w.beta, w.log_z)
    pos = torch.from_numpy(w.positions()).to(dev)
    typ = torch.from_numpy(w.types()).to(dev)
    b.build_cells(pos, typ)
    b.build_microcells(1.0)
    b.run_moves_micro(w.seed, 0, min(M, 20_000), mix)
    b.build_cells(pos, typ)
    b.total_energy()
    b.build_microcells(1.0)
    flush.fill_(3)
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.run_moves_micro(w.seed + 1, 0, M, mix)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    return {"moves_per_s": M / (ms / 1e3), "moves": M, "precision": precision, "n": w.n,
            "microcells_per_side": b.microcells()[0]}


def _du_err(tg, to, sabs):
    """Per-move err = |dU_gpu - dU_oracle| / max(|dU_oracle|, 1e-3 sum_j |u_j|)
    over the moves before the first decision that differs (0 where no pair
    lies within the cutoff on either side); and the number of moves compared."""
    import numpy as np
    n = len(to)
    same = np.ones(n, bool)
    for k in ("type", "species", "index", "accepted"):
        same &= tg[k] == to[k]
    stop = n if same.all() else int(np.argmin(same))
    tg, to, sabs = tg[:stop], to[:stop], sabs[:stop]
    ok = np.isfinite(to["lnA"]) & np.isfinite(to["dU"])
    den = np.maximum(np.abs(to["dU"]), 1e-3 * sabs)
    err = np.zeros(stop)
    nz = ok & (den > 0)
    err[nz] = np.abs(tg["dU"][nz] - to["dU"][nz]) / den[nz]
    return err, stop


def _err_summary(err, n_total, decisions_identical):
    import numpy as np
    return {"moves": int(n_total), "max": float(err.max()) if err.size else 0.0,
            "p99_99": float(np.quantile(err, 0.9999)) if err.size else 0.0,
            "frac_above_1e-5": float((err > 1e-5).mean()) if err.size else 0.0,
            "frac_above_1e-12": float((err > 1e-12).mean()) if err.size else 0.0,
            "identical_decisions": bool(decisions_identical)}


def _precision(dev, pool, iso_traces, iso_moves, c1_fut, c2_fut, tot_futs):
    """The FP32 path against the FP64 oracle (per-move dU error, full-system
    energy error, running-energy drift) on the same seeded inputs: the GPU
    runs the oracle sample's moves again with traces (untimed)."""
    import numpy as np
    import torch
    from paper_1408_3764_gb300 import workloads as W
    from paper_1408_3764_gb300.gcmc import Batch, Box, Mix
    out = {"measure": "|dU_gpu - dU_oracle| / max(|dU_oracle|, 1e-3 sum_j |u_j|), every move",
           "precision": "fp32 (compensated pair terms)"}
    # the isotherm sample: 64 chains x iso_moves from the initial configurations
    chains = W.isotherm_chains()
    boxes = [Box(w.L, w.rc, w.eps, w.sigma, precision="fp32", device=dev) for w in chains]
    for b, w in zip(boxes, chains):
        b.build_cells(torch.from_numpy(w.positions()).to(dev), torch.from_numpy(w.types()).to(dev))
    batch = Batch(boxes)
    mixes = [Mix(w.p_disp, w.p_ins, w.p_del, w.max_disp, w.beta, w.log_z) for w in chains]
    _, tg = batch.run_moves([w.seed for w in chains], 0, iso_moves, mixes, trace=True)
    errs, same, n = [], True, 0
    for k in range(len(chains)):
        to, sabs = iso_traces[k]
        e, stop = _du_err(tg[k], to, sabs)
        errs.append(e)
        same &= stop == len(to)
        n += len(to)
    out["isotherm_64_chains"] = _err_summary(np.concatenate(errs), n, same)
    batch.close()
    del boxes
    # the 2,048-particle chain, 10^4 moves
    w1 = W.c1_plain_fp64()
    b1 = Box(w1.L, w1.rc, w1.eps, w1.sigma, precision="fp32", device=dev)
    b1.build_cells(torch.from_numpy(w1.positions()).to(dev), torch.from_numpy(w1.types()).to(dev))
    _, t1 = b1.run_moves(w1.seed, 0, w1.moves, Mix(w1.p_disp, w1.p_ins, w1.p_del, w1.max_disp, w1.beta, w1.log_z),
                         trace=True)
    to1, sabs1 = c1_fut.result()[:2]
    e1, stop1 = _du_err(t1, to1, sabs1)
    out["plain_2048_10k"] = _err_summary(e1, len(to1), stop1 == len(to1))
    # the 131,072-particle chain: 10^5 moves of relaxation, then 10^6 moves
    w2 = W.c2_fp32_vs_fp64()
    b2 = Box(w2.L, w2.rc, w2.eps, w2.sigma, precision="fp32", device=dev)
    b2.build_cells(torch.from_numpy(w2.positions()).to(dev), torch.from_numpy(w2.types()).to(dev))
    e_init_gpu = b2.total_energy()
    mix2 = Mix(w2.p_disp, w2.p_ins, w2.p_del, w2.max_disp, w2.beta, w2.log_z)
    b2.run_moves(w2.seed, 0, 100_000, mix2)
    e_start_gpu = b2.total_energy()
    to2, sabs2, e_start, e_run_o, e_final, n_final = c2_fut.result()
    # both running energies start from the oracle's full-system energy of
    # the relaxed configuration, so that the drifts compare the chains alone
    b2.restore(*b2.get_state()[:4], energy=e_start)
    st2, t2 = b2.run_moves(w2.seed, 100_000, 1_000_000, mix2, trace=True)
    e2, stop2 = _du_err(t2, to2, sabs2)
    out["n131072_1M"] = _err_summary(e2, len(to2), stop2 == len(to2))
    acc = to2["accepted"] == 1
    scale = float(np.abs(to2["dU"][acc]).sum())
    out["n131072_1M"]["drift"] = {
        "definition": "running energy after the 10^6 moves minus the oracle's full-system energy of the final "
                      "configuration; both chains start from the oracle's full-system energy of the configuration "
                      "10^5 moves after the uniform start (its remaining overlaps make that energy ~1e20, so FP64 "
                      "rounding of the running sums dominates both drifts); gpu_minus_oracle_running is the FP32 "
                      "path's own share",
        "gpu": st2["energy"] - e_final, "oracle": e_run_o - e_final,
        "gpu_minus_oracle_running": st2["energy"] - e_run_o,
        "gpu_minus_oracle_running_over_sum_abs_dU": (st2["energy"] - e_run_o) / scale if scale else None,
        "start_energy": e_start, "gpu_fp32_start_energy_rel_err": (e_start_gpu - e_start) / abs(e_start),
        "final_energy": e_final, "n_final": n_final}
    # full-system energies of the initial configurations (FP32 path)
    e_c2 = tot_futs["c2"].result()
    out["total_energy_131072"] = {"gpu_fp32": e_init_gpu, "oracle": e_c2,
                                  "rel_err": abs(e_init_gpu - e_c2) / abs(e_c2)}
    w3 = W.c3_mixture_1m()
    b3 = Box(w3.L, w3.rc, w3.eps, w3.sigma, precision="fp32", device=dev)
    b3.build_cells(torch.from_numpy(w3.positions()).to(dev), torch.from_numpy(w3.types()).to(dev))
    e3 = b3.total_energy()
    e_c3 = tot_futs["c3"].result()
    out["total_energy_mixture_1m"] = {"gpu_fp32": e3, "oracle": e_c3, "rel_err": abs(e3 - e_c3) / abs(e_c3)}
    return out


def _cutoff_sweep(dev, flush, M):
    """One chain of 87,296 particles in 131,072 sigma^3 at each cutoff of the
    sweep, FP32 and FP64: chain moves/s (device time of the chain launch), the
    27-cell candidates and the within-cutoff partners of a trial point."""
    from paper_1408_3764_gb300 import workloads as W
    out = {}
    for rc in W.SWEEP_RC:
        w = W.cutoff_sweep(rc)
        T = max(3, int(w.L // rc))
        row = {"T": T, "candidates_per_point": 27.0 * w.n / T ** 3,
               "pairs_in_rc_per_point": 4.0 / 3.0 * math.pi * rc ** 3 * w.rho}
        for prec in ("fp32", "fp64"):
            r = _single_chain_rate(w, prec, M, dev, flush)
            row[prec + "_moves_per_s"] = r["moves_per_s"]
        # the paper's microcell list: cube of (2D+1)^3 microcells of edge ~sigma
        row["micro_fp32_moves_per_s"] = _micro_chain_rate(w, "fp32", M, dev, flush)["moves_per_s"]
        out["%.2f" % rc] = row
    base = out["%.2f" % W.SWEEP_RC[0]]
    for row in out.values():
        row["fp32_rate_vs_rc2.5"] = row["fp32_moves_per_s"] / base["fp32_moves_per_s"]
    return {"workload": "lj-87296-V131072 (rho 0.666), T* 1.5, one chain, %d moves per point" % M,
            "rc": out}


def _pipe_peaks(stream_ptr):
    """Measured FP32 / FP64 FMA and special-function (reciprocal) throughput
    and the SM count of the device (gcmc_probe_pipes); the HBM copy peak
    from MEASURED_PEAKS.json when present."""
    import ctypes as C
    from paper_1408_3764_gb300 import _lib
    pk = _lib.PipePeaks()
    rc = _lib.load().gcmc_probe_pipes(C.c_void_p(stream_ptr), C.byref(pk))
    out = {"fp32_tflops": pk.fp32_tflops, "fp64_tflops": pk.fp64_tflops, "mufu_gops": pk.mufu_gops,
           "sms": int(pk.sms), "source": "measured in this run by gcmc_probe_pipes" if rc == 0 else "probe failed"}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            out["hbm_gbs"] = float(json.load(f)["hbm_gbs"])
            out["hbm_source"] = "MEASURED_PEAKS.json (measured copy bandwidth)"
    except (OSError, KeyError, ValueError):
        out["hbm_gbs"], out["hbm_source"] = 6800.0, "fallback (no measured figure)"
    return out


def _kernel_figures(dev, flush, peaks):
    """Throughput kernels on the million-particle mixture and the gradient
    workload: trial energies, full-system energy, gradient, cell build."""
    import torch
    from paper_1408_3764_gb300 import workloads as W
    from paper_1408_3764_gb300.gcmc import Box, Mix
    out = {}
    fp32_peak = peaks["fp32_tflops"]

    def ev_time(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    w = W.c3_mixture_1m()
    pos = torch.from_numpy(w.positions()).to(dev)
    typ = torch.from_numpy(w.types()).to(dev)
    b = Box(w.L, w.rc, w.eps, w.sigma, precision="fp32", device=dev)
    ms_build = ev_time(lambda: b.build_cells(pos, typ))
    b.build_cells(pos, typ)
    # relaxed by 10^4 displacements, as the workload states
    b.run_moves(w.seed, 0, 10_000, Mix(1.0, 0.0, 0.0, w.max_disp, w.beta, w.log_z))
    g = b.geometry()
    ncell, N = g["n_cells"], w.n
    rho = N / w.L ** 3
    cand = 27.0 * N / ncell                       # candidates per trial point (27 cells)
    inr = 4.0 / 3.0 * math.pi * w.rc ** 3 * rho  # partners within rc per point
    m = 1_000_000
    tp, ts = W.insertion_points(m, w.L, 2, 7)
    tpd = torch.from_numpy(tp).to(dev)
    tsd = torch.from_numpy(ts).to(dev)
    tout = torch.empty(m, dtype=torch.float64, device=dev)
    b.trial_energy_raw(tpd, tsd, tout)
    ms_trial = ev_time(lambda: b.trial_energy_raw(tpd, tsd, tout))
    ms_total = ev_time(lambda: b.total_energy())

    # algorithmic work: pairs within the cutoff only (the other candidates of
    # the 27 cells are overhead), 20 FLOP per pair forward, 30 backward
    def alu(pairs, flop_per_pair, ms):
        ach = pairs * flop_per_pair / (ms / 1e3) / 1e12
        return {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak,
                "traffic": None, "flop_model": "%d per pair within rc" % flop_per_pair,
                "peak_source": "FP32 FMA throughput " + peaks["source"]}

    out["trial_energy_mixture_1m"] = {"points": m, "ms": ms_trial, "points_per_s": m / (ms_trial / 1e3),
                                      "candidates_per_point": cand, "pairs_in_rc_per_point": inr,
                                      "roofline": alu(m * inr, 20, ms_trial)}
    out["total_energy_mixture_1m"] = {"particles": N, "ms": ms_total, "unique_pairs_in_rc": N * inr / 2,
                                      "roofline": alu(N * inr / 2, 20, ms_total)}
    # the cell build moves 16 B in (FP64 positions are 24 B, species 4 B) and
    # 16 B out per particle for each layout written, plus 8 B of index traffic:
    # 28 + 2 * 16 + 8 = 68 B per particle as algorithmic bytes
    gbs = N * 68 / (ms_build / 1e3) / 1e9
    out["cell_build_mixture_1m"] = {"particles": N, "ms": ms_build, "particles_per_s": N / (ms_build / 1e3),
                                    "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"],
                                                 "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"], "traffic": None,
                                                 "byte_model": "68 B per particle (28 in, 2 x 16 out, 8 index)",
                                                 "peak_source": peaks["hbm_source"]}}
    del b, tpd, tsd, tout
    w5 = W.c5_gradient()
    b5 = Box(w5.L, w5.rc, w5.eps, w5.sigma, precision="fp32", device=dev)
    b5.build_cells(torch.from_numpy(w5.positions()).to(dev), torch.from_numpy(w5.types()).to(dev))
    ms_grad = ev_time(lambda: b5.energy_grad(want_pos=True))
    inr5 = 4.0 / 3.0 * math.pi * w5.rc ** 3 * (w5.n / w5.L ** 3)
    out["energy_grad_262k"] = {"particles": w5.n, "ms": ms_grad, "particles_per_s": w5.n / (ms_grad / 1e3),
                               "unique_pairs_in_rc": w5.n * inr5 / 2,
                               "roofline": alu(w5.n * inr5 / 2, 30, ms_grad)}
    for name, v in out.items():
        v["roofline"]["traffic"] = _kernel_traffic(name)
    return out


def main():
    a = _args()
    if a.impl == "reference":
        return run_reference(a)
    import ctypes as C

    import torch
    import torch.distributed as dist

    from paper_1408_3764_gb300 import _lib
    from paper_1408_3764_gb300 import workloads as W

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.kernels_only:
        torch.cuda.set_device(local)
        dev = torch.device("cuda", local)
        flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
        peaks = _pipe_peaks(torch.cuda.current_stream(dev).cuda_stream)
        print(json.dumps({"kernels": _kernel_figures(dev, flush, peaks), "peaks": peaks}))
        return 0
    if a.micro_only:
        torch.cuda.set_device(local)
        dev = torch.device("cuda", local)
        flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
        M = a.moves or 100_000
        out = {}
        if a.workload == "c2":  # one workload: the 131,072-particle chain in the given precision
            prec = a.precision or "fp32"
            out["c2_131072_" + prec] = _micro_chain_rate(W.c2_fp32_vs_fp64(), prec, M, dev, flush)
        else:
            out["c1_2048_fp64"] = _micro_chain_rate(W.c1_plain_fp64(), "fp64", M, dev, flush)
            for prec in ("fp32", "fp64"):
                out["c2_131072_" + prec] = _micro_chain_rate(W.c2_fp32_vs_fp64(), prec, M, dev, flush)
            for rc in (2.5, 4.25):
                out["sweep_87296_rc%.2f_fp32" % rc] = _micro_chain_rate(W.cutoff_sweep(rc), "fp32", M, dev, flush)
        print(json.dumps({"micro": out}))
        return 0
    chains = _chains(a.workload)
    K = len(chains)
    # the CPU baseline's worker processes are spawned before the first GPU call
    pool = None
    if rank == 0 and not a.no_cpu_baseline:
        pool = OraclePool(a.workload, _cpu_workers(a))
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    M = a.moves
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    run = Runner(chains, a.precision, dev, rank)

    for k in range(a.warmup):
        run.step(k, M)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    launches0 = run.launches()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        times, chain_times, last = _time_steps(run, a.warmup, a.steps, M, flush)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    launches = run.launches() - launches0
    clocks = clk.summary()
    total_ms = sum(times)
    if ws > 1:
        total_ms = max_over_ranks(total_ms, dev)
    value = ws * a.steps * K * M / (total_ms / 1e3)
    stats = last[0]
    tuned = run.batch.config()
    run_acc = [sum(s["accepted"][i] for s in stats) / max(1, sum(s["attempted"][i] for s in stats)) for i in range(3)]
    final_n = int(sum(sum(s["n"]) for s in stats))
    flagged = int(sum(s["flagged"] for s in stats))

    # end to end through the public API: every step's configuration comes
    # from pinned host memory, the forces and the final configuration go back
    e2e_run = Runner(chains, a.precision, dev, rank, host_inputs=True)
    for k in range(a.warmup):
        e2e_run.step(k, M)
    torch.cuda.synchronize()
    e2e_run.h2d_bytes = e2e_run.d2h_bytes = 0
    if ws > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(a.steps):
        st_e2e = e2e_run.step(a.warmup + k, M)[0]
        _ = [s_["energy"] for s_ in st_e2e]  # the statistics are host values already
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if ws > 1:
        dist.barrier()
        e2e_s = max_over_ranks(e2e_s, dev)  # the job's time is its slowest replica's
    stats_bytes = K * (C.sizeof(_lib.MoveStats) + 2 * 8 + 8)  # statistics, energies, virials, prepared energies
    e2e = {"value": ws * a.steps * K * M / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(e2e_run.h2d_bytes / a.steps),
           "d2h_bytes_per_step": int(e2e_run.d2h_bytes / a.steps + stats_bytes),
           "what": "per step: each chain's configuration in (FP64 positions + species), forces, final configuration "
                   "and statistics out"}
    e2e_run.close()

    # roofline of the dominant kernel: the chain kernel against the latency
    # floor of one move (one dependent L2 round trip), one chain per CTA
    probe = _lib.ProbeResult()
    rc = _lib.load().gcmc_probe_latency(C.c_void_p(run.stream.cuda_stream), 8 << 20, C.byref(probe))
    peaks = _pipe_peaks(run.stream.cuda_stream)
    chain_ms = sum(chain_times) / len(chain_times)
    achieved = K * M / (chain_ms / 1e3)
    peak = K * 1e9 / probe.floor_ns if rc == 0 and probe.floor_ns > 0 else None
    traffic = None
    try:
        import hashlib
        src = os.path.join(ROOT, "paper_1408_3764_gb300", "csrc", "gcmc_chain.cu")
        if hashlib.sha256(open(src, "rb").read()).hexdigest().startswith(CHAIN_TRAFFIC["sha256_prefix"]):
            traffic = CHAIN_TRAFFIC["bytes"] * (K * M) / CHAIN_TRAFFIC["moves"]
    except OSError:
        pass
    # one more step, outside the timed region, with the chain kernel's
    # per-role cycle counters compiled in (they cost the kernel ~2.5 %)
    for b in run.boxes:
        b.set_chain_profile(True)
    run.step(a.warmup + a.steps, M)
    torch.cuda.synchronize()
    prof = {}
    for kk, b in enumerate(run.boxes):
        for key, v in b.chain_profile().items():
            prof[key] = prof.get(key, 0.0) + v
        b.set_chain_profile(False)
    moves_all = K * M
    roofline = {"bound": "latency", "achieved": achieved, "peak": peak, "unit": UNIT,
                "frac": (achieved / peak) if peak else None, "traffic": traffic, "kernel": "k_chain",
                "launch_ms": chain_ms,
                "floor_ns_per_move": probe.floor_ns,
                "context_ns": {"l2_hop": probe.l2_hop_ns, "cta_reduction": probe.sync_round_ns,
                               "philox_2_blocks": probe.philox_ns, "fp64_log": probe.log_ns},
                "committer_cycles_per_move": {k: prof[k] / moves_all for k in
                                              ("commit_wait", "commit_valid", "commit_decide", "commit_apply",
                                               "commit_book", "commit_total")},
                "peak_source": "measured in this run by gcmc_probe_latency: %d chains x 1 / (one dependent "
                               "L2 round trip per move)" % K}

    # the CPU baseline's oracle jobs run on the host cores while the GPU
    # measures the rest (they only read their own inputs)
    prec_jobs = None
    if pool is not None and not a.no_precision and a.workload == "isotherm":
        prec_jobs = {"c1": pool.submit(_oracle_chain_trace, "c1", 10_000, 0),
                     "c2": pool.submit(_oracle_chain_trace, "c2", 1_000_000, 100_000),
                     "tot": {"c2": pool.submit(_oracle_total_energy, "c2"),
                             "c3": pool.submit(_oracle_total_energy, "c3")}}

    compare, kernels = {}, None
    if rank == 0 and not a.no_compare:
        if a.workload != "c1":
            compare["plain_fp64_single_chain_2048"] = _single_chain_rate(W.c1_plain_fp64(), "fp64", 10_000, dev,
                                                                         flush)
        if a.workload != "c2":
            for prec in ("fp32", "fp64"):
                compare["single_chain_131072_" + prec] = _single_chain_rate(W.c2_fp32_vs_fp64(), prec, 200_000,
                                                                            dev, flush)
        # the same single chains evaluated over the microcell list (Sec. 3.3)
        compare["micro_single_chain_2048_fp64"] = _micro_chain_rate(W.c1_plain_fp64(), "fp64", 10_000, dev, flush)
        for prec in ("fp32", "fp64"):
            compare["micro_single_chain_131072_" + prec] = _micro_chain_rate(W.c2_fp32_vs_fp64(), prec, 200_000,
                                                                             dev, flush)
        if a.workload == "isotherm":
            other = "fp64" if a.precision == "fp32" else "fp32"
            r2 = Runner(chains, other, dev, 0)
            r2.step(0, M)
            t2, c2, _ = _time_steps(r2, 1, 1, M, flush)
            r2.close()
            compare["isotherm_batched_" + other] = {"moves_per_s": K * M / (c2[0] / 1e3),
                                                     "step_moves_per_s": K * M / (t2[0] / 1e3)}
            # the same isotherm keeping the running virial (virial pressure)
            r3 = Runner(chains, a.precision, dev, 0, virial=True)
            r3.step(0, M)
            t3, c3, _ = _time_steps(r3, 1, 1, M, flush)
            r3.close()
            compare["isotherm_batched_%s_virial" % a.precision] = {
                "moves_per_s": K * M / (c3[0] / 1e3), "step_moves_per_s": K * M / (t3[0] / 1e3)}
    if rank == 0 and not a.no_kernels:
        kernels = _kernel_figures(dev, flush, peaks)
    sweep = None
    if rank == 0 and not a.no_sweep:
        sweep = _cutoff_sweep(dev, flush, a.sweep_moves)

    cpu, precision = None, None
    if pool is not None:
        want = prec_jobs is not None
        if want:  # the precision jobs finish first: the baseline's sample gets every worker
            for f in (prec_jobs["c1"], prec_jobs["c2"], *prec_jobs["tot"].values()):
                f.result()
        m, dt, iso_traces = pool.step(0, a.cpu_moves, want_trace=want)
        cpu = {"value": m / dt, "unit": UNIT, "cores": pool.workers, "kind": "oracle",
               "sample": "%d chain(s) x %d moves (bin + total energy + moves + gradient per chain) from the initial "
                         "configurations, FP64 oracle, %d worker process(es), %.1f s wall" %
                         (K, a.cpu_moves, pool.workers, dt)}
        if want:
            precision = _precision(dev, pool, iso_traces, a.cpu_moves, prec_jobs["c1"], prec_jobs["c2"],
                                   prec_jobs["tot"])
        pool.close()

    if rank == 0:
        cfg = _workload_config(a.workload, chains, M, a.precision)
        cfg["parallelism"] = ("replicas x%d" % ws) if ws > 1 else ("batched, one CTA per chain" if K > 1
                                                                    else "single chain")
        cfg["start"] = ("step 1 from seeded uniform random positions, later steps from the previous step's "
                        "final configuration (warm-up %d steps)" % a.warmup)
        base = compare.get("plain_fp64_single_chain_2048")
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if a.precision == "fp32" else "f64",
                "data": "synthetic (seeded uniform random positions)", "config": cfg,
                "fp32_batched_over_plain_fp64": (value / base["step_moves_per_s"]) if base else None,
                "chain_moves_per_s": achieved, "team_shape": tuned[0],
                "tuner_probe_ms": [float(x) for x in tuned[1]] if tuned[1] is not None else None,
                "acceptance": run_acc, "final_n_total": final_n, "flagged": flagged,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "precision": precision, "peaks": peaks, "compare": compare,
                "kernels": kernels, "cutoff_sweep": sweep}
        print(json.dumps(line))
    run.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
