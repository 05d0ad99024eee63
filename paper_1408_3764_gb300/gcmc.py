"""Python front end of the GB300 GCMC library.

``Box`` wraps one C-ABI context: PyTorch tensors provide the device memory
and the CUDA stream, every step of the hot path runs in the library's CUDA
kernels.  ``cell_list_energy`` is the differentiable full-system energy.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import MAX_SPECIES, MoveMix, MoveStats, Params, check, load

TRACE_DTYPE = np.dtype([("dU", "<f8"), ("lnA", "<f8"), ("uabs", "<f8"), ("index", "<i4"),
                        ("type", "u1"), ("species", "u1"), ("accepted", "u1"),
                        ("flagged", "u1")])


def _ptr(t: Optional[torch.Tensor]):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _dev(t, dtype, device):
    t = torch.as_tensor(t, dtype=dtype)
    return t.to(device).contiguous()


@dataclass
class Mix:
    """Move mix and thermodynamic state (Algorithm 1, Eqs. 3-5)."""
    p_disp: float
    p_ins: float
    p_del: float
    max_disp: float
    beta: float
    log_z: Sequence[float]
    virial: bool = False  # also keep the running virial (stats virial, sum_virial)

    def to_c(self) -> MoveMix:
        m = MoveMix()
        m.p_disp, m.p_ins, m.p_del = self.p_disp, self.p_ins, self.p_del
        m.max_disp, m.beta = self.max_disp, self.beta
        lz = list(self.log_z)
        for s in range(MAX_SPECIES):
            m.log_z[s] = float(lz[s]) if s < len(lz) else 0.0
        m.flags = _lib.MIX_VIRIAL if self.virial else 0
        m.reserved = 0
        return m


def stats_dict(st: MoveStats, n_species: int) -> dict:
    return dict(attempted=list(st.attempted), accepted=list(st.accepted), flagged=int(st.flagged),
                moves_done=int(st.moves_done), energy=float(st.energy),
                sum_energy=float(st.sum_energy), sum_n=float(st.sum_n),
                n=[int(st.n[s]) for s in range(n_species)], virial=float(st.virial),
                sum_virial=float(st.sum_virial), chain_ms=float(st.chain_ms))


class Box:
    """One simulation box on the current CUDA device."""

    def __init__(self, L: float, rc: float, eps, sigma, precision: str = "fp64",
                 max_particles: int = 0, cell_capacity: int = 0,
                 stream: Optional[torch.cuda.Stream] = None, device=None):
        self._lib = load()
        eps = np.ascontiguousarray(np.asarray(eps, dtype=np.float64).reshape(-1))
        sigma = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64).reshape(-1))
        S = int(round(np.sqrt(eps.size)))
        if S * S != eps.size or sigma.size != eps.size:
            raise ValueError("eps and sigma must be S x S tables")
        self.S = S
        self.L, self.rc = float(L), float(rc)
        self.eps = eps.reshape(S, S).copy()
        self.sigma = sigma.reshape(S, S).copy()
        self.precision = precision
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        p = Params()
        p.L, p.rc, p.n_species = self.L, self.rc, S
        p.precision = _lib.FP32 if precision == "fp32" else _lib.FP64
        p.eps = eps.ctypes.data_as(C.POINTER(C.c_double))
        p.sigma = sigma.ctypes.data_as(C.POINTER(C.c_double))
        p.max_particles = int(max_particles)
        p.cell_capacity = int(cell_capacity)
        p.reserved = 0
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            check(self._lib.gcmc_create(C.byref(p), C.c_void_p(self.stream.cuda_stream), C.byref(h)),
                  None, "gcmc_create")
        self._h = h

    def close(self):
        """Frees the context and its device memory."""
        if getattr(self, "_h", None):
            self._lib.gcmc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def geometry(self) -> dict:
        """Cells per side T, cell count, cell capacity, per-species capacity, grid cutoff, grid spacing."""
        g = _lib.Geometry()
        check(self._lib.gcmc_get_geometry(self._h, C.byref(g)), self._h)
        return dict(T=g.T, n_cells=g.n_cells, cell_capacity=g.cell_capacity,
                    max_particles=g.max_particles, cutoff_grid2=g.cutoff_grid2, h=g.h)

    def build_cells(self, pos, species):
        """Bins n positions ([n, 3] FP64, box coordinates) of the given species into the cell list (Sec. 3.2.1)."""
        pos = _dev(pos, torch.float64, self.device).reshape(-1, 3)
        species = _dev(species, torch.int32, self.device).reshape(-1)
        if species.numel() != pos.shape[0]:
            raise ValueError("pos and species disagree in length")
        with torch.cuda.device(self.device):
            check(self._lib.gcmc_build_cells(self._h, _ptr(pos), _ptr(species), pos.shape[0]),
                  self._h, "gcmc_build_cells")
        self._n_build = pos.shape[0]
        return self

    def export_positions(self, pos_buf: Optional[torch.Tensor] = None, species_buf: Optional[torch.Tensor] = None):
        """The current configuration as build_cells input (device [N, 3] FP64 and [N] int32,
        species-major): building from it reproduces the configuration.  Given buffers
        (large enough) are filled without a host synchronisation; the N rows in use are returned."""
        n = int(self.counts().sum())
        if pos_buf is None:
            pos_buf = torch.empty((max(n, 1), 3), dtype=torch.float64, device=self.device)
        if species_buf is None:
            species_buf = torch.empty(max(n, 1), dtype=torch.int32, device=self.device)
        if pos_buf.shape[0] < n or species_buf.shape[0] < n:
            raise ValueError("export buffers hold %d rows, %d needed" % (min(pos_buf.shape[0], species_buf.shape[0]), n))
        out = C.c_int64()
        check(self._lib.gcmc_export_positions(self._h, _ptr(pos_buf), _ptr(species_buf), C.byref(out)), self._h,
              "gcmc_export_positions")
        return pos_buf[: out.value], species_buf[: out.value]

    def cell_list(self):
        """The last build's compact cell list: (cell starts, cell counts, input indices sorted by cell)."""
        g = self.geometry()
        cs = torch.empty(g["n_cells"], dtype=torch.int32, device=self.device)
        cc = torch.empty_like(cs)
        order = torch.empty(max(self._n_build, 1), dtype=torch.int32, device=self.device)
        check(self._lib.gcmc_cell_list(self._h, _ptr(cs), _ptr(cc), _ptr(order)), self._h)
        return cs, cc, order[: self._n_build]

    def launches(self) -> int:
        """Kernels this box has launched so far."""
        out = np.zeros(1, np.int64)
        check(self._lib.gcmc_kernel_launches(self._h, out.ctypes.data_as(C.c_void_p)), self._h)
        return int(out[0])

    def set_chain_config(self, config: int):
        """Team shape of the chain kernel: 0..3, or -1 = tuned on the next run."""
        check(self._lib.gcmc_set_chain_config(self._h, int(config)), self._h)

    def chain_config(self) -> int:
        """The chain kernel's current team shape (0..3; -1 before the tuner has run)."""
        out = C.c_int32()
        check(self._lib.gcmc_get_chain_config(self._h, C.byref(out)), self._h)
        return out.value

    def chain_counters(self) -> dict:
        """Moves of the last run evaluated again (refetched) and trials decided in FP64 (refined)."""
        out = np.zeros(2, np.int64)
        check(self._lib.gcmc_chain_counters(self._h, out[0:].ctypes.data_as(C.c_void_p),
                                            out[1:].ctypes.data_as(C.c_void_p)), self._h)
        return dict(refetched=int(out[0]), refined=int(out[1]))

    def set_chain_profile(self, on: bool = True):
        """Whether the following chain runs count cycles per role (chain_profile); off by default,
        since the clock reads slow the kernel by about 2.5 %."""
        check(self._lib.gcmc_set_chain_profile(self._h, 1 if on else 0), self._h)

    def chain_profile(self) -> dict:
        """SM cycles of the last chain run by role (zeros unless set_chain_profile was on):
        committer waiting, validity, decision, applying, loop total; team leaders idle, teams
        evaluating, evaluations."""
        out = np.zeros(12, np.float64)
        check(self._lib.gcmc_chain_profile(self._h, out.ctypes.data_as(C.c_void_p)), self._h)
        keys = ("commit_wait", "commit_valid", "commit_decide", "commit_apply", "commit_total",
                "leader_idle", "team_eval", "evaluations", "valid_epoch", "valid_logs", "valid_pick",
                "commit_book")
        return dict(zip(keys, out.tolist()))

    def counts(self) -> np.ndarray:
        """Particles per species."""
        out = np.zeros(MAX_SPECIES, np.int64)
        check(self._lib.gcmc_counts(self._h, out.ctypes.data_as(C.c_void_p)), self._h)
        return out[: self.S]

    def trial_energy(self, pos, species, exclude=None, with_abs=False):
        """Energy of trial points ([m, 3] FP64) of the given species against their 27 cells, each
        excluding one particle id (s << 32 | i) or none; with_abs also returns the |rep| + |att| sums."""
        pos = _dev(pos, torch.float64, self.device).reshape(-1, 3)
        species = _dev(species, torch.int32, self.device).reshape(-1)
        m = pos.shape[0]
        ex = None if exclude is None else _dev(exclude, torch.int64, self.device).reshape(-1)
        out = torch.empty(m, dtype=torch.float64, device=self.device)
        oabs = torch.empty(m, dtype=torch.float64, device=self.device) if with_abs else None
        check(self._lib.gcmc_trial_energy(self._h, _ptr(pos), _ptr(species), _ptr(ex), m, _ptr(out),
                                          _ptr(oabs)), self._h, "gcmc_trial_energy")
        return (out, oabs) if with_abs else out

    def trial_energy_raw(self, pos: torch.Tensor, species: torch.Tensor, out: torch.Tensor,
                         exclude: Optional[torch.Tensor] = None, out_abs=None):
        """No-copy variant on prepared device tensors (used by the benchmark)."""
        return self._lib.gcmc_trial_energy(self._h, _ptr(pos), _ptr(species), _ptr(exclude),
                                           pos.shape[0], _ptr(out), _ptr(out_abs))

    def total_energy(self) -> float:
        """Full-system energy (Sec. 3.1.1, over the 27 cells); also resets the chain's running energy."""
        e = C.c_double()
        check(self._lib.gcmc_total_energy(self._h, C.byref(e)), self._h, "gcmc_total_energy")
        return e.value

    def energy_grad(self, want_pos=True):
        """Energy, virial and gradients: forces per particle (species-major, on the device),
        dE/deps and dE/dsigma tables."""
        n = int(self.counts().sum())
        dpos = torch.empty((max(n, 1), 3), dtype=torch.float32, device=self.device) if want_pos else None
        S = self.S
        deps = np.zeros(S * S, np.float64)
        dsig = np.zeros(S * S, np.float64)
        e = C.c_double()
        w = C.c_double()
        check(self._lib.gcmc_energy_grad(self._h, _ptr(dpos), deps.ctypes.data_as(C.c_void_p),
                                         dsig.ctypes.data_as(C.c_void_p), C.byref(e), C.byref(w)),
              self._h, "gcmc_energy_grad")
        return dict(dpos=dpos[:n] if dpos is not None else None, deps=deps.reshape(S, S),
                    dsigma=dsig.reshape(S, S), energy=e.value, virial=w.value)

    def run_moves(self, seed: int, first_move: int, n_moves: int, mix: Mix, trace: bool = False,
                  trace_buf: Optional[torch.Tensor] = None, check_status: bool = True):
        """Moves first_move .. first_move + n_moves - 1 of the chain (Algorithm 1) on the device.
        Returns the statistics (and the per-move trace with trace=True)."""
        cm = mix.to_c()
        st = MoveStats()
        tb = trace_buf
        if trace and tb is None:
            tb = torch.empty((max(n_moves, 1), _lib.TRACE_BYTES), dtype=torch.uint8, device=self.device)
        rc = self._lib.gcmc_run_moves(self._h, seed, first_move, n_moves, C.byref(cm), C.byref(st),
                                      _ptr(tb) if (trace or trace_buf is not None) else None)
        if check_status:
            check(rc, self._h, "gcmc_run_moves")
        stats = stats_dict(st, self.S)
        stats["status"] = rc
        if trace:
            arr = tb[:n_moves].cpu().numpy().copy().view(TRACE_DTYPE).reshape(-1)
            return stats, arr
        return stats

    def check_state(self) -> None:
        """Host-side consistency check of the configuration (raises on a violation)."""
        check(self._lib.gcmc_check_state(self._h), self._h, "gcmc_check_state")

    def set_wait_limit(self, ns: int, stall_move: int = -1) -> None:
        """Diagnostic hook: the chain kernel's wait limit in ns (0: the default)
        and a move at which the committer waits on a flag nothing sets (-1: none)."""
        check(self._lib.gcmc_set_wait_limit(self._h, int(ns), int(stall_move)), self._h)

    def build_microcells(self, edge: float = 1.0, capacity: int = 0) -> None:
        """Microcell list of the current particles (Sec. 3.3)."""
        check(self._lib.gcmc_build_microcells(self._h, float(edge), int(capacity)), self._h,
              "gcmc_build_microcells")

    def microcells(self):
        """(M, capacity, counts [M^3] uint8, slots [capacity, M^3, 4] uint32 (X, Y, Z, tag))."""
        M = C.c_int64()
        cap = C.c_int32()
        check(self._lib.gcmc_microcells(self._h, C.byref(M), C.byref(cap), None, None), self._h, "gcmc_microcells")
        n3 = M.value ** 3
        counts = np.zeros(n3, np.uint8)
        slots = np.zeros((cap.value, n3, 4), np.uint32)
        check(self._lib.gcmc_microcells(self._h, None, None, counts.ctypes.data_as(C.c_void_p),
                                        slots.ctypes.data_as(C.c_void_p)), self._h, "gcmc_microcells")
        return M.value, cap.value, counts, slots

    def run_moves_micro(self, seed: int, first_move: int, n_moves: int, mix: Mix, trace: bool = False,
                        check_status: bool = True):
        """The chain of run_moves evaluated over the microcell list."""
        cm = mix.to_c()
        st = MoveStats()
        tb = None
        if trace:
            tb = torch.empty((max(n_moves, 1), _lib.TRACE_BYTES), dtype=torch.uint8, device=self.device)
        rc = self._lib.gcmc_run_moves_micro(self._h, seed, first_move, n_moves, C.byref(cm), C.byref(st),
                                            _ptr(tb) if trace else None)
        if check_status:
            check(rc, self._h, "gcmc_run_moves_micro")
        stats = stats_dict(st, self.S)
        stats["status"] = rc
        if trace:
            return stats, tb[:n_moves].cpu().numpy().copy().view(TRACE_DTYPE).reshape(-1)
        return stats

    def get_state(self):
        """(counts per species, grid positions species-major, cell counts, cell references, running energy)."""
        n = self.counts()
        N = int(n.sum())
        g = self.geometry()
        pos = np.zeros((max(N, 1), 3), np.uint32)
        cc = np.zeros(g["n_cells"], np.int32)
        refs = np.zeros(max(N, 1), np.uint32)
        e = C.c_double()
        check(self._lib.gcmc_get_state(self._h, pos.ctypes.data_as(C.c_void_p),
                                       cc.ctypes.data_as(C.c_void_p), refs.ctypes.data_as(C.c_void_p),
                                       C.byref(e)), self._h)
        return n, pos[:N], cc, refs[:N], e.value

    def restore(self, n_per_species, pos, cell_count, cell_refs, energy=float("nan")):
        """Imports a state from get_state (validated in full before anything changes)."""
        n = np.ascontiguousarray(np.asarray(n_per_species, np.int64))
        pos = np.ascontiguousarray(np.asarray(pos, np.uint32).reshape(-1, 3))
        cc = np.ascontiguousarray(np.asarray(cell_count, np.int32))
        refs = np.ascontiguousarray(np.asarray(cell_refs, np.uint32))
        check(self._lib.gcmc_set_state(self._h, n.ctypes.data_as(C.c_void_p),
                                       pos.ctypes.data_as(C.c_void_p), cc.ctypes.data_as(C.c_void_p),
                                       refs.ctypes.data_as(C.c_void_p), float(energy)), self._h,
              "gcmc_set_state")


class Batch:
    """Independent chains (e.g. the points of an isotherm) run in one launch,
    one CTA per chain, replayed as a CUDA graph."""

    def __init__(self, boxes: Sequence[Box]):
        self._lib = load()
        self.boxes = list(boxes)
        arr = (C.c_void_p * len(self.boxes))(*[b.handle for b in self.boxes])
        h = C.c_void_p()
        check(self._lib.gcmc_batch_create(arr, len(self.boxes), C.byref(h)), None, "gcmc_batch_create")
        self._h = h

    def close(self):
        """Frees the batch (the boxes stay)."""
        if getattr(self, "_h", None):
            self._lib.gcmc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run_moves(self, seeds, first_move: int, n_moves: int, mixes: Sequence[Mix], check_status=True,
                  trace: bool = False):
        """Moves first_move .. first_move + n_moves - 1 of every chain in one launch; per-chain
        statistics (and with trace=True the per-chain move records, as Box.run_moves gives them)."""
        K = len(self.boxes)
        sd = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64).reshape(K))
        cm = (MoveMix * K)(*[m.to_c() for m in mixes])
        st = (MoveStats * K)()
        bufs = None
        if trace:
            dev = self.boxes[0].device
            bufs = [torch.empty((max(n_moves, 1), _lib.TRACE_BYTES), dtype=torch.uint8, device=dev)
                    for _ in range(K)]
            arr = (C.c_void_p * K)(*[t.data_ptr() for t in bufs])
            check(self._lib.gcmc_batch_set_traces(self._h, arr), None, "gcmc_batch_set_traces")
        try:
            rc = self._lib.gcmc_batch_run_moves(self._h, sd.ctypes.data_as(C.c_void_p), int(first_move),
                                                int(n_moves), cm, st)
        finally:
            if trace:
                self._lib.gcmc_batch_set_traces(self._h, None)
        if check_status and rc != 0:
            raise _lib.GcmcError(rc, self._lib.gcmc_batch_last_error(self._h).decode(errors="replace"))
        stats = [stats_dict(st[k], self.boxes[k].S) for k in range(K)]
        if trace:
            return stats, [b[:n_moves].cpu().numpy().copy().view(TRACE_DTYPE).reshape(-1) for b in bufs]
        return stats

    def prepare(self, positions: Sequence[torch.Tensor], species: Sequence[torch.Tensor]) -> np.ndarray:
        """Builds every box's cells from device tensors ([n_k, 3] FP64, [n_k] int32) and
        returns the full-system energies (two host synchronisations in all)."""
        K = len(self.boxes)
        pp = (C.c_void_p * K)(*[p.data_ptr() for p in positions])
        sp = (C.c_void_p * K)(*[t.data_ptr() for t in species])
        n = np.ascontiguousarray([int(p.shape[0]) for p in positions], dtype=np.int64)
        e = np.zeros(K, np.float64)
        rc = self._lib.gcmc_batch_prepare(self._h, pp, sp, n.ctypes.data_as(C.c_void_p), e.ctypes.data_as(C.c_void_p))
        if rc != 0:
            raise _lib.GcmcError(rc, self._lib.gcmc_batch_last_error(self._h).decode(errors="replace"))
        return e

    def energy_grad(self, dpos: Optional[Sequence[Optional[torch.Tensor]]] = None):
        """Forces (into the given device tensors, [N_k, 3] FP32, species-major), energies and
        virials of every box (one host synchronisation in all)."""
        K = len(self.boxes)
        dp = None
        if dpos is not None:
            dp = (C.c_void_p * K)(*[(t.data_ptr() if t is not None else None) for t in dpos])
        e = np.zeros(K, np.float64)
        w = np.zeros(K, np.float64)
        rc = self._lib.gcmc_batch_energy_grad(self._h, dp, e.ctypes.data_as(C.c_void_p), w.ctypes.data_as(C.c_void_p))
        if rc != 0:
            raise _lib.GcmcError(rc, self._lib.gcmc_batch_last_error(self._h).decode(errors="replace"))
        return e, w

    def export_positions(self, positions: Sequence[torch.Tensor], species: Sequence[torch.Tensor]) -> np.ndarray:
        """Every box's current configuration into the given device tensors ([>= N_k, 3] FP64,
        [>= N_k] int32, species-major; build input for the next prepare) without a host
        synchronisation; returns the counts N_k."""
        K = len(self.boxes)
        for k in range(K):
            need = int(self.boxes[k].counts().sum())
            if positions[k].shape[0] < need or species[k].shape[0] < need:
                raise ValueError("export buffers of box %d hold fewer than %d rows" % (k, need))
        pp = (C.c_void_p * K)(*[p.data_ptr() for p in positions])
        sp = (C.c_void_p * K)(*[t.data_ptr() for t in species])
        n = np.zeros(K, np.int64)
        rc = self._lib.gcmc_batch_export_positions(self._h, pp, sp, n.ctypes.data_as(C.c_void_p))
        if rc != 0:
            raise _lib.GcmcError(rc, self._lib.gcmc_batch_last_error(self._h).decode(errors="replace"))
        return n

    def config(self, set_config: int = -2):
        """Sets the team shape (-1 automatic, -2 unchanged); returns it and the tuner's per-shape times."""
        out = C.c_int32()
        probe = np.zeros(_lib.CHAIN_CONFIGS, np.float64)
        check(self._lib.gcmc_batch_config(self._h, int(set_config), C.byref(out),
                                          probe.ctypes.data_as(C.c_void_p)), None, "gcmc_batch_config")
        return out.value, probe

    def launches(self) -> int:
        """Chain launches of this batch so far."""
        out = np.zeros(1, np.int64)
        check(self._lib.gcmc_batch_launches(self._h, out.ctypes.data_as(C.c_void_p)), None)
        return int(out[0])

    def device_ms(self) -> float:
        """Device time of the chain launches of the last run_moves call."""
        out = C.c_double()
        check(self._lib.gcmc_batch_device_ms(self._h, C.byref(out)), None)
        return out.value


def species_major_order(species) -> np.ndarray:
    """Input indices listed in species-major order (species 0 first, input
    order within a species): row r of a species-major array belongs to input
    particle order[r]."""
    s = np.asarray(species).reshape(-1)
    return np.argsort(s, kind="stable")


class _BoxCache:
    """A few contexts kept for the differentiable energy, keyed by box, cutoff,
    force-field tables, precision and device, so that repeated calls build
    cells in an existing context instead of creating and freeing one."""

    def __init__(self, size: int = 4):
        self.size = size
        self.items = []  # (key, Box), most recent last
        self.builds = 0  # cell builds done through the cache (counts reuse in tests)
        self.creates = 0

    def get(self, L, rc, eps, sigma, precision, device) -> "Box":
        key = (float(L), float(rc), tuple(np.asarray(eps, np.float64).ravel().tolist()),
               tuple(np.asarray(sigma, np.float64).ravel().tolist()), precision, str(device))
        for i, (k, b) in enumerate(self.items):
            if k == key:
                self.items.append(self.items.pop(i))
                return b
        b = Box(L, rc, eps, sigma, precision=precision, device=device)
        self.creates += 1
        self.items.append((key, b))
        if len(self.items) > self.size:
            self.items.pop(0)[1].close()
        return b


_box_cache = _BoxCache()


class _CellListEnergy(torch.autograd.Function):
    """Full-system cell-list energy with its hand-written backward.  The
    forward pass bins the positions into a cached context and runs the
    energy kernel only; the backward pass runs the gradient kernel (dE/dpos,
    dE/deps, dE/dsigma in one pass) on the same cells, rebinning first if
    another call used the context in between."""

    @staticmethod
    def forward(ctx, pos, eps, sigma, species, L, rc, precision):
        device = pos.device if pos.is_cuda else torch.device("cuda", torch.cuda.current_device())
        box = _box_cache.get(L, rc, eps.detach().cpu().numpy(), sigma.detach().cpu().numpy(), precision, device)
        pos64 = pos.detach().to(device=device, dtype=torch.float64).contiguous()
        box.build_cells(pos64, species)
        _box_cache.builds += 1
        box._token = ctx.token = object()  # the cells in the context now belong to this call
        E = box.total_energy()
        ctx.box = box
        ctx.pos64 = pos64
        ctx.species = species
        ctx.pos_dtype = pos.dtype
        ctx.e_dtype, ctx.s_dtype = eps.dtype, sigma.dtype
        return torch.tensor(E, dtype=torch.float64, device=pos.device)

    @staticmethod
    def backward(ctx, go):
        box = ctx.box
        if getattr(box, "_token", None) is not ctx.token:
            box.build_cells(ctx.pos64, ctx.species)
            _box_cache.builds += 1
            box._token = ctx.token
        g = box.energy_grad(want_pos=ctx.needs_input_grad[0])
        gp = None
        if ctx.needs_input_grad[0]:
            sm = torch.as_tensor(species_major_order(ctx.species.detach().cpu().numpy()), device=g["dpos"].device)
            dpos = torch.empty_like(g["dpos"])
            dpos[sm] = g["dpos"]  # species-major rows back to input order
            gp = go.to(dpos.dtype) * dpos
            gp = gp.to(ctx.pos_dtype)
        ge = go.detach().cpu().to(ctx.e_dtype) * torch.as_tensor(g["deps"], dtype=ctx.e_dtype)
        gs = go.detach().cpu().to(ctx.s_dtype) * torch.as_tensor(g["dsigma"], dtype=ctx.s_dtype)
        ctx.box = None
        return gp, ge, gs, None, None, None, None


def cell_list_energy(pos: torch.Tensor, eps: torch.Tensor, sigma: torch.Tensor, species: torch.Tensor,
                     L: float, rc: float, precision: str = "fp32") -> torch.Tensor:
    """E = 1/2 sum_{i != j} U(r_ij) over the cell list, differentiable with
    respect to pos ([N, 3], CUDA), eps and sigma ([S, S] tables, CPU float64).
    dE/deps[a][b] is half of the sum over ordered type pairs (a, b), so a
    symmetric change of both entries sees the full cross-term sum."""
    return _CellListEnergy.apply(pos, eps, sigma, species, L, rc, precision)
