"""CPU oracle for the GCMC hot path of arXiv 1408.3764 (plain C, FP64).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The product library
never loads it, and it shares no code with the CUDA path: the two meet only
through the seeded input generators in ``paper_1408_3764_gb300.workloads``.

The arithmetic lives in ``gcmc_oracle.c``; this module only marshals numpy
arrays through ``ctypes``.  Every function cites the passage of the paper it
follows in the C source.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

MAX_SPECIES = 8

_lib = None


def lib():
    """Loads (building if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        d, i64, u64, i32, u32, vp = (C.c_double, C.c_int64, C.c_uint64, C.c_int32, C.c_uint32,
                                      C.c_void_p)
        L.orc_philox4x32_10.argtypes = [vp, vp, vp]
        L.orc_lj.argtypes = [d, d, d, vp, vp]
        L.orc_lj.restype = d
        L.orc_lj_dr.argtypes = [d, d, d]
        L.orc_lj_dr.restype = d
        L.orc_lj_dsigma.argtypes = [d, d, d]
        L.orc_lj_dsigma.restype = d
        L.orc_cells_per_side.argtypes = [d, d]
        L.orc_cells_per_side.restype = C.c_int
        L.orc_quantize.argtypes = [d, d, vp]
        L.orc_quantize.restype = C.c_int
        L.orc_cutoff_grid2.argtypes = [d, d]
        L.orc_cutoff_grid2.restype = u64
        L.orc_disp_grid.argtypes = [d, d]
        L.orc_disp_grid.restype = i64
        L.orc_create.argtypes = [d, d, C.c_int, vp, vp]
        L.orc_create.restype = vp
        L.orc_destroy.argtypes = [vp]
        L.orc_geometry.argtypes = [vp, vp, vp, vp, vp]
        L.orc_build.argtypes = [vp, vp, vp, i64, vp, vp, vp]
        L.orc_build.restype = C.c_int
        L.orc_trial_energy.argtypes = [vp, vp, vp, vp, i64, vp, vp, C.c_int]
        L.orc_trial_energy.restype = C.c_int
        L.orc_total_energy_brute.argtypes = [vp]
        L.orc_total_energy_brute.restype = d
        L.orc_total_energy_cells.argtypes = [vp]
        L.orc_total_energy_cells.restype = d
        L.orc_particle_energies.argtypes = [vp, vp]
        L.orc_energy_grad.argtypes = [vp, vp, vp, vp, vp, vp, C.c_int]
        L.orc_energy_grad.restype = C.c_int
        L.orc_set_energy.argtypes = [vp, d]
        L.orc_get_energy.argtypes = [vp]
        L.orc_get_energy.restype = d
        L.orc_set_virial.argtypes = [vp, d]
        L.orc_get_virial.argtypes = [vp]
        L.orc_get_virial.restype = d
        L.orc_move_words.argtypes = [u64, u64, u32, vp]
        L.orc_pick_index.argtypes = [i64, vp, C.c_int]
        L.orc_pick_index.restype = i64
        L.orc_run_moves.argtypes = [vp, u64, u32, u64, i64, vp, d, vp, vp]
        L.orc_run_moves.restype = C.c_int
        L.orc_run_moves_ex.argtypes = [vp, u64, u32, u64, i64, vp, d, vp, vp, vp]
        L.orc_run_moves_ex.restype = C.c_int
        L.orc_count.argtypes = [vp, C.c_int]
        L.orc_count.restype = i64
        L.orc_get_state.argtypes = [vp, vp, vp, vp]
        L.orc_widom.argtypes = [vp, C.c_int, d, u64, i64]
        L.orc_widom.restype = d
        L.orc_micro_build.argtypes = [vp, d]
        L.orc_micro_build.restype = C.c_int
        L.orc_micro_state.argtypes = [vp, vp, vp]
        L.orc_micro_state.restype = i64
        L.orc_micro_per_side.argtypes = [vp]
        L.orc_micro_per_side.restype = C.c_int
        L.orc_micro_cube.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, vp]
        L.orc_micro_cube.restype = i64
        L.orc_energy_micro.argtypes = [vp, vp, C.c_int, C.c_int, i64, C.c_int, vp]
        L.orc_energy_micro.restype = d
        L.orc_energy_brute.argtypes = [vp, vp, C.c_int, C.c_int, i64, vp]
        L.orc_energy_brute.restype = d
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class Mix(C.Structure):
    _fields_ = [("p_disp", C.c_double), ("p_ins", C.c_double), ("p_del", C.c_double),
                ("max_disp", C.c_double), ("beta", C.c_double),
                ("log_z", C.c_double * MAX_SPECIES)]


TRACE_DTYPE = np.dtype([("dU", "<f8"), ("lnA", "<f8"), ("uabs", "<f8"), ("index", "<i4"),
                        ("type", "u1"), ("species", "u1"), ("accepted", "u1"),
                        ("flagged", "u1")])
assert TRACE_DTYPE.itemsize == 32


class Stats(C.Structure):
    _fields_ = [("attempted", C.c_int64 * 3), ("accepted", C.c_int64 * 3),
                ("flagged", C.c_int64), ("moves_done", C.c_int64), ("energy", C.c_double),
                ("sum_energy", C.c_double), ("sum_n", C.c_double),
                ("n", C.c_int64 * MAX_SPECIES), ("virial", C.c_double), ("sum_virial", C.c_double)]


def philox4x32_10(counter, key) -> np.ndarray:
    """Philox4x32-10 block for a 4-word counter and a 2-word key."""
    c = np.asarray(counter, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def move_words(seed: int, move: int, chain: int = 0) -> np.ndarray:
    """The eight random words of one move."""
    out = np.zeros(8, dtype=np.uint32)
    lib().orc_move_words(seed, move, chain, _p(out))
    return out


def pick_index(n: int, words, move_type: int) -> int:
    """The index a displacement (move_type 0) or deletion (2) picks among n >= 1
    candidates from the move's eight words."""
    w = np.ascontiguousarray(words, dtype=np.uint32)
    assert w.shape == (8,) and n >= 1
    return int(lib().orc_pick_index(int(n), _p(w), int(move_type)))


def lj(r2: float, eps: float, sigma: float):
    """Eq. 1 pair energy with its repulsive and attractive magnitudes."""
    rep = C.c_double()
    att = C.c_double()
    u = lib().orc_lj(r2, eps, sigma, C.byref(rep), C.byref(att))
    return u, rep.value, att.value


def lj_dr(r2: float, eps: float, sigma: float) -> float:
    return lib().orc_lj_dr(r2, eps, sigma)


def lj_dsigma(r2: float, eps: float, sigma: float) -> float:
    return lib().orc_lj_dsigma(r2, eps, sigma)


def cells_per_side(L: float, rc: float) -> int:
    return lib().orc_cells_per_side(L, rc)


def quantize(x: float, L: float) -> int:
    X = np.zeros(1, dtype=np.uint32)
    if lib().orc_quantize(float(x), float(L), _p(X)) != 0:
        raise ValueError("coordinate not finite")
    return int(X[0])


def cutoff_grid2(L: float, rc: float) -> int:
    return int(lib().orc_cutoff_grid2(L, rc))


def disp_grid(max_disp: float, L: float) -> int:
    return int(lib().orc_disp_grid(max_disp, L))


@dataclass
class CellList:
    cell_start: np.ndarray
    cell_count: np.ndarray
    order: np.ndarray


class System:
    """An oracle GCMC system: box, force field, particles and cell list."""

    def __init__(self, L: float, rc: float, eps, sigma):
        eps = np.ascontiguousarray(np.asarray(eps, dtype=np.float64).reshape(-1))
        sigma = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64).reshape(-1))
        S = int(round(np.sqrt(eps.size)))
        if S * S != eps.size or sigma.size != eps.size:
            raise ValueError("eps/sigma must be S x S")
        self.S = S
        self.L = float(L)
        self.rc = float(rc)
        self._h = lib().orc_create(self.L, self.rc, S, _p(eps), _p(sigma))
        if not self._h:
            raise ValueError("invalid box/cutoff/species")
        T = np.zeros(1, np.int64)
        nc = np.zeros(1, np.int64)
        r2 = np.zeros(1, np.uint64)
        h = np.zeros(1, np.float64)
        lib().orc_geometry(self._h, _p(T), _p(nc), _p(r2), _p(h))
        self.T, self.ncell, self.R2, self.h = int(T[0]), int(nc[0]), int(r2[0]), float(h[0])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def build(self, pos, types) -> CellList:
        pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
        types = np.ascontiguousarray(np.asarray(types, dtype=np.int32).reshape(-1))
        n = pos.shape[0]
        cs = np.zeros(self.ncell, np.int64)
        cc = np.zeros(self.ncell, np.int64)
        order = np.zeros(max(n, 1), np.int64)
        if lib().orc_build(self._h, _p(pos), _p(types), n, _p(cs), _p(cc), _p(order)) != 0:
            raise ValueError("bad positions or species")
        return CellList(cs, cc, order[:n])

    def counts(self) -> np.ndarray:
        return np.array([lib().orc_count(self._h, s) for s in range(self.S)], dtype=np.int64)

    def trial_energy(self, pos, species, exclude=None, brute=False, with_abs=False):
        pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
        m = pos.shape[0]
        species = np.ascontiguousarray(np.asarray(species, dtype=np.int32).reshape(-1))
        ex = None
        if exclude is not None:
            ex = np.ascontiguousarray(np.asarray(exclude, dtype=np.int64).reshape(-1))
        out = np.zeros(m, np.float64)
        oabs = np.zeros(m, np.float64)
        rc = lib().orc_trial_energy(self._h, _p(pos), _p(species), _p(ex), m, _p(out), _p(oabs),
                                    1 if brute else 0)
        if rc != 0:
            raise ValueError("bad trial positions")
        return (out, oabs) if with_abs else out

    def total_energy(self, brute=False) -> float:
        return (lib().orc_total_energy_brute(self._h) if brute
                else lib().orc_total_energy_cells(self._h))

    def particle_energies(self) -> np.ndarray:
        e = np.zeros(max(int(self.counts().sum()), 1), np.float64)
        lib().orc_particle_energies(self._h, _p(e))
        return e[: int(self.counts().sum())]

    def energy_grad(self, brute=False):
        n = int(self.counts().sum())
        dpos = np.zeros((max(n, 1), 3), np.float64)
        deps = np.zeros(self.S * self.S, np.float64)
        dsig = np.zeros(self.S * self.S, np.float64)
        e = np.zeros(1, np.float64)
        w = np.zeros(1, np.float64)
        lib().orc_energy_grad(self._h, _p(dpos), _p(deps), _p(dsig), _p(e), _p(w),
                              1 if brute else 0)
        return dict(dpos=dpos[:n], deps=deps.reshape(self.S, self.S),
                    dsigma=dsig.reshape(self.S, self.S), energy=float(e[0]), virial=float(w[0]))

    def set_energy(self, E: float):
        lib().orc_set_energy(self._h, float(E))

    def energy(self) -> float:
        return lib().orc_get_energy(self._h)

    def set_virial(self, W: float):
        """Running virial sum_{i<j} r U'(r); NaN lets run_moves compute it."""
        lib().orc_set_virial(self._h, float(W))

    def virial(self) -> float:
        return lib().orc_get_virial(self._h)

    def run_moves(self, seed, first, n_moves, p_disp, p_ins, p_del, max_disp, beta, log_z,
                  tol=1e-12, chain=0, trace=True, with_sabs=False):
        """Moves [first, first + n_moves) of the chain; returns (trace, stats),
        and with with_sabs also the per-move sum of |u_j| over the evaluated
        pair terms (the floor of the per-move dU error measure)."""
        mix = Mix()
        mix.p_disp, mix.p_ins, mix.p_del = p_disp, p_ins, p_del
        mix.max_disp, mix.beta = max_disp, beta
        lz = list(np.atleast_1d(np.asarray(log_z, dtype=np.float64)))
        for s in range(MAX_SPECIES):
            mix.log_z[s] = lz[s] if s < len(lz) else 0.0
        tr = np.zeros(n_moves if trace else 0, TRACE_DTYPE)
        st = Stats()
        sabs = np.zeros(n_moves, np.float64) if with_sabs else None
        rc = lib().orc_run_moves_ex(self._h, seed, chain, first, n_moves, C.byref(mix), tol,
                                    _p(tr) if trace else None, C.byref(st), _p(sabs))
        if rc != 0:
            raise RuntimeError("energy not set: call set_energy(total_energy()) first")
        if with_sabs:
            return tr, st, sabs
        return tr, st

    def state(self):
        """(counts per species, grid positions species-major, cell counts, cell refs)."""
        cnt = self.counts()
        n = int(cnt.sum())
        pos = np.zeros((max(n, 1), 3), np.uint32)
        cc = np.zeros(self.ncell, np.int64)
        refs = np.zeros(max(n, 1), np.uint32)
        lib().orc_get_state(self._h, _p(pos), _p(cc), _p(refs))
        return cnt, pos[:n], cc, refs[:n]

    def widom(self, species, beta, seed, n) -> float:
        return lib().orc_widom(self._h, species, beta, seed, n)

    def micro_build(self, edge: float = 1.0) -> int:
        """Builds the microcells (Sec. 3.3) of the current particles; later
        accepted moves keep them up to date.  Returns M (cells per side)."""
        M = lib().orc_micro_build(self._h, float(edge))
        if M < 0:
            raise ValueError("bad microcell edge")
        return M

    def micro_cube(self, centre, D: int) -> np.ndarray:
        """Microcell ids of the cube of half-width D around microcell `centre`
        (x, y, z), in thread order (x fastest), Sec. 3.3.2."""
        M = lib().orc_micro_per_side(self._h)
        n = min(2 * D + 1, M)
        out = np.zeros(n ** 3, np.int64)
        k = lib().orc_micro_cube(self._h, int(centre[0]), int(centre[1]), int(centre[2]), int(D), _p(out))
        return out[:k]

    def energy_micro(self, P_grid, species: int, exclude=(-1, -1), D: int = 3):
        """(energy, uabs) of a particle at grid position P_grid summed over the
        cube of microcells around it."""
        P = np.ascontiguousarray(np.asarray(P_grid, dtype=np.uint32).reshape(3))
        ua = np.zeros(1, np.float64)
        e = lib().orc_energy_micro(self._h, _p(P), int(species), int(exclude[0]), int(exclude[1]), int(D), _p(ua))
        return e, float(ua[0])

    def energy_brute_grid(self, P_grid, species: int, exclude=(-1, -1)):
        """(energy, uabs) of a particle at grid position P_grid against every
        particle but `exclude` (the definition)."""
        P = np.ascontiguousarray(np.asarray(P_grid, dtype=np.uint32).reshape(3))
        ua = np.zeros(1, np.float64)
        e = lib().orc_energy_brute(self._h, _p(P), int(species), int(exclude[0]), int(exclude[1]), _p(ua))
        return e, float(ua[0])

    def micro_state(self):
        """(M, per-microcell counts, concatenated per-cell lists of (i << 8) | s,
        largest count)."""
        M = lib().orc_micro_per_side(self._h)
        cnt = np.zeros(max(M ** 3, 1), np.int64)
        n = int(self.counts().sum())
        refs = np.zeros(max(n, 1), np.uint32)
        mx = lib().orc_micro_state(self._h, _p(cnt), _p(refs))
        return M, cnt[: M ** 3], refs[:n], int(mx)


def lib_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libgcmc_oracle.so")
