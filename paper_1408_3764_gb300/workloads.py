"""Seeded synthetic inputs shaped like the paper's workloads.

This module is the one place both the CUDA path's tests and the CPU oracle
draw their inputs from.  It holds none of the method's arithmetic: it only
makes boxes, positions, species labels and force-field tables, and lists the
workload configurations.

The paper measures on uniform single-species Lennard-Jones fluids at reduced
densities 0.6-0.67 with a 2.5 sigma cutoff and 512 to about a million
particles (Sec. 4, Table 1 and the microcell study); no dataset is involved.
The configurations below keep those shapes and add the two-species mixture,
the batched isotherm and the gradient workload of the hot-path scope.
"""
from __future__ import annotations

import functools
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


def box_edge(n: int, rho: float) -> float:
    """Edge of the cubic box holding n particles at reduced density rho."""
    return float((n / rho) ** (1.0 / 3.0))


def uniform_positions(n: int, L: float, seed: int) -> np.ndarray:
    """n positions uniform in [0, L)^3 (float64, shape (n, 3))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.random((n, 3)) * L


def separated_positions(n: int, L: float, dmin: float, seed: int) -> np.ndarray:
    """n positions in the periodic box [0, L)^3 with no two closer than dmin
    (minimum image): random sequential addition -- uniform candidates, each
    kept if it keeps dmin from every position kept before.  The candidates
    come from one PCG64 stream, so the result depends only on the arguments.
    Raises ValueError when 1000 n candidates do not suffice (a packing beyond
    what random sequential addition reaches)."""
    return _separated(int(n), float(L), float(dmin), int(seed)).copy()


@functools.lru_cache(maxsize=4)
def _separated(n: int, L: float, dmin: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    g = max(1, int(L // dmin))  # hash cells of edge >= dmin: partners lie in the 27 around
    h, half, d2 = L / g, 0.5 * L, dmin * dmin
    cells = {}
    out = []
    tried = 0
    while len(out) < n:
        tried += 4096
        if tried > 1000 * max(n, 1) + 4096:
            raise ValueError("separated_positions: %d points %.3g apart do not fit in a box of %.3g"
                             % (n, dmin, L))
        for px, py, pz in (rng.random((4096, 3)) * L).tolist():
            cx, cy, cz = int(px / h) % g, int(py / h) % g, int(pz / h) % g
            ok = True
            for ix in ((cx - 1) % g, cx, (cx + 1) % g):
                for iy in ((cy - 1) % g, cy, (cy + 1) % g):
                    for iz in ((cz - 1) % g, cz, (cz + 1) % g):
                        for qx, qy, qz in cells.get((ix, iy, iz), ()):
                            dx, dy, dz = px - qx, py - qy, pz - qz
                            dx = dx - L if dx > half else (dx + L if dx < -half else dx)
                            dy = dy - L if dy > half else (dy + L if dy < -half else dy)
                            dz = dz - L if dz > half else (dz + L if dz < -half else dz)
                            if dx * dx + dy * dy + dz * dz < d2:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                cells.setdefault((cx, cy, cz), []).append((px, py, pz))
                out.append((px, py, pz))
                if len(out) == n:
                    break
    arr = np.array(out, dtype=np.float64)
    arr.setflags(write=False)
    return arr


def species_labels(n: int, fractions, seed: int) -> np.ndarray:
    """int32 species labels drawn independently with the given fractions."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x5EED))
    fr = np.asarray(fractions, dtype=np.float64)
    return rng.choice(len(fr), size=n, p=fr / fr.sum()).astype(np.int32)


def lorentz_berthelot(eps_species, sigma_species):
    """Pair tables from per-species parameters: sigma_ab = (sigma_a + sigma_b)/2,
    eps_ab = sqrt(eps_a eps_b) (the caller-side mixing rule)."""
    e = np.asarray(eps_species, dtype=np.float64)
    s = np.asarray(sigma_species, dtype=np.float64)
    return np.sqrt(np.outer(e, e)), 0.5 * (s[:, None] + s[None, :])


@dataclass
class Workload:
    name: str
    n: int
    rho: float
    rc: float
    temperature: float
    eps: np.ndarray
    sigma: np.ndarray
    fractions: List[float]
    log_z: List[float]
    p_disp: float = 1.0 / 3.0
    p_ins: float = 1.0 / 3.0
    p_del: float = 1.0 / 3.0
    max_disp: float = 0.3
    moves: int = 10_000
    seed: int = 1
    L: float = field(default=0.0)
    dmin: float = 0.0  # > 0: initial positions at least dmin apart (random sequential addition)

    def __post_init__(self):
        if self.L == 0.0:
            self.L = box_edge(self.n, self.rho)

    @property
    def beta(self) -> float:
        return 1.0 / self.temperature

    def positions(self) -> np.ndarray:
        if self.dmin > 0.0:
            return separated_positions(self.n, self.L, self.dmin, self.seed)
        return uniform_positions(self.n, self.L, self.seed)

    def types(self) -> np.ndarray:
        if len(self.fractions) == 1:
            return np.zeros(self.n, np.int32)
        return species_labels(self.n, self.fractions, self.seed)


def _single(eps=1.0, sigma=1.0):
    return np.array([[eps]]), np.array([[sigma]])


# Chemical potentials: ln z = beta mu (Lambda = 1).  The values were set with
# the oracle's Widom test-particle average on configurations equilibrated by
# the oracle's own chain at the target density (oracle/estimate_mu.py); they
# only steer <N> towards N0 and enter every comparison as plain inputs.
LOGZ_C1 = -2.786
LOGZ_C2 = -1.405
LOGZ_C3 = (-0.012, 0.817)
LOGZ_C5 = (-1.193, -1.086)

# ln z along the T* = 1.2, rc = 2.5 isotherm at these densities (same script)
ISO_RHO = (0.1, 0.15, 0.2, 0.25, 0.3, 0.35, 0.4, 0.45, 0.5, 0.55, 0.6, 0.65, 0.7)
ISO_LOGZ = (-2.9274, -2.7906, -2.7883, -2.7456, -2.7257, -2.7801, -2.7521, -2.7273, -2.7114,
            -2.729, -2.3514, -2.2062, -1.9642)


# The cutoff sweep (Sec. 4, "Performance impact of different cutoffs"): a fixed
# initial configuration of 87,296 particles in 131,072 sigma^3 (rho ~ 0.666)
# with rc from 2.5 to 4.25 sigma.  The temperature is not printed; T* 1.5 keeps
# the fluid supercritical at every cutoff.
SWEEP_N = 87296
SWEEP_V = 131072.0
SWEEP_T = 1.5
SWEEP_RC = (2.5, 2.75, 3.0, 3.25, 3.5, 3.75, 4.0, 4.25)
SWEEP_LOGZ = (-0.6439, -0.7842, -0.8303, -0.9137, -0.8561, -0.9926, -1.1244, -1.0134)


def c1_plain_fp64() -> Workload:
    """2,048 particles, rho 0.5 (L = 16), rc 2.5, T* 1.2, 1e4 moves, seed 1."""
    e, s = _single()
    return Workload("lj-2048-rho0.5-rc2.5", 2048, 0.5, 2.5, 1.2, e, s, [1.0], [LOGZ_C1],
                    moves=10_000, seed=1)


def c2_fp32_vs_fp64() -> Workload:
    """131,072 particles, rho 0.6, rc 3.0, T* 1.5, 1e6 moves."""
    e, s = _single()
    return Workload("lj-131072-rho0.6-rc3.0", 131072, 0.6, 3.0, 1.5, e, s, [1.0], [LOGZ_C2],
                    moves=1_000_000, seed=2)


def c3_mixture_1m() -> Workload:
    """1,048,576 particles, 80/20 mixture (sigma 1/1.2, eps 1/0.8, Lorentz-Berthelot),
    rho 0.7, rc = 2.5 sigma_max = 3.0, T* 1.3."""
    e, s = lorentz_berthelot([1.0, 0.8], [1.0, 1.2])
    return Workload("ljmix-1048576-rho0.7-rc3.0", 1 << 20, 0.7, 3.0, 1.3, e, s, [0.8, 0.2],
                    list(LOGZ_C3), moves=1_000_000, seed=3)


def c5_gradient() -> Workload:
    """262,144 particles of the C3 mixture at rho 0.65, rc 3.0."""
    e, s = lorentz_berthelot([1.0, 0.8], [1.0, 1.2])
    return Workload("ljmix-262144-rho0.65-rc3.0", 1 << 18, 0.65, 3.0, 1.3, e, s, [0.8, 0.2],
                    list(LOGZ_C5), moves=0, seed=5)


def cutoff_sweep(rc: float, moves: int = 1_000_000) -> Workload:
    """87,296 particles, V = 131,072 (L = 50.80), T* 1.5, cutoff rc (one of
    SWEEP_RC); one fixed initial configuration for every cutoff: random
    sequential addition with pairs at least 0.9 sigma apart (seed 6)."""
    k = SWEEP_RC.index(rc)
    e, s = _single()
    return Workload("lj-87296-V131072-rc%.2f" % rc, SWEEP_N, SWEEP_N / SWEEP_V, rc, SWEEP_T, e, s, [1.0],
                    [SWEEP_LOGZ[k]], moves=moves, seed=6, L=SWEEP_V ** (1.0 / 3.0), dmin=0.9)


def isotherm_chains(n_chains: int = 64, seed: int = 4, n_min: int = 500, n_max: int = 20000,
                    rho_min: float = 0.1, rho_max: float = 0.7) -> List[Workload]:
    """The batched isotherm: n_chains single-species chains with N0 log-uniform in
    [n_min, n_max], rho linearly spaced, rc 2.5, T* 1.2, 1e5 moves each.
    ln z per chain is interpolated from the isotherm table above."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.exp(rng.uniform(np.log(n_min), np.log(n_max), n_chains)).astype(np.int64)
    rhos = np.linspace(rho_min, rho_max, n_chains)
    e, s = _single()
    out = []
    for k in range(n_chains):
        lz = float(np.interp(rhos[k], ISO_RHO, ISO_LOGZ))
        out.append(Workload("iso-%02d" % k, int(ns[k]), float(rhos[k]), 2.5, 1.2, e, s, [1.0],
                            [lz], moves=100_000, seed=1000 + k))
    return out



def tiny_system(n: int = 48, L: float = 7.5, rc: float = 2.5, n_species: int = 1,
                seed: int = 11):
    """A small random system for brute-force comparisons: (pos, types, eps, sigma)."""
    pos = uniform_positions(n, L, seed)
    if n_species == 1:
        e, s = _single()
        t = np.zeros(n, np.int32)
    else:
        eps_sp = np.linspace(1.0, 0.6, n_species)
        sig_sp = np.linspace(1.0, 1.3, n_species)
        e, s = lorentz_berthelot(eps_sp, sig_sp)
        t = species_labels(n, np.ones(n_species) / n_species, seed)
    return pos, t, e, s


def insertion_points(m: int, L: float, n_species: int, seed: int):
    """m uniform trial positions with uniform species labels."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x1F5))
    pos = rng.random((m, 3)) * L
    sp = rng.integers(0, n_species, m).astype(np.int32)
    return pos, sp
