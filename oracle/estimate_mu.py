"""Estimates ln z = beta mu (Lambda = 1) for the synthetic workloads with the oracle.

For each (density, temperature, cutoff, force field) it equilibrates a small
box at that density with the oracle's own canonical chain (displacements
only), then averages the Widom test-particle factor <exp(-beta e)> over
random insertion points:  beta mu_ex = -ln <exp(-beta e)>, and
ln z_s = ln(rho x_s) + beta mu_ex,s  for species s at mole fraction x_s.

The numbers it prints are pasted into paper_1408_3764_gb300/workloads.py as
plain input parameters; nothing reads this script at run time.
"""
from __future__ import annotations

import sys

import numpy as np

import oracle as O
from paper_1408_3764_gb300 import workloads as W


def estimate(rho, T, rc, eps, sigma, fractions, n=1000, sweeps=150, widom=200_000, seed=7):
    L = W.box_edge(n, rho)
    pos = W.uniform_positions(n, L, seed)
    types = (np.zeros(n, np.int32) if len(fractions) == 1
             else W.species_labels(n, fractions, seed))
    s = O.System(L, rc, eps, sigma)
    s.build(pos, types)
    s.set_energy(s.total_energy())
    beta = 1.0 / T
    s.run_moves(seed, 0, sweeps * n, 1.0, 0.0, 0.0, 0.15, beta, [0.0] * len(fractions),
                trace=False)
    out = []
    for sp, x in enumerate(fractions):
        w = s.widom(sp, beta, seed + 17 * sp, widom)
        out.append(float(np.log(rho * x) - np.log(w)))
    return out


def sweep():
    """ln z along the cutoff sweep (87,296 particles in 131,072 sigma^3, T* 1.5)."""
    e1, s1 = np.array([[1.0]]), np.array([[1.0]])
    rho = W.SWEEP_N / W.SWEEP_V
    vals = [estimate(rho, W.SWEEP_T, rc, e1, s1, [1.0], n=2000, sweeps=100, widom=100_000)[0]
            for rc in W.SWEEP_RC]
    print("SWEEP_LOGZ", [round(v, 4) for v in vals])
    sys.stdout.flush()


def main():
    if sys.argv[1:] == ["sweep"]:
        return sweep()
    e1, s1 = np.array([[1.0]]), np.array([[1.0]])
    em, sm = W.lorentz_berthelot([1.0, 0.8], [1.0, 1.2])
    print("C1", estimate(0.5, 1.2, 2.5, e1, s1, [1.0]))
    print("C2", estimate(0.6, 1.5, 3.0, e1, s1, [1.0]))
    print("C3", estimate(0.7, 1.3, 3.0, em, sm, [0.8, 0.2]))
    print("C5", estimate(0.65, 1.3, 3.0, em, sm, [0.8, 0.2]))
    grid = np.linspace(0.1, 0.7, 13)
    vals = [estimate(r, 1.2, 2.5, e1, s1, [1.0], n=600, sweeps=100, widom=100_000)[0]
            for r in grid]
    print("ISO_RHO", [round(float(r), 4) for r in grid])
    print("ISO_LOGZ", [round(v, 4) for v in vals])
    sys.stdout.flush()


if __name__ == "__main__":
    main()
