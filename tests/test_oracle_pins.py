"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: a closed form of Eq. 1, a
worked example printed in the paper (tests/golden/), a textbook numpy
evaluation written independently of the C code, an invariant, a library
implementation of Philox, or an exact statistical law of the ensemble.
"""
import math
import os
import subprocess
import sys
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1408_3764_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- Eq. 1 ----

def test_lj_closed_forms():
    """Eq. 1: U(sigma) = 0, U(2^(1/6) sigma) = -eps, U'(2^(1/6) sigma) = 0."""
    for eps, sig in [(1.0, 1.0), (0.8, 1.2), (0.5, 0.9)]:
        u, rep, att = O.lj(sig * sig, eps, sig)
        assert abs(u) <= 1e-14 * rep
        rmin2 = (2.0 ** (1.0 / 6.0) * sig) ** 2
        u, _, _ = O.lj(rmin2, eps, sig)
        assert u == pytest.approx(-eps, rel=1e-14)
        assert abs(O.lj_dr(rmin2, eps, sig)) <= 1e-12 * eps / sig
        # rep and att are the two terms of Eq. 1
        u, rep, att = O.lj(2.0, eps, sig)
        assert rep == pytest.approx(4 * eps * (sig * sig / 2.0) ** 6, rel=1e-15)
        assert att == pytest.approx(4 * eps * (sig * sig / 2.0) ** 3, rel=1e-15)


def test_lj_value_at_cutoff():
    """U(2.5) = 4 (2.5^-12 - 2.5^-6) = -0.0163168911...; the jump the cutoff makes."""
    u, _, _ = O.lj(6.25, 1.0, 1.0)
    assert u == pytest.approx(-0.016316891136, rel=1e-10)


def test_lj_derivatives_against_finite_differences():
    """U'(r) and dU/dsigma against central differences of U (which is pinned above)."""
    for r in [0.95, 1.1, 1.5, 2.2]:
        for eps, sig in [(1.0, 1.0), (0.894, 1.1)]:
            h = 1e-6
            fd = (O.lj((r + h) ** 2, eps, sig)[0] - O.lj((r - h) ** 2, eps, sig)[0]) / (2 * h)
            assert O.lj_dr(r * r, eps, sig) == pytest.approx(fd, rel=1e-7, abs=1e-9)
            fd = (O.lj(r * r, eps, sig + h)[0] - O.lj(r * r, eps, sig - h)[0]) / (2 * h)
            assert O.lj_dsigma(r * r, eps, sig) == pytest.approx(fd, rel=1e-7, abs=1e-9)


def test_lj_zero_distance_is_infinite():
    assert O.lj(0.0, 1.0, 1.0)[0] == math.inf


# ------------------------------------------------------- Sec. 3.2.2 -------

def test_cell_size_worked_example():
    """Sec. 3.2.2: rc 2.5, L 23.9 -> S 2.656, T 9; L < 3 rc -> S = L/3."""
    for L, rc, T, S in _golden("cell_size_example.txt"):
        L, rc, T, S = float(L), float(rc), int(T), float(S)
        assert O.cells_per_side(L, rc) == T
        assert round(L / T, 3) == S


def test_volume_examples():
    """Sec. 3.3: the sphere/27-cell volumes quoted in the paper."""
    g = {k: float(v) for k, v in _golden("volume_examples.txt")}
    assert round(4.0 / 3.0 * math.pi * 2.5 ** 3, 2) == g["sphere_rc2.5"]
    assert 27 * 2.75 ** 3 == pytest.approx(g["cells27_S2.75"], abs=0.05)
    assert 27 * 2.5 ** 3 == g["cells27_S2.5"]
    assert 4.0 / 3.0 * math.pi * 2.5 ** 3 / (27 * 2.5 ** 3) < g["inside_fraction_S2.5"]


def test_cells_per_side_maximal():
    """T is the largest integer with L/T >= rc (and at least 3)."""
    rng = np.random.default_rng(5)
    for _ in range(200):
        rc = rng.uniform(1.0, 4.0)
        L = rng.uniform(2 * rc, 40.0)
        T = O.cells_per_side(L, rc)
        if L >= 3 * rc:
            assert Fraction(L) / T >= Fraction(rc)
            assert Fraction(L) / (T + 1) < Fraction(rc)
        else:
            assert T == 3


# ----------------------------------------------------------- binning ------

@pytest.mark.parametrize("n,L,rc", [(300, 7.5, 2.5), (700, 16.0, 2.5), (500, 11.0, 3.0)])
def test_build_cells_exact(n, L, rc):
    """Every particle sits in the cell floor(x/S) of its grid position (exact
    rational arithmetic), cells list particles in input order, counts sum to N."""
    pos = W.uniform_positions(n, L, 3)
    types = np.zeros(n, np.int32)
    s = O.System(L, rc, [[1.0]], [[1.0]])
    cl = s.build(pos, types)
    T = s.T
    assert cl.cell_count.sum() == n
    assert sorted(cl.order.tolist()) == list(range(n))
    _, gpos, _, _ = s.state()
    S = Fraction(L) / T
    h = Fraction(L) / 2 ** 32
    for c in range(s.ncell):
        members = cl.order[cl.cell_start[c]: cl.cell_start[c] + cl.cell_count[c]]
        assert list(members) == sorted(members)
        for p in members:
            cx = [int((int(gpos[p, a]) * h) // S) for a in range(3)]
            assert (cx[2] * T + cx[1]) * T + cx[0] == c
    # quantisation: the grid point is within one grid step below the input
    for p in range(0, n, 37):
        for a in range(3):
            x = Fraction(float(pos[p, a]))
            X = int(gpos[p, a])
            assert 0 <= x - X * h <= h * Fraction(1000001, 1000000)


def test_quantize_wraps_periodically():
    L = 10.0
    assert O.quantize(0.0, L) == 0
    assert O.quantize(L, L) == 0
    assert O.quantize(-L / 2, L) == 2 ** 31
    assert O.quantize(2.5 * L, L) == 2 ** 31


# ------------------------------------------- textbook brute force ----------

def _textbook_energy(P, t, X, types, eps, sigma, L, rc, exclude=None):
    """Independent numpy restatement: real coordinates, d -= L rint(d/L), r < rc."""
    h = L / 2.0 ** 32
    x = X.astype(np.float64) * h
    p = np.asarray(P, np.float64) * h
    d = p[None, :] - x
    d -= L * np.rint(d / L)
    r2 = (d * d).sum(1)
    keep = r2 < rc * rc
    if exclude is not None:
        keep[exclude] = False
    e = eps[t, types[keep]]
    sg = sigma[t, types[keep]]
    sr6 = (sg * sg / r2[keep]) ** 3
    u = 4 * e * (sr6 * sr6 - sr6)
    return u.sum(), np.abs(4 * e * sr6 * sr6).sum() + np.abs(4 * e * sr6).sum()


@pytest.mark.parametrize("n,L,rc,S", [(60, 7.5, 2.5, 1), (200, 9.0, 2.5, 2), (500, 13.0, 3.0, 2),
                                      (400, 14.0, 2.5, 3)])
def test_energies_match_textbook_brute_force(n, L, rc, S):
    pos, types, eps, sigma = W.tiny_system(n=n, L=L, rc=rc, n_species=S, seed=n)
    s = O.System(L, rc, eps, sigma)
    s.build(pos, types)
    cnt, X, _, _ = s.state()
    # species-major order of the oracle's particles
    tsm = np.repeat(np.arange(S), cnt).astype(np.int64)
    # trial insertions
    tp, ts = W.insertion_points(40, L, S, 9)
    e_cells, uabs = s.trial_energy(tp, ts, with_abs=True)
    e_brute = s.trial_energy(tp, ts, brute=True)
    for k in range(len(tp)):
        P = np.array([O.quantize(v, L) for v in tp[k]], dtype=np.uint64)
        ref, scale = _textbook_energy(P, ts[k], X, tsm, eps, sigma, L, rc)
        assert abs(e_cells[k] - ref) <= 1e-12 * scale + 1e-300
        assert abs(e_brute[k] - ref) <= 1e-12 * scale + 1e-300
        assert uabs[k] == pytest.approx(scale, rel=1e-10)
    # total energy: cells, brute, textbook pair sum
    tot = 0.0
    for a in range(len(X)):
        tot += _textbook_energy(X[a].astype(np.uint64), tsm[a], X, tsm, eps, sigma, L, rc,
                                exclude=a)[0]
    tot *= 0.5
    assert s.total_energy() == pytest.approx(tot, rel=1e-11)
    assert s.total_energy(brute=True) == pytest.approx(tot, rel=1e-11)


def test_total_energy_is_half_sum_of_particle_energies():
    pos, types, eps, sigma = W.tiny_system(n=300, L=10.0, n_species=2, seed=4)
    s = O.System(10.0, 2.5, eps, sigma)
    s.build(pos, types)
    assert s.total_energy() == pytest.approx(0.5 * s.particle_energies().sum(), rel=1e-13)


def test_translation_invariance_exact():
    """A global periodic translation by a whole number of grid steps leaves every
    pair separation, hence the total energy, bit-for-bit unchanged."""
    L, rc = 9.0, 2.5
    pos, types, eps, sigma = W.tiny_system(n=250, L=L, n_species=2, seed=8)
    a = O.System(L, rc, eps, sigma)
    a.build(pos, types)
    _, X, _, _ = a.state()
    h = L / 2.0 ** 32
    cnt = a.counts()
    tsm = np.repeat(np.arange(2), cnt).astype(np.int32)
    shift = np.array([123456789, 3000000000, 77], dtype=np.uint64)
    X2 = (X.astype(np.uint64) + shift) % (2 ** 32)
    # grid points are exactly representable as X * h (X < 2^32, h a power-of-two
    # scaling of L); add half a step so the floor lands on X
    pos2 = (X2.astype(np.float64) + 0.5) * h
    b = O.System(L, rc, eps, sigma)
    b.build(pos2, tsm)
    _, Xb, _, _ = b.state()
    assert np.array_equal(Xb.astype(np.uint64), X2)
    ea, eb = a.total_energy(brute=True), b.total_energy(brute=True)
    assert ea == pytest.approx(eb, rel=1e-14)


def test_insertion_then_deletion_energy_cancels():
    """dU of inserting a particle at p equals minus dU of deleting it again."""
    L, rc = 10.0, 2.5
    pos, types, eps, sigma = W.tiny_system(n=300, L=L, n_species=2, seed=21)
    s = O.System(L, rc, eps, sigma)
    s.build(pos, types)
    tp, ts = W.insertion_points(10, L, 2, 5)
    e_ins = s.trial_energy(tp, ts)
    for k in range(len(tp)):
        s2 = O.System(L, rc, eps, sigma)
        s2.build(np.vstack([pos, tp[k:k + 1]]), np.concatenate([types, ts[k:k + 1]]))
        i_new = int((types == ts[k]).sum())  # its index within its species
        e_del = s2.trial_energy(tp[k:k + 1], ts[k:k + 1],
                                exclude=[(int(ts[k]) << 32) | i_new])[0]
        assert e_ins[k] == pytest.approx(e_del, rel=1e-13, abs=1e-13)


# --------------------------------------------------------------- Philox ----

_TRITON_SCRIPT = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl
from triton.language.random import philox

@triton.jit
def k(c_ptr, s_ptr, out_ptr):
    c0 = tl.load(c_ptr + 0).to(tl.uint32)
    c1 = tl.load(c_ptr + 1).to(tl.uint32)
    c2 = tl.load(c_ptr + 2).to(tl.uint32)
    c3 = tl.load(c_ptr + 3).to(tl.uint32)
    seed = tl.load(s_ptr).to(tl.uint64)
    a, b, c, d = philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 0, a.to(tl.int64))
    tl.store(out_ptr + 1, b.to(tl.int64))
    tl.store(out_ptr + 2, c.to(tl.int64))
    tl.store(out_ptr + 3, d.to(tl.int64))

res = []
for ctr, seed in json.loads(sys.argv[1]):
    c = torch.tensor(ctr, dtype=torch.int64)
    s = torch.tensor([seed], dtype=torch.uint64)
    out = torch.zeros(4, dtype=torch.int64)
    k[(1,)](c, s, out)
    res.append([int(v) & 0xffffffff for v in out])
print(json.dumps(res))
"""


def test_philox_matches_triton_library():
    """The oracle's Philox4x32-10 against triton's implementation, run on the CPU
    through triton's interpreter (a library pin, not a retyping)."""
    pytest.importorskip("triton")
    import json
    cases = [([0, 0, 0, 0], 0), ([1, 0, 0, 0], 0), ([0xFFFFFFFF] * 4, 0xFFFFFFFFFFFFFFFF),
             ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], 0x299F31D0A4093822),
             ([12345, 678, 3, 1], 1), ([7, 0, 63, 0], (2 ** 40) + 99)]
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT, json.dumps(cases)],
                       capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + r.stderr[-300:])
    ref = json.loads(r.stdout.strip().splitlines()[-1])
    for (ctr, seed), want in zip(cases, ref):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        got = O.philox4x32_10(ctr, key)
        assert [int(v) for v in got] == want


def test_move_words_layout():
    """Move m of chain c uses counters (m_lo, m_hi, c, 0) and (m_lo, m_hi, c, 1)."""
    seed, m, c = 0x1234_5678_9ABC_DEF0, 2 ** 33 + 5, 3
    w = O.move_words(seed, m, c)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    assert list(w[:4]) == list(O.philox4x32_10([m & 0xFFFFFFFF, m >> 32, c, 0], key))
    assert list(w[4:]) == list(O.philox4x32_10([m & 0xFFFFFFFF, m >> 32, c, 1], key))


# ------------------------------------------------------------- gradient ----

def _fd_system(L, rc, eps, sigma, pos, types):
    s = O.System(L, rc, eps, sigma)
    s.build(pos, types)
    return s


def test_gradient_cells_equals_brute():
    pos, types, eps, sigma = W.tiny_system(n=120, L=9.0, n_species=2, seed=31)
    s = _fd_system(9.0, 2.5, eps, sigma, pos, types)
    g, gb = s.energy_grad(), s.energy_grad(brute=True)
    assert g["energy"] == pytest.approx(gb["energy"], rel=1e-12)
    assert np.allclose(g["dpos"], gb["dpos"], rtol=1e-10, atol=1e-10 * np.abs(gb["dpos"]).max())
    assert np.allclose(g["deps"], gb["deps"], rtol=1e-12)
    assert np.allclose(g["dsigma"], gb["dsigma"], rtol=1e-12)
    assert g["virial"] == pytest.approx(gb["virial"], rel=1e-12)
    assert g["energy"] == pytest.approx(s.total_energy(brute=True), rel=1e-12)


def _relaxed_small(n=80, L=8.0, S=2, seed=41):
    """A low-overlap configuration (so that finite differences are well scaled)."""
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n:
        p = rng.random(3) * L
        ok = True
        for q in pts:
            d = p - q
            d -= L * np.rint(d / L)
            if (d * d).sum() < 0.9 ** 2:
                ok = False
                break
        if ok:
            pts.append(p)
    pos = np.array(pts)
    types = (np.arange(n) % S).astype(np.int32)
    eps, sigma = W.lorentz_berthelot(np.linspace(1.0, 0.8, S), np.linspace(1.0, 1.2, S))
    return pos, types, eps, sigma


def _min_pair_gap_to_cutoff(pos, L, rc):
    d = pos[:, None, :] - pos[None, :, :]
    d -= L * np.rint(d / L)
    r = np.sqrt((d * d).sum(-1))
    np.fill_diagonal(r, 0.0)
    return np.abs(r[r > 0] - rc).min()


def test_gradient_positions_finite_differences():
    L, rc = 8.0, 2.5
    pos, types, eps, sigma = _relaxed_small(L=L)
    s = _fd_system(L, rc, eps, sigma, pos, types)
    g = s.energy_grad()
    # species-major order of the oracle rows
    order = np.concatenate([np.nonzero(types == t)[0] for t in range(2)])
    h = 1e-5
    d = pos[:, None, :] - pos[None, :, :]
    d -= L * np.rint(d / L)
    r = np.sqrt((d * d).sum(-1))
    checked = 0
    for row, p in enumerate(order[:30]):
        if np.any(np.abs(np.delete(r[p], p) - rc) < 4 * h):
            continue
        for a in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[p, a] += h
            pm[p, a] -= h
            ep = _fd_system(L, rc, eps, sigma, pp, types).total_energy(brute=True)
            em = _fd_system(L, rc, eps, sigma, pm, types).total_energy(brute=True)
            fd = (ep - em) / (2 * h)
            assert g["dpos"][row, a] == pytest.approx(fd, rel=2e-4, abs=2e-4)
            checked += 1
    assert checked >= 30


def test_gradient_tables_finite_differences():
    """dE/deps and dE/dsigma: E is linear in eps, so central differences are exact;
    a symmetric change of both table entries of a cross pair gives the full sum."""
    L, rc = 8.0, 2.5
    pos, types, eps, sigma = _relaxed_small(L=L)
    g = _fd_system(L, rc, eps, sigma, pos, types).energy_grad()
    for a in range(2):
        for b in range(a, 2):
            for name, tab in (("deps", eps), ("dsigma", sigma)):
                dh = 1e-6
                tp, tm = tab.copy(), tab.copy()
                tp[a, b] += dh
                tm[a, b] -= dh
                if a != b:
                    tp[b, a] += dh
                    tm[b, a] -= dh
                if name == "deps":
                    ep = _fd_system(L, rc, tp, sigma, pos, types).total_energy(brute=True)
                    em = _fd_system(L, rc, tm, sigma, pos, types).total_energy(brute=True)
                else:
                    ep = _fd_system(L, rc, eps, tp, pos, types).total_energy(brute=True)
                    em = _fd_system(L, rc, eps, tm, pos, types).total_energy(brute=True)
                fd = (ep - em) / (2 * dh)
                want = g[name][a, b] + (g[name][b, a] if a != b else 0.0)
                assert want == pytest.approx(fd, rel=1e-5, abs=1e-6)


def test_virial_is_scaling_derivative():
    """virial = sum_{i<j} r U'(r) = dE/dlambda when box and positions scale by lambda."""
    L, rc = 8.0, 2.5
    pos, types, eps, sigma = _relaxed_small(L=L)
    lam = 1e-7
    assert _min_pair_gap_to_cutoff(pos, L, rc) > 100 * lam * L
    g = _fd_system(L, rc, eps, sigma, pos, types).energy_grad()
    ep = _fd_system(L * (1 + lam), rc, eps, sigma, pos * (1 + lam), types).total_energy(True)
    em = _fd_system(L * (1 - lam), rc, eps, sigma, pos * (1 - lam), types).total_energy(True)
    assert g["virial"] == pytest.approx((ep - em) / (2 * lam), rel=1e-5)
