"""Oracle microcells (Sec. 3.3): the microcell lists against their definition,
their upkeep over a chain, and the cube of microcells that covers the cutoff.

* Build: M = ceil(L / edge) cells per side of edge L / M; a particle at real
  coordinate x lies in microcell floor(x / (L / M)) on each axis (checked
  with exact rational arithmetic from x = X L / 2^32); every particle is
  listed once; lists run species by species, index by index (Sec. 3.3.1).
* Moves: after a chain with microcells built, every particle is still listed
  exactly once, in the microcell of its current position, and the chain's
  decisions are those of a chain without microcells.
* Cube: every pair within the cutoff lies within D microcells of each other
  along each axis (minimum image), D = 1 + floor((rcg - 1) M / 2^32), rcg the
  smallest integer with rcg^2 >= R2 -- the half-width of the cube of
  microcells the GPU evaluates; the paper's mapping example of threads to
  microcells (Sec. 3.3.2, tests/golden/microcell_mapping.txt); a particle's
  energy summed over its cube equals the brute-force sum over all particles.
"""
import os
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1408_3764_gb300 import workloads as W


def _lists(o):
    M, cnt, refs, mx = o.micro_state()
    out, k = [], 0
    for c in range(M ** 3):
        out.append([(int(r) & 0xFF, int(r) >> 8) for r in refs[k:k + cnt[c]]])
        k += cnt[c]
    return M, out, mx


def _positions(o):
    cnt, X, _, _ = o.state()
    ids = [(s, i) for s in range(len(cnt)) for i in range(cnt[s])]
    return ids, X


def _micro_exact(X, M):
    # x = X L / 2^32; cell = floor(x / (L / M)) = floor(X M / 2^32), as a fraction
    return tuple(math.floor(Fraction(int(v) * M, 2 ** 32)) for v in X)


@pytest.mark.parametrize("n,L,S,edge", [(300, 8.3, 1, 1.0), (700, 11.0, 2, 1.0), (500, 9.7, 1, 0.8)])
def test_micro_build_matches_definition(n, L, S, edge):
    pos, types, eps, sigma = W.tiny_system(n=n, L=L, rc=2.5, n_species=S, seed=n)
    o = O.System(L, 2.5, eps, sigma)
    o.build(pos, types)
    M = o.micro_build(edge)
    assert M == math.ceil(L / edge)
    M_, lists, mx = _lists(o)
    ids, X = _positions(o)
    where = {}
    for c, lst in enumerate(lists):
        for r in lst:
            assert r not in where, "listed twice"
            where[r] = c
        assert lst == sorted(lst), "lists run species by species, index by index"
    assert len(where) == len(ids)
    for (s, i), P in zip(ids, X):
        cx, cy, cz = _micro_exact(P, M)
        assert where[(s, i)] == (cz * M + cy) * M + cx
    assert mx == max(len(lst) for lst in lists)


def test_micro_lists_follow_the_moves():
    L, n = 10.0, 600
    pos, types, eps, sigma = W.tiny_system(n=n, L=L, rc=2.5, n_species=2, seed=5)
    args = (0.4, 0.3, 0.3, 0.4, 1 / 1.2, [-2.3, -2.6])
    a = O.System(L, 2.5, eps, sigma)
    a.build(pos, types)
    a.set_energy(a.total_energy())
    b = O.System(L, 2.5, eps, sigma)
    b.build(pos, types)
    b.set_energy(b.total_energy())
    M = b.micro_build(1.0)
    ta, _ = a.run_moves(3, 0, 20_000, *args)
    tb, sb = b.run_moves(3, 0, 20_000, *args)
    assert np.array_equal(ta, tb)  # the microcells change no decision
    assert sb.accepted[1] > 100 and sb.accepted[2] > 100 and sb.accepted[0] > 1000
    _, lists, _ = _lists(b)
    ids, X = _positions(b)
    where = {}
    for c, lst in enumerate(lists):
        for r in lst:
            assert r not in where, "listed twice"
            where[r] = c
    assert len(where) == len(ids)
    for (s, i), P in zip(ids, X):
        cx, cy, cz = _micro_exact(P, M)
        assert where[(s, i)] == (cz * M + cy) * M + cx
    # a fresh build lists the same particles per cell (in species-major order)
    fresh = O.System(L, 2.5, eps, sigma)
    cnt, Xg, _, _ = b.state()
    fresh.build(Xg.astype(np.float64) * (L / 2.0 ** 32), np.repeat(np.arange(2), cnt).astype(np.int32))
    fresh.micro_build(1.0)
    _, lists_f, _ = _lists(fresh)
    assert [sorted(x) for x in lists] == lists_f


@pytest.mark.parametrize("n,L,rc,edge", [(2500, 12.0, 2.5, 1.0), (3000, 14.2, 4.25, 1.0), (400, 7.3, 3.0, 1.0),
                                         (1200, 10.0, 3.0, 1.0), (1500, 11.1, 2.75, 0.9)])
def test_micro_cube_covers_the_cutoff(n, L, rc, edge):
    o = O.System(L, rc, [[1.0]], [[1.0]])
    o.build(W.uniform_positions(n, L, 11), np.zeros(n, np.int32))
    M = o.micro_build(edge)
    R2 = o.R2
    rcg = math.isqrt(R2 - 1) + 1  # smallest integer with rcg^2 >= R2
    assert rcg * rcg >= R2 and (rcg - 1) ** 2 < R2
    D = 1 + ((rcg - 1) * M >> 32)
    _, X = _positions(o)
    X = X.astype(np.int64)
    cell = (X * M) >> 32
    worst = 0
    for p in range(len(X)):
        d = X[p + 1:] - X[p]
        d = np.where(d >= 2 ** 31, d - 2 ** 32, np.where(d < -(2 ** 31), d + 2 ** 32, d))
        # each square is below 2^62, so the sum of three fits in uint64
        g = (d * d).astype(np.uint64).sum(1)
        inside = g < np.uint64(R2)
        if not inside.any():
            continue
        dc = np.abs(cell[p + 1:][inside] - cell[p])
        dc = np.minimum(dc, M - dc)
        worst = max(worst, int(dc.max()))
        assert (dc <= D).all()
    # the bound is attained or one cell short of it (it is not loose)
    assert worst >= min(D, M // 2) - 1


GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cube_half_width(o, M):
    rcg = math.isqrt(o.R2 - 1) + 1
    return 1 + ((rcg - 1) * M >> 32)


def test_microcell_mapping_example():
    rows = [list(map(int, ln.split())) for ln in open(os.path.join(GOLDEN, "microcell_mapping.txt"))
            if ln.strip() and not ln.startswith("#")]
    o = O.System(20.0, 2.5, [[1.0]], [[1.0]])
    o.build(np.zeros((0, 3)), np.zeros(0, np.int32))
    M = o.micro_build(1.0)
    assert M == 20
    D = _cube_half_width(o, M)
    for cx, cy, cz, n, tx, ty, tz, x, y, z in rows:
        assert 2 * D + 1 == n  # a 2.5 sigma cutoff needs the 7 x 7 x 7 cube
        cube = o.micro_cube((cx, cy, cz), D)
        assert len(cube) == n ** 3 == 343
        c = int(cube[tx + n * ty + n * n * tz])
        assert (c % M, (c // M) % M, c // (M * M)) == (x, y, z)
    # a 2.75 sigma cutoff needs the same cube
    o2 = O.System(20.0, 2.75, [[1.0]], [[1.0]])
    o2.build(np.zeros((0, 3)), np.zeros(0, np.int32))
    assert 2 * _cube_half_width(o2, o2.micro_build(1.0)) + 1 == 7


@pytest.mark.parametrize("n,L,rc,S", [(900, 11.0, 2.5, 2), (1200, 12.5, 3.75, 1),
                                      (150, 6.3, 3.0, 1)])
def test_micro_cube_energy_equals_brute_force(n, L, rc, S):
    pos, types, eps, sigma = W.tiny_system(n=n, L=L, rc=rc, n_species=S, seed=n + 3)
    o = O.System(L, rc, eps, sigma)
    o.build(pos, types)
    M = o.micro_build(1.0)
    D = _cube_half_width(o, M)
    cnt, X, _, _ = o.state()
    ids = [(s, i) for s in range(S) for i in range(cnt[s])]
    rng = np.random.default_rng(n)
    for r in rng.choice(len(ids), size=min(60, len(ids)), replace=False):
        s, i = ids[r]
        e_m, u_m = o.energy_micro(X[r], s, (s, i), D)
        e_b, u_b = o.energy_brute_grid(X[r], s, (s, i))
        assert e_m == pytest.approx(e_b, rel=1e-13, abs=1e-13 * u_b) and u_m == pytest.approx(u_b, rel=1e-13)
    for P in rng.integers(0, 2 ** 32, size=(40, 3), dtype=np.uint64).astype(np.uint32):
        e_m, u_m = o.energy_micro(P, 0, (-1, -1), D)
        e_b, u_b = o.energy_brute_grid(P, 0, (-1, -1))
        assert e_m == pytest.approx(e_b, rel=1e-13, abs=1e-13 * u_b) and u_m == pytest.approx(u_b, rel=1e-13)
