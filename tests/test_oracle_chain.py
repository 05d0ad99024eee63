"""Pins of the oracle's Markov chain against exact laws of the grand canonical
ensemble (Sec. 2, Eqs. 3-5) and against the cell-list bookkeeping rules of
Sec. 3.2.5.  None of the expected values comes from the oracle.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1408_3764_gb300 import workloads as W


def _n_trajectory(trace, n0):
    step = np.zeros(len(trace), np.int64)
    acc = trace["accepted"].astype(bool)
    step[acc & (trace["type"] == 1)] = 1
    step[acc & (trace["type"] == 2)] = -1
    return n0 + np.cumsum(step)


def _batch_error(x, nb=50):
    b = np.array_split(x, nb)
    m = np.array([v.mean() for v in b])
    return m.std(ddof=1) / math.sqrt(nb)


def test_ideal_gas_is_poisson():
    """eps = 0: P(N) is Poisson(zV), so <N> = Var N = zV, and every displacement
    is accepted.  The paper's printed sign of mu in Eqs. 4-5 would give
    <N> = V/z instead; this fixes the textbook reading."""
    L = 10.0
    V = L ** 3
    z = 0.05
    s = O.System(L, 2.5, [[0.0]], [[1.0]])
    s.build(W.uniform_positions(20, L, 1), np.zeros(20, np.int32))
    s.set_energy(s.total_energy())
    tr, st = s.run_moves(7, 0, 400_000, 1 / 3, 1 / 3, 1 / 3, 0.3, 1.0, [math.log(z)])
    n = _n_trajectory(tr, 20)[50_000:]
    assert st.accepted[0] == st.attempted[0]
    err = _batch_error(n.astype(float))
    assert abs(n.mean() - z * V) < max(6 * err, 0.5)
    assert n.var() / (z * V) == pytest.approx(1.0, abs=0.15)
    assert st.energy == 0.0


def test_ideal_gas_mixture_each_species_poisson():
    """Two ideal species: <N_s> = z_s V independently (per-species insertion and
    deletion with the per-species acceptance rule)."""
    L = 10.0
    V = L ** 3
    z = [0.03, 0.08]
    s = O.System(L, 2.5, np.zeros((2, 2)), np.ones((2, 2)))
    s.build(W.uniform_positions(10, L, 2), (np.arange(10) % 2).astype(np.int32))
    s.set_energy(0.0)
    tr, st = s.run_moves(9, 0, 600_000, 0.2, 0.4, 0.4, 0.3, 1.0, [math.log(v) for v in z])
    acc = tr["accepted"].astype(bool)
    for sp in range(2):
        mine = tr["species"] == sp
        step = np.zeros(len(tr), np.int64)
        step[acc & mine & (tr["type"] == 1)] = 1
        step[acc & mine & (tr["type"] == 2)] = -1
        n = 5 + np.cumsum(step)
        n = n[100_000:]
        err = _batch_error(n.astype(float))
        assert abs(n.mean() - z[sp] * V) < max(6 * err, 0.6)
        assert n.var() / (z[sp] * V) == pytest.approx(1.0, abs=0.15)


def test_dimer_separation_distribution():
    """Two particles, displacements only: the separation is distributed as
    r^2 exp(-beta U(r)) for r < L/2 (detailed balance of Eq. 3)."""
    from scipy.integrate import quad

    L, rc, beta = 6.0, 2.5, 1.0 / 1.2
    s = O.System(L, rc, [[1.0]], [[1.0]])
    s.build(np.array([[1.0, 1.0, 1.0], [2.2, 1.0, 1.0]]), np.zeros(2, np.int32))
    s.set_energy(s.total_energy())

    def u(r):
        return 4 * (r ** -12 - r ** -6) if r < rc else 0.0

    def w(r):
        return r * r * math.exp(-beta * u(r))

    edges = np.array([0.9, 1.0, 1.1, 1.25, 1.5, 1.8, 2.1, 2.5, 2.8, 3.0])
    norm = quad(w, 0.7, 3.0, points=[1.12, 2.5], limit=200)[0]
    want = np.array([quad(w, a, b, limit=200)[0] / norm for a, b in zip(edges[:-1], edges[1:])])
    rs = []
    h = L / 2 ** 32
    for k in range(150_000):
        s.run_moves(3, 10 * k, 10, 1.0, 0.0, 0.0, 0.9, beta, [0.0], trace=False)
        _, X, _, _ = s.state()
        d = (X[0].astype(np.int64) - X[1].astype(np.int64) + 2 ** 31) % 2 ** 32 - 2 ** 31
        rs.append(math.sqrt(float(((d * h) ** 2).sum())))
    rs = np.array(rs)
    rs = rs[rs < 3.0]
    got = np.histogram(rs, bins=edges)[0] / len(rs)
    # the mass below 0.9 is ~1e-4; compare bin fractions
    assert np.allclose(got, want, atol=0.012), (got, want)


def test_second_virial_coefficient_low_density():
    """Low-density interacting gas: <N>/V = z - 2 B2 z^2 + O(z^3) with
    B2 = -2 pi int_0^rc (exp(-beta U) - 1) r^2 dr for the truncated potential."""
    from scipy.integrate import quad

    beta, rc = 1.0 / 1.2, 2.5
    B2 = -2 * math.pi * quad(lambda r: (math.exp(-beta * 4 * (r ** -12 - r ** -6)) - 1) * r * r,
                             1e-3, rc, points=[1.0, 1.12], limit=400)[0]
    assert B2 < -1.0  # attractive at T* = 1.2
    z = 0.005
    L = (20000.0) ** (1 / 3)
    V = L ** 3
    s = O.System(L, rc, [[1.0]], [[1.0]])
    n0 = 100
    s.build(W.uniform_positions(n0, L, 4), np.zeros(n0, np.int32))
    s.set_energy(s.total_energy())
    tr, st = s.run_moves(5, 0, 1_500_000, 0.2, 0.4, 0.4, 1.0, beta, [math.log(z)])
    n = _n_trajectory(tr, n0)[200_000:].astype(float)
    want = (z - 2 * B2 * z * z) * V
    err = _batch_error(n)
    assert abs(n.mean() - want) < max(5 * err, 0.8), (n.mean(), want, z * V, err)
    assert n.mean() - z * V > 0.5 * (want - z * V)


def _relaxed(n, L, seed, dmin=0.85):
    rng = np.random.default_rng(seed)
    pts = np.zeros((0, 3))
    while len(pts) < n:
        p = rng.random(3) * L
        if len(pts):
            d = pts - p
            d -= L * np.rint(d / L)
            if ((d * d).sum(1) < dmin * dmin).any():
                continue
        pts = np.vstack([pts, p])
    return pts


def test_chain_bookkeeping_and_energy_consistency():
    """After many moves of a two-species system: every particle is listed once,
    in the cell of its position; the running energy equals the recomputed total
    energy up to the rounding of the accumulated increments."""
    L, rc = 11.0, 2.5
    pos = _relaxed(500, L, 3)
    types = (np.arange(500) % 3 == 0).astype(np.int32)
    eps, sigma = W.lorentz_berthelot([1.0, 0.8], [1.0, 1.1])
    s = O.System(L, rc, eps, sigma)
    s.build(pos, types)
    E0 = s.total_energy()
    s.set_energy(E0)
    tr, st = s.run_moves(11, 0, 30_000, 0.5, 0.25, 0.25, 0.3, 1 / 1.3, [-2.0, -2.5])
    cnt, X, cc, refs = s.state()
    assert cc.sum() == cnt.sum()
    T = s.T
    start = np.concatenate([[0], np.cumsum(cc)])
    seen = set()
    base = np.concatenate([[0], np.cumsum(cnt)])
    for c in range(s.ncell):
        for r in refs[start[c]:start[c + 1]]:
            sp, i = int(r & 0xFF), int(r >> 8)
            assert i < cnt[sp]
            assert (sp, i) not in seen
            seen.add((sp, i))
            Pp = X[base[sp] + i].astype(np.uint64)
            cx = [int((int(v) * T) >> 32) for v in Pp]
            assert (cx[2] * T + cx[1]) * T + cx[0] == c
    assert len(seen) == cnt.sum()
    Ef = s.total_energy()
    assert st.energy == pytest.approx(Ef, abs=1e-9 * max(1.0, abs(E0)) * 10)
    assert st.accepted[1] > 0 and st.accepted[2] > 0 and st.accepted[0] > 0
    # the trace's energy increments add up to the final running energy
    assert E0 + tr["dU"][tr["accepted"] == 1].sum() == pytest.approx(st.energy, rel=1e-12,
                                                                      abs=1e-9)


def test_chain_is_counter_based_resumable():
    """Moves [0, a) then [a, b) give the same chain as [0, b) (Philox counters)."""
    L, rc = 9.0, 2.5
    pos = _relaxed(200, L, 5)
    a = O.System(L, rc, [[1.0]], [[1.0]])
    a.build(pos, np.zeros(200, np.int32))
    a.set_energy(a.total_energy())
    b = O.System(L, rc, [[1.0]], [[1.0]])
    b.build(pos, np.zeros(200, np.int32))
    b.set_energy(b.total_energy())
    ta, _ = a.run_moves(3, 0, 5000, 1 / 3, 1 / 3, 1 / 3, 0.3, 0.8, [-2.5])
    tb1, _ = b.run_moves(3, 0, 2000, 1 / 3, 1 / 3, 1 / 3, 0.3, 0.8, [-2.5])
    tb2, _ = b.run_moves(3, 2000, 3000, 1 / 3, 1 / 3, 1 / 3, 0.3, 0.8, [-2.5])
    assert np.array_equal(ta, np.concatenate([tb1, tb2]))
    sa, sb = a.state(), b.state()
    for x, y in zip(sa, sb):
        assert np.array_equal(x, y)


def test_running_virial_equals_the_recomputed_virial():
    """The chain's running virial W = sum_{i<j} r U'(r), kept by adding each
    accepted trial's dW, equals W recomputed from the final configuration
    (all pairs, analytic derivative) up to the rounding of the increments;
    its per-move sum is the running value summed over the moves."""
    L, rc = 11.0, 2.5
    pos = _relaxed(500, L, 5)
    types = (np.arange(500) % 3 == 0).astype(np.int32)
    eps, sigma = W.lorentz_berthelot([1.0, 0.8], [1.0, 1.1])
    s = O.System(L, rc, eps, sigma)
    s.build(pos, types)
    s.set_energy(s.total_energy())
    W0 = s.energy_grad(brute=True)["virial"]
    _, st1 = s.run_moves(13, 0, 20_000, 0.5, 0.25, 0.25, 0.3, 1 / 1.3, [-2.0, -2.5], trace=False)
    Wf = s.energy_grad(brute=True)["virial"]
    assert st1.virial == pytest.approx(Wf, rel=1e-9, abs=1e-9 * abs(W0))
    assert st1.accepted[1] > 0 and st1.accepted[2] > 0
    assert s.virial() == st1.virial
    # one more move: the sum over the moves grows by the running value
    _, st2 = s.run_moves(13, 20_000, 1, 0.5, 0.25, 0.25, 0.3, 1 / 1.3, [-2.0, -2.5], trace=False)
    assert st2.sum_virial == pytest.approx(st2.virial, rel=1e-15)


def test_ideal_gas_virial_is_zero():
    L = 8.0
    s = O.System(L, 2.5, [[0.0]], [[1.0]])
    s.build(W.uniform_positions(50, L, 6), np.zeros(50, np.int32))
    s.set_energy(0.0)
    _, st = s.run_moves(3, 0, 5_000, 0.4, 0.3, 0.3, 0.5, 1.0, [math.log(0.1)], trace=False)
    assert st.virial == 0.0 and st.sum_virial == 0.0


def test_low_density_virial_matches_the_pair_integral():
    """Low-density interacting gas: the pair correlation is exp(-beta U(r)), so
    <W> = <N (N-1)> / (2V) * 4 pi int_0^rc r^3 U'(r) exp(-beta U(r)) dr up to
    O(rho) corrections (a few per cent here) -- the virial route of the
    pressure P = rho k T - <W> / (3V) for the truncated potential."""
    from scipy.integrate import quad

    beta, rc = 1.0 / 1.2, 2.5

    def du(r):
        return 4 * (-12 * r ** -13 + 6 * r ** -7)

    I = 4 * math.pi * quad(lambda r: r ** 3 * du(r) * math.exp(-beta * 4 * (r ** -12 - r ** -6)),
                           0.5, rc, points=[1.0, 1.12], limit=400)[0]
    z = 0.02
    L = (8000.0) ** (1 / 3)
    V = L ** 3
    s = O.System(L, rc, [[1.0]], [[1.0]])
    n0 = 170
    s.build(W.uniform_positions(n0, L, 8), np.zeros(n0, np.int32))
    s.set_energy(s.total_energy())
    s.run_moves(9, 0, 100_000, 0.2, 0.4, 0.4, 1.0, beta, [math.log(z)], trace=False)  # settle
    means, want = [], []
    n = None
    for k in range(16):
        tr, st = s.run_moves(9, 100_000 + k * 100_000, 100_000, 0.2, 0.4, 0.4, 1.0, beta, [math.log(z)])
        if n is None:
            n0k = int(st.n[0]) - int((tr["accepted"] & (tr["type"] == 1)).sum()) + \
                int((tr["accepted"] & (tr["type"] == 2)).sum())
        else:
            n0k = int(n[-1])
        n = _n_trajectory(tr, n0k).astype(float)
        means.append(st.sum_virial / st.moves_done)
        want.append((n * (n - 1)).mean() / (2 * V) * I)
    means, want = np.array(means), np.array(want)
    err = means.std(ddof=1) / math.sqrt(len(means))
    assert I > 0  # attraction (U' > 0 beyond the minimum) dominates at T* = 1.2: the pressure drops
    assert abs(means.mean() - want.mean()) < max(5 * err, 0.06 * abs(want.mean())), (means.mean(), want.mean(), err)


def test_move_types_follow_the_mix():
    """The attempted move types follow p_disp / p_ins / p_del (unequal here)
    within a 6-sigma binomial bound; swapping two probabilities, or reading
    the thresholds from the wrong side, moves a count by thousands of sigma."""
    L = 8.0
    s = O.System(L, 2.5, [[0.0]], [[1.0]])
    s.build(W.uniform_positions(30, L, 3), np.zeros(30, np.int32))
    s.set_energy(0.0)
    p = (0.5, 0.3, 0.2)
    n = 200_000
    tr, st = s.run_moves(17, 0, n, *p, 0.3, 1.0, [math.log(0.05)])
    for t in range(3):
        cnt = int((tr["type"] == t).sum())
        assert cnt == st.attempted[t]
        sd = math.sqrt(n * p[t] * (1 - p[t]))
        assert abs(cnt - n * p[t]) <= 6 * sd, (t, cnt)


def test_displacement_steps_are_uniform_on_the_grid():
    """An accepted displacement moves each coordinate by a whole number of grid
    steps in [-D, D], D = floor(delta * 2^32 / L) (exact rational arithmetic
    here), uniformly: the extreme steps are reached and a 10-bin histogram
    of each axis passes a chi-square test.  Ideal gas, so every displacement
    is accepted."""
    from fractions import Fraction
    L, delta = 8.0, 0.3
    D = int(Fraction(delta) * (1 << 32) / Fraction(L))
    s = O.System(L, 2.5, [[0.0]], [[1.0]])
    n = 40
    s.build(W.uniform_positions(n, L, 4), np.zeros(n, np.int32))
    s.set_energy(0.0)
    _, X0, _, _ = s.state()
    steps = []
    for m in range(3000):
        tr, _ = s.run_moves(23, m, 1, 1.0, 0.0, 0.0, delta, 1.0, [0.0])
        _, X1, _, _ = s.state()
        i = int(tr["index"][0])
        assert tr["accepted"][0] == 1
        d = (X1[i].astype(np.int64) - X0[i].astype(np.int64) + (1 << 31)) % (1 << 32) - (1 << 31)
        steps.append(d)
        moved = np.ones(n, bool)
        moved[i] = False
        assert np.array_equal(X1[moved], X0[moved])
        X0 = X1
    steps = np.array(steps)
    assert np.abs(steps).max() <= D
    assert np.abs(steps).max() >= 0.99 * D
    for ax in range(3):
        h, _ = np.histogram(steps[:, ax], bins=10, range=(-D - 0.5, D + 0.5))
        expect = len(steps) / 10
        chi2 = ((h - expect) ** 2 / expect).sum()
        assert chi2 < 33.7, (ax, h)  # 9 degrees of freedom, p = 1e-4


def test_sum_abs_u_matches_textbook_brute_force():
    """The per-move sum of |u_j| (the floor of the per-move error measure) of
    insertion trials equals an independent numpy evaluation over all
    particles at the trial's grid point (its Philox words 2-4)."""
    L, rc = 7.5, 2.5
    pos, types, eps, sigma = W.tiny_system(n=60, L=L, rc=rc, n_species=1, seed=5)
    s = O.System(L, rc, eps, sigma)
    s.build(pos, types)
    s.set_energy(s.total_energy())
    _, X, _, _ = s.state()
    Xr = X.astype(np.float64) * (L / 2.0 ** 32)
    tr, _, sabs = s.run_moves(31, 0, 200, 0.0, 1.0, 0.0, 0.3, 1e-9, [-50.0], with_sabs=True)
    assert not tr["accepted"].any()
    for m in range(200):
        w = O.move_words(31, m)
        P = w[2:5].astype(np.float64) * (L / 2.0 ** 32)
        d = Xr - P
        d -= L * np.rint(d / L)
        r2 = (d * d).sum(1)
        r2 = r2[r2 < rc * rc]
        sr6 = (sigma[0, 0] ** 2 / r2) ** 3
        want = np.abs(4 * eps[0, 0] * (sr6 * sr6 - sr6)).sum()
        assert sabs[m] == pytest.approx(want, rel=1e-9, abs=1e-12)
        assert abs(tr["dU"][m]) <= sabs[m] * (1 + 1e-12)


# ---- the particle pick (Algorithm 1: a particle chosen uniformly at random)
def _words(**kv):
    w = np.zeros(8, np.uint32)
    for k, v in kv.items():
        w[int(k[1:])] = v
    return w


def test_pick_index_worked_cases():
    """Values worked out by hand from the rule: 2^k the smallest power of two
    >= n, the top k bits of the tries (deletion: w1, w2, w3; displacement: w1,
    then the top k bits of w1's low half when k <= 16), the first below n
    wins, else floor(f n / 2^32) with f = w4 (deletion) or w5 (displacement)."""
    full = 0xFFFFFFFF
    assert O.pick_index(1, _words(w1=full, w2=full, w3=full, w4=full, w5=full), 2) == 0
    assert O.pick_index(1, _words(w1=full, w5=full), 0) == 0
    # n = 5, k = 3: 0x6... -> top three bits 011 = 3
    assert O.pick_index(5, _words(w1=0x60000000), 2) == 3
    assert O.pick_index(5, _words(w1=0x60000000), 0) == 3
    # first try 7 >= 5, the second (w2 = 0x2...: 001) wins
    assert O.pick_index(5, _words(w1=0xE0000000, w2=0x20000000), 2) == 1
    # displacement: 7 >= 5, then w1's low half 0x4000 -> top three bits 010 = 2
    assert O.pick_index(5, _words(w1=0xE0004000), 0) == 2
    # every try fails: floor(2^31 * 5 / 2^32) = 2 from w4; floor(3 * 2^30 * 5 / 2^32) = 3 from w5
    assert O.pick_index(5, _words(w1=full, w2=full, w3=full, w4=0x80000000, w5=0), 2) == 2
    assert O.pick_index(5, _words(w1=full, w4=0, w5=0xC0000000), 0) == 3
    # n a power of two: the first try always wins
    assert O.pick_index(8, _words(w1=full), 2) == 7
    assert O.pick_index(8, _words(w1=full), 0) == 7
    # n = 70,000, k = 17 > 16: one try (0x8000 >> 15 = 1), else w5 (2^30 * 70000 / 2^32 = 17500)
    assert O.pick_index(70_000, _words(w1=0x8000), 0) == 1
    assert O.pick_index(70_000, _words(w1=full, w5=0x40000000), 0) == 17_500
    assert O.pick_index(70_000, _words(w1=full, w2=0x8000, w3=full, w4=full), 2) == 1


@pytest.mark.parametrize("n,bins", [(3, 3), (5, 5), (100, 10), (1000, 20), (70_000, 20)])
@pytest.mark.parametrize("move_type", [0, 2])
def test_pick_index_is_uniform(n, bins, move_type):
    """Over random words every index is equally likely: a chi-square test on
    `bins` equal groups of indices (p = 1e-4).  Taking the tries modulo n, or
    a fallback word that is not independent of the failed tries, piles the
    picks onto some indices and fails it."""
    rng = np.random.default_rng(n * 7 + move_type)
    draws = 40_000
    words = rng.integers(0, 1 << 32, size=(draws, 8), dtype=np.uint64).astype(np.uint32)
    idx = np.array([O.pick_index(n, w, move_type) for w in words])
    assert idx.min() >= 0 and idx.max() < n
    group = idx * bins // n
    h = np.bincount(group, minlength=bins)
    sizes = np.bincount(np.arange(n) * bins // n, minlength=bins)
    expect = draws * sizes / n
    chi2 = ((h - expect) ** 2 / expect).sum()
    limit = {2: 18.4, 4: 23.5, 9: 33.7, 19: 47.2}[bins - 1]
    assert chi2 < limit, (n, move_type, h)


@pytest.mark.parametrize("move_type,limit", [(2, 0.04), (0, 0.08)])
def test_pick_index_barely_depends_on_the_count(move_type, limit):
    """The reason for the rule: 700 and 701 candidates pick the same index
    unless a try lands on 700 or every try fails (then the fallback's
    floor(f n / 2^32) moves in about half the cases): about 2 % of deletions
    and 5 % of displacements, where floor(w1 n / 2^32) would differ for about
    half of them."""
    rng = np.random.default_rng(700 + move_type)
    words = rng.integers(0, 1 << 32, size=(20_000, 8), dtype=np.uint64).astype(np.uint32)
    diff = np.mean([O.pick_index(700, w, move_type) != O.pick_index(701, w, move_type) for w in words])
    assert diff < limit, diff


def test_chain_picks_by_the_rule():
    """Every displacement and deletion of an ideal-gas chain takes the index
    the rule gives for its move's words and the count before the move."""
    L = 9.0
    s = O.System(L, 2.5, [[0.0]], [[1.0]])
    n0 = 37
    s.build(W.uniform_positions(n0, L, 8), np.zeros(n0, np.int32))
    s.set_energy(0.0)
    seed, n_moves = 29, 6000
    tr, _ = s.run_moves(seed, 0, n_moves, 0.4, 0.3, 0.3, 0.3, 1.0, [math.log(4.0)])
    n_after = _n_trajectory(tr, n0)
    n_before = np.concatenate([[n0], n_after[:-1]])
    checked = 0
    for m in range(n_moves):
        t = int(tr["type"][m])
        if t == 1 or n_before[m] == 0:
            continue
        w = O.move_words(seed, m, 0)
        assert int(tr["index"][m]) == O.pick_index(int(n_before[m]), w, t), m
        checked += 1
    assert checked > 3000
