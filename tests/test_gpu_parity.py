"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.

Tolerances:
  * cell assignment, ordering, positions, particle counts, chain decisions:
    bit-exact (integer work);
  * energies: |gpu - oracle| <= tol * uabs, where uabs is the sum over the
    pair terms of |4 eps s^12| + |4 eps s^6| -- the scale of the rounding
    error of any evaluation -- with tol = 1e-12 (FP64 mode) or 1e-5 (FP32
    pair terms; the measured FP32 maximum is about 1e-6).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_1408_3764_gb300 import workloads as W  # noqa: E402
from paper_1408_3764_gb300.gcmc import Box, Mix, species_major_order  # noqa: E402

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def _pair(L, rc, eps, sigma, pos, types, precision="fp64", **kw):
    o = O.System(L, rc, eps, sigma)
    cl = o.build(pos, types)
    b = Box(L, rc, eps, sigma, precision=precision, **kw)
    b.build_cells(torch.as_tensor(pos), torch.as_tensor(types))
    return o, cl, b


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


# ----------------------------------------------------------------- cells ---

@pytest.mark.parametrize("n,L,rc,S", [(0, 8.0, 2.5, 1), (1, 8.0, 2.5, 1), (37, 6.0, 2.5, 2),
                                      (1000, 12.0, 2.5, 1), (2048, 16.0, 2.5, 1),
                                      (5000, 20.0, 3.0, 3), (20011, 31.0, 2.5, 2)])
def test_build_cells_bit_exact(n, L, rc, S):
    pos, types, eps, sigma = W.tiny_system(n=max(n, 1), L=L, rc=rc, n_species=S, seed=n + 1)
    pos, types = pos[:n], types[:n]
    o, cl, b = _pair(L, rc, eps, sigma, pos, types)
    cs, cc, order = b.cell_list()
    assert np.array_equal(cc.cpu().numpy(), cl.cell_count)
    assert np.array_equal(cs.cpu().numpy(), cl.cell_start)
    assert np.array_equal(order.cpu().numpy(), cl.order)
    n_o, X_o, cc_o, refs_o = o.state()
    n_g, X_g, cc_g, refs_g, _ = b.get_state()
    assert np.array_equal(n_g, n_o)
    assert np.array_equal(X_g, X_o)
    assert np.array_equal(cc_g, cc_o)
    assert np.array_equal(refs_g, refs_o)


@pytest.mark.parametrize("wl", [W.c1_plain_fp64, W.c2_fp32_vs_fp64, W.c3_mixture_1m, W.c5_gradient])
def test_build_cells_bit_exact_full_size(wl):
    w = wl()
    o, cl, b = _pair(w.L, w.rc, w.eps, w.sigma, w.positions(), w.types())
    cs, cc, order = b.cell_list()
    assert np.array_equal(cc.cpu().numpy(), cl.cell_count)
    assert np.array_equal(cs.cpu().numpy(), cl.cell_start)
    assert np.array_equal(order.cpu().numpy(), cl.order)


def test_build_rejects_bad_input():
    b = Box(10.0, 2.5, [[1.0]], [[1.0]])
    with pytest.raises(RuntimeError):
        b.build_cells(torch.tensor([[1.0, float("nan"), 2.0]]), torch.tensor([0]))
    with pytest.raises(RuntimeError):
        b.build_cells(torch.tensor([[1.0, 1.0, 2.0]]), torch.tensor([3]))


def test_build_quantisation_edges_match_the_oracle():
    """Grid quantisation at its edges: negative coordinates and coordinates
    beyond the box wrap as the oracle's floor(x 2^32 / L) mod 2^32 does, and
    both reject the same values (non-finite, |x 2^32 / L| > 4e18)."""
    L = 10.0
    q = 2.0 ** 32 / L
    lim = 4.0e18 / q
    xs = [0.0, -0.0, 1e-300, -1e-300, L, -L, 2.5 * L, -7.25 * L, np.nextafter(L, 0.0),
          np.nextafter(0.0, -1.0), 123456.789, -98765.4321, lim, -lim, np.nextafter(lim, 0.0),
          np.nextafter(lim, np.inf), np.nextafter(-lim, -np.inf), float("inf"), float("-inf"), float("nan")]
    b = Box(L, 2.5, [[1.0]], [[1.0]])
    for x in xs:
        try:
            want = O.quantize(x, L)
        except ValueError:
            want = None
        p = torch.tensor([[x, 1.0, 2.0]], dtype=torch.float64)
        if want is None:
            with pytest.raises(RuntimeError):
                b.build_cells(p, torch.tensor([0], dtype=torch.int32))
        else:
            b.build_cells(p, torch.tensor([0], dtype=torch.int32))
            got = b.get_state()[1]
            assert int(got[0, 0]) == want, x
            assert int(got[0, 1]) == O.quantize(1.0, L) and int(got[0, 2]) == O.quantize(2.0, L)


# -------------------------------------------------------- trial energies ---

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,L,rc,S", [(50, 6.0, 2.5, 1), (700, 11.0, 2.5, 2), (4000, 19.0, 3.0, 2),
                                      (2048, 16.0, 2.5, 1)])
def test_trial_energy_parity(precision, n, L, rc, S):
    pos, types, eps, sigma = W.tiny_system(n=n, L=L, rc=rc, n_species=S, seed=3 * n)
    o, _, b = _pair(L, rc, eps, sigma, pos, types, precision)
    tp, ts = W.insertion_points(777, L, S, n)
    ref, uabs = o.trial_energy(tp, ts, with_abs=True)
    got, gabs = b.trial_energy(tp, ts, with_abs=True)
    got, gabs = got.cpu().numpy(), gabs.cpu().numpy()
    assert np.all(np.abs(got - ref) <= TOL[precision] * uabs + 1e-300)
    assert np.allclose(gabs, uabs, rtol=1e-5)
    # existing particles, excluding themselves (deletion energies)
    cnt = o.counts()
    rows = np.arange(0, n, max(1, n // 300))
    sm = species_major_order(types)
    excl = []
    for r in rows:
        p = sm[r]
        s = int(types[p])
        i = r - int(cnt[:s].sum())
        excl.append((s << 32) | i)
    ref, uabs = o.trial_energy(pos[sm[rows]], types[sm[rows]], exclude=excl, with_abs=True)
    got = b.trial_energy(pos[sm[rows]], types[sm[rows]], exclude=excl).cpu().numpy()
    assert np.all(np.abs(got - ref) <= TOL[precision] * uabs + 1e-300)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_trial_energy_full_size_sampled(precision):
    """The million-particle mixture: 2,000 of a batch of 200,000 trial points
    are checked one by one against the oracle."""
    w = W.c3_mixture_1m()
    o, _, b = _pair(w.L, w.rc, w.eps, w.sigma, w.positions(), w.types(), precision)
    tp, ts = W.insertion_points(200_000, w.L, 2, 17)
    got = b.trial_energy(tp, ts).cpu().numpy()
    pick = np.arange(0, 200_000, 100)
    ref, uabs = o.trial_energy(tp[pick], ts[pick], with_abs=True)
    assert np.all(np.abs(got[pick] - ref) <= TOL[precision] * uabs + 1e-300)


def test_trial_energy_empty_and_bad():
    b = Box(10.0, 2.5, [[1.0]], [[1.0]])
    b.build_cells(torch.zeros((0, 3), dtype=torch.float64), torch.zeros(0, dtype=torch.int32))
    out = b.trial_energy(np.array([[1.0, 2.0, 3.0]]), np.array([0]))
    assert out.item() == 0.0
    assert b.trial_energy(np.zeros((0, 3)), np.zeros(0)).numel() == 0
    with pytest.raises(RuntimeError):
        b.trial_energy(np.array([[1.0, 2.0, 3.0]]), np.array([1]))


# ----------------------------------------------------------- total energy --

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,L,rc,S", [(300, 8.0, 2.5, 2), (2048, 16.0, 2.5, 1), (9000, 25.0, 3.0, 2)])
def test_total_energy_parity(precision, n, L, rc, S):
    pos = _relaxed(n, L, n) if n <= 2048 else W.uniform_positions(n, L, 5)
    types = (np.arange(n) % S).astype(np.int32)
    eps, sigma = W.lorentz_berthelot(np.linspace(1.0, 0.8, S), np.linspace(1.0, 1.2, S))
    o, _, b = _pair(L, rc, eps, sigma, pos, types, precision)
    ref = o.total_energy()
    scale = 0.5 * o.trial_energy(*_all_particles(o, pos, types), with_abs=True)[1].sum()
    got = b.total_energy()
    assert abs(got - ref) <= TOL[precision] * scale


def _all_particles(o, pos, types):
    sm = species_major_order(types)
    cnt = o.counts()
    ex = []
    for r, p in enumerate(sm):
        s = int(types[p])
        ex.append((s << 32) | (r - int(cnt[:s].sum())))
    return pos[sm], types[sm], ex


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_total_energy_full_size(precision):
    w = W.c2_fp32_vs_fp64()
    o, _, b = _pair(w.L, w.rc, w.eps, w.sigma, w.positions(), w.types(), precision)
    ref = o.total_energy()
    got = b.total_energy()
    # uniform random start: dominated by near-overlaps; relative check
    assert got == pytest.approx(ref, rel=TOL[precision])


# ---------------------------------------------------------------- gradient --

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_gradient_parity(precision):
    L, rc, n = 12.0, 3.0, 900
    pos = _relaxed(n, L, 9)
    types = (np.arange(n) % 5 == 0).astype(np.int32)
    eps, sigma = W.lorentz_berthelot([1.0, 0.8], [1.0, 1.2])
    o, _, b = _pair(L, rc, eps, sigma, pos, types, precision)
    ref = o.energy_grad()
    got = b.energy_grad()
    tol = TOL[precision]
    fscale = np.abs(ref["dpos"]).max()
    assert np.allclose(got["dpos"].cpu().numpy(), ref["dpos"], rtol=max(tol, 2e-7) * 10,
                       atol=max(tol, 1e-7) * 10 * fscale)
    for k in ("deps", "dsigma"):
        assert np.allclose(got[k], ref[k], rtol=tol * 10, atol=tol * 10 * np.abs(ref[k]).max())
    assert got["energy"] == pytest.approx(ref["energy"], rel=tol * 10)
    assert got["virial"] == pytest.approx(ref["virial"], rel=tol * 10)


# ------------------------------------------------------------------ chain --

def _compare_traces(tg, to, tol, allow_divergence=True):
    """Identical decisions move by move; energies within tol * uabs.  A
    divergence is only allowed at a trial both sides flag as near the
    threshold; the comparison stops there."""
    n = len(to)
    for k in ("type", "species", "index"):
        same = tg[k] == to[k]
        if not same.all():
            first = int(np.argmin(same))
            return _diverged(tg, to, first, allow_divergence)
    dec = tg["accepted"] == to["accepted"]
    if not dec.all():
        return _diverged(tg, to, int(np.argmin(dec)), allow_divergence)
    possible = np.isfinite(to["lnA"])
    err = np.abs(tg["dU"] - to["dU"])[possible]
    assert np.all(err <= tol * to["uabs"][possible] + 1e-300), np.max(err / (to["uabs"][possible] + 1e-300))
    return n


def _diverged(tg, to, k, allow):
    assert allow, "decisions differ at move %d" % k
    assert (tg["flagged"][k] & 1) and (to["flagged"][k] & 1), "unflagged divergence at move %d" % k
    return k


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_chain_parity_c1(precision):
    """The plain workload: 2,048 particles, rho 0.5, 10^4 moves, seed 1 -- every
    decision and the final configuration equal the oracle's."""
    w = W.c1_plain_fp64()
    o, _, b = _pair(w.L, w.rc, w.eps, w.sigma, w.positions(), w.types(), precision)
    o.set_energy(o.total_energy())
    mix = Mix(w.p_disp, w.p_ins, w.p_del, w.max_disp, w.beta, w.log_z)
    to, so = o.run_moves(w.seed, 0, w.moves, w.p_disp, w.p_ins, w.p_del, w.max_disp, w.beta, w.log_z,
                         tol=TOL[precision])
    sg, tg = b.run_moves(w.seed, 0, w.moves, mix, trace=True)
    k = _compare_traces(tg, to, TOL[precision])
    assert k == len(to)
    assert sg["accepted"] == list(so.accepted) and sg["attempted"] == list(so.attempted)
    n_o, X_o, cc_o, refs_o = o.state()
    n_g, X_g, cc_g, refs_g, _ = b.get_state()
    assert np.array_equal(n_g, n_o) and np.array_equal(X_g, X_o)
    assert np.array_equal(cc_g, cc_o) and np.array_equal(refs_g, refs_o)
    assert sg["accepted"][1] > 0 and sg["accepted"][2] > 0


def _relaxed_workload(n, rho, seed):
    L = W.box_edge(n, rho)
    return L, _relaxed(n, L, seed, dmin=0.8)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_chain_parity_mixture(precision):
    L, pos = _relaxed_workload(1500, 0.55, 4)
    types = (np.arange(1500) % 4 == 0).astype(np.int32)
    eps, sigma = W.lorentz_berthelot([1.0, 0.8], [1.0, 1.2])
    o, _, b = _pair(L, 2.5, eps, sigma, pos, types, precision)
    o.set_energy(o.total_energy())
    args = (0.4, 0.3, 0.3, 0.35, 1 / 1.3, [-2.2, -3.0])
    to, so = o.run_moves(77, 1000, 20_000, *args, tol=TOL[precision])
    sg, tg = b.run_moves(77, 1000, 20_000, Mix(*args), trace=True)
    assert _compare_traces(tg, to, TOL[precision]) == len(to)
    st_o, st_g = o.state(), b.get_state()
    for x, y in zip(st_o, st_g[:4]):
        assert np.array_equal(x, y)


def test_chain_parity_small_box_and_overflow_growth():
    """T = 3 (every cell neighbours every other) with an ideal gas at high
    activity: <N> = zV ~ 1,370 forces the library to grow both the cell slot
    arrays and the per-species capacity mid-run; the chain must not notice."""
    L = 6.5
    pos = W.uniform_positions(40, L, 8)
    types = np.zeros(40, np.int32)
    o, _, b = _pair(L, 2.5, [[0.0]], [[1.0]], pos, types, "fp64")
    g0 = b.geometry()
    o.set_energy(o.total_energy())
    args = (0.2, 0.5, 0.3, 0.5, 1.0, [math.log(5.0)])
    to, so = o.run_moves(5, 0, 20_000, *args, tol=1e-12)
    sg, tg = b.run_moves(5, 0, 20_000, Mix(*args), trace=True)
    assert _compare_traces(tg, to, 1e-12) == len(to)
    g1 = b.geometry()
    assert g1["cell_capacity"] > g0["cell_capacity"]
    assert g1["max_particles"] > g0["max_particles"]
    assert sg["n"][0] > 1100
    st_o, st_g = o.state(), b.get_state()
    for x, y in zip(st_o, st_g[:4]):
        assert np.array_equal(x, y)


def test_explicit_capacity_overflow_is_reported():
    """With an explicit cell capacity the chain stops before the overflowing
    move and reports CELL_OVERFLOW with the number of moves completed."""
    L = 6.5
    b = Box(L, 2.5, [[0.0]], [[1.0]], cell_capacity=8)
    b.build_cells(torch.as_tensor(W.uniform_positions(40, L, 8)), torch.zeros(40, dtype=torch.int32))
    st = b.run_moves(5, 0, 20_000, Mix(0.2, 0.5, 0.3, 0.5, 1.0, [math.log(5.0)]), check_status=False)
    assert st["status"] == 2
    assert 0 < st["moves_done"] < 20_000
    cnt, _, cc, _, _ = b.get_state()
    assert cc.max() <= 8 and cc.sum() == cnt.sum()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("L,max_disp", [(13.0, 3.0), (10.4, 2.9), (16.0, 5.5)])
def test_chain_parity_far_displacements(precision, L, max_disp):
    """Displacements longer than a cell edge (T = 5, 4, 6): the old and new
    neighbourhoods are visited separately; decisions still match move by move."""
    n = int(0.45 * L ** 3)
    pos = _relaxed(n, L, 77, dmin=0.8)
    o, _, b = _pair(L, 2.5, [[1.0]], [[1.0]], pos, np.zeros(n, np.int32), precision)
    o.set_energy(o.total_energy())
    args = (0.6, 0.2, 0.2, max_disp, 1 / 1.2, [-2.7])
    to, _ = o.run_moves(13, 0, 20_000, *args, tol=TOL[precision])
    sg, tg = b.run_moves(13, 0, 20_000, Mix(*args), trace=True)
    assert _compare_traces(tg, to, TOL[precision]) == len(to)
    st_o, st_g = o.state(), b.get_state()
    for x, y in zip(st_o, st_g[:4]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_chain_parity_full_size_c2(precision):
    """131,072 particles, rho 0.6, rc 3: 10^5 moves of the full-size workload,
    decision by decision against the oracle."""
    w = W.c2_fp32_vs_fp64()
    o, _, b = _pair(w.L, w.rc, w.eps, w.sigma, w.positions(), w.types(), precision)
    o.set_energy(o.total_energy())
    mix = Mix(w.p_disp, w.p_ins, w.p_del, w.max_disp, w.beta, w.log_z)
    n = 100_000
    to, so = o.run_moves(w.seed, 0, n, w.p_disp, w.p_ins, w.p_del, w.max_disp, w.beta, w.log_z,
                         tol=TOL[precision])
    sg, tg = b.run_moves(w.seed, 0, n, mix, trace=True)
    assert _compare_traces(tg, to, TOL[precision]) == n
    assert sg["n"] == list(so.n[:1])


def _same_moves(t1, t2, tol):
    """The same moves and decisions; dU within tol * uabs (the speculative
    evaluation may split a trial's pair terms among warps differently from
    one run to the next, so the last bits of dU may differ)."""
    for k in ("type", "species", "index", "accepted"):
        assert np.array_equal(t1[k], t2[k]), k
    ok = np.isfinite(t1["lnA"])
    assert np.all(np.abs(t1["dU"] - t2["dU"])[ok] <= tol * t1["uabs"][ok] + 1e-300)


def test_chain_resume_is_exact():
    """Counter-based moves: [0, a) + [a, b) == [0, b); state export/import
    resumes: identical moves, decisions and configurations (dU and the
    running energy agree to rounding)."""
    L, pos = _relaxed_workload(800, 0.5, 12)
    types = np.zeros(800, np.int32)
    mix = Mix(1 / 3, 1 / 3, 1 / 3, 0.3, 0.8, [-2.6])
    a = Box(L, 2.5, [[1.0]], [[1.0]])
    a.set_chain_config(1)
    a.build_cells(torch.as_tensor(pos), torch.as_tensor(types))
    b = Box(L, 2.5, [[1.0]], [[1.0]])
    b.set_chain_config(1)
    b.build_cells(torch.as_tensor(pos), torch.as_tensor(types))
    _, ta = a.run_moves(3, 0, 6000, mix, trace=True)
    _, tb1 = b.run_moves(3, 0, 2500, mix, trace=True)
    snap = b.get_state()
    _, tb2 = b.run_moves(3, 2500, 3500, mix, trace=True)
    _same_moves(ta, np.concatenate([tb1, tb2]), TOL["fp64"])
    c = Box(L, 2.5, [[1.0]], [[1.0]])
    c.set_chain_config(1)
    c.restore(*snap)
    _, tc = c.run_moves(3, 2500, 3500, mix, trace=True)
    _same_moves(tc, tb2, TOL["fp64"])
    sa, sc = a.get_state(), c.get_state()
    for x, y in zip(sa[:4], sc[:4]):
        assert np.array_equal(np.asarray(x), np.asarray(y))
    drift = TOL["fp64"] * ta["uabs"][ta["accepted"] == 1].sum() + 1e-9
    assert abs(sa[4] - sc[4]) <= 2 * drift


def test_chain_energy_bookkeeping():
    """Running energy = initial energy + sum of accepted dU = recomputed total."""
    L, pos = _relaxed_workload(1200, 0.5, 21)
    b = Box(L, 2.5, [[1.0]], [[1.0]])
    b.build_cells(torch.as_tensor(pos), torch.zeros(1200, dtype=torch.int32))
    E0 = b.total_energy()
    st, tr = b.run_moves(9, 0, 30_000, Mix(1 / 3, 1 / 3, 1 / 3, 0.3, 1 / 1.2, [-2.786]), trace=True)
    assert E0 + tr["dU"][tr["accepted"] == 1].sum() == pytest.approx(st["energy"], rel=1e-12, abs=1e-9)
    assert b.total_energy() == pytest.approx(st["energy"], rel=1e-10, abs=1e-8)


def test_gradient_autograd_function():
    from paper_1408_3764_gb300 import gcmc as G
    from paper_1408_3764_gb300.gcmc import cell_list_energy
    L, n = 10.0, 400
    pos = torch.tensor(_relaxed(n, L, 31), dtype=torch.float32, device="cuda", requires_grad=True)
    types = torch.tensor((np.arange(n) % 3 == 0).astype(np.int32))
    eps, sigma = W.lorentz_berthelot([1.0, 0.8], [1.0, 1.2])
    e_t = torch.tensor(eps, requires_grad=True)
    s_t = torch.tensor(sigma, requires_grad=True)
    E = cell_list_energy(pos, e_t, s_t, types, L, 2.5, "fp32")
    E.backward()
    o = O.System(L, 2.5, eps, sigma)
    o.build(pos.detach().cpu().double().numpy(), types.numpy())
    ref = o.energy_grad()
    sm = species_major_order(types.numpy())
    want = np.empty_like(ref["dpos"])
    want[sm] = ref["dpos"]
    assert E.item() == pytest.approx(ref["energy"], rel=1e-5)
    fs = np.abs(want).max()
    assert np.allclose(pos.grad.cpu().numpy(), want, atol=1e-4 * fs, rtol=1e-4)
    assert np.allclose(e_t.grad.numpy(), ref["deps"], rtol=1e-4)
    assert np.allclose(s_t.grad.numpy(), ref["dsigma"], rtol=1e-4)
    # repeated calls reuse one context; a forward-only call runs no gradient
    creates = G._box_cache.creates
    for _ in range(3):
        pos.grad = None
        E2 = cell_list_energy(pos, e_t.detach(), s_t.detach(), types, L, 2.5, "fp32")
        E2.backward()
        assert E2.item() == E.item()
        assert np.allclose(pos.grad.cpu().numpy(), want, atol=1e-4 * fs, rtol=1e-4)
    assert G._box_cache.creates == creates
    with torch.no_grad():
        E3 = cell_list_energy(pos, e_t, s_t, types, L, 2.5, "fp32")
    assert E3.item() == E.item()
    # two forwards, then the first one's backward: its cells are rebuilt
    p2 = (pos.detach() * 0.999).requires_grad_(True)
    Ea = cell_list_energy(pos, e_t.detach(), s_t.detach(), types, L, 2.5, "fp32")
    Eb = cell_list_energy(p2, e_t.detach(), s_t.detach(), types, L, 2.5, "fp32")
    pos.grad = None
    Ea.backward()
    assert np.allclose(pos.grad.cpu().numpy(), want, atol=1e-4 * fs, rtol=1e-4)
    del Eb
