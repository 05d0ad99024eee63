"""GPU: the microcell list (Sec. 3.3) and the chain evaluated over it,
against the oracle's microcell lists and chain.

* Build: per-cell counts, the order of every list (species by species, index
  by index) and each slot's record (grid position and tag) bit-exact.
* Chain: the same decisions as the oracle move by move, dU within tol * uabs
  (tol = 1e-12 FP64, 1e-5 FP32; uabs = sum of |rep| + |att| over the
  evaluated pairs), and afterwards the 27-cell state and the microcell lists
  bit-exact (appends and swap-with-last removals, Sec. 3.3.3).  Cases: the
  plain 2,048-particle fluid, a two-species mixture, the largest cutoff of the
  sweep (an 11^3 cube), a box narrower than the cube (every cell once), an
  empty start, growth of the microcell capacity, and runs that alternate with
  the 27-cell chain.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_1408_3764_gb300 import workloads as W  # noqa: E402
from paper_1408_3764_gb300.gcmc import Box, Mix  # noqa: E402

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def _pair(L, rc, eps, sigma, pos, types, precision="fp64", **kw):
    o = O.System(L, rc, eps, sigma)
    o.build(pos, types)
    o.set_energy(o.total_energy())
    b = Box(L, rc, eps, sigma, precision=precision, **kw)
    b.build_cells(torch.as_tensor(pos), torch.as_tensor(types))
    return o, b


def _same_microcells(o, b):
    M_o, cnt_o, refs_o, _ = o.micro_state()
    M, cap, cnt, slots = b.microcells()
    assert M == M_o
    assert np.array_equal(cnt.astype(np.int64), cnt_o)
    assert cap >= cnt.max(initial=0)
    # lists in order: the tags of slots 0 .. count-1 of every cell
    k = np.arange(cap)[:, None] < cnt[None, :].astype(np.int64)
    tags = slots[:, :, 3].T[k.T]  # cell-major walk over the filled slots
    assert np.array_equal(tags, refs_o)
    # every record holds its particle's current grid position
    n_g, X_g, _, _, _ = b.get_state()
    first = np.concatenate([[0], np.cumsum(n_g)])
    rows = first[tags & 0xFF] + (tags >> 8)
    xyz = slots[:, :, :3].transpose(1, 0, 2)[k.T]
    assert np.array_equal(xyz, X_g[rows])


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


def _chain(o, b, seed, first, n, args, precision, micro=True):
    to, so = o.run_moves(seed, first, n, *args, tol=TOL[precision])
    run = b.run_moves_micro if micro else b.run_moves
    sg, tg = run(seed, first, n, Mix(*args), trace=True)
    for k in ("type", "species", "index", "accepted"):
        assert np.array_equal(tg[k], to[k]), k
    ok = np.isfinite(to["lnA"])
    err = np.abs(tg["dU"] - to["dU"])[ok]
    assert np.all(err <= TOL[precision] * to["uabs"][ok] + 1e-300)
    assert sg["accepted"] == list(so.accepted) and sg["attempted"] == list(so.attempted)
    for x, y in zip(o.state(), b.get_state()[:4]):
        assert np.array_equal(x, y)
    return sg, so


@pytest.mark.parametrize("case", ["c1", "mixture", "sweep_rc4.25"])
def test_micro_build_matches_oracle(case):
    if case == "c1":
        w = W.c1_plain_fp64()
        pos, types, L, rc, eps, sigma = w.positions(), w.types(), w.L, w.rc, w.eps, w.sigma
    elif case == "mixture":
        L = W.box_edge(1500, 0.55)
        pos, types = _relaxed(1500, L, 4, 0.8), (np.arange(1500) % 4 == 0).astype(np.int32)
        eps, sigma = W.lorentz_berthelot([1.0, 0.8], [1.0, 1.2])
        rc = 2.5
    else:
        w = W.cutoff_sweep(4.25)
        pos, types, L, rc, eps, sigma = w.positions(), w.types(), w.L, w.rc, w.eps, w.sigma
    o, b = _pair(L, rc, eps, sigma, pos, types)
    o.micro_build(1.0)
    b.build_microcells(1.0, 15)
    _same_microcells(o, b)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["c1", "mixture", "sweep_rc4.25", "narrow_box"])
def test_micro_chain_parity(precision, case):
    if case == "c1":
        w = W.c1_plain_fp64()
        o, b = _pair(w.L, w.rc, w.eps, w.sigma, w.positions(), w.types(), precision)
        args, seed, n = (w.p_disp, w.p_ins, w.p_del, w.max_disp, w.beta, w.log_z), w.seed, 10_000
    elif case == "mixture":
        L = W.box_edge(1500, 0.55)
        eps, sigma = W.lorentz_berthelot([1.0, 0.8], [1.0, 1.2])
        o, b = _pair(L, 2.5, eps, sigma, _relaxed(1500, L, 4, 0.8), (np.arange(1500) % 4 == 0).astype(np.int32),
                     precision)
        args, seed, n = (0.4, 0.3, 0.3, 0.35, 1 / 1.3, [-2.2, -3.0]), 77, 20_000
    elif case == "sweep_rc4.25":
        w = W.cutoff_sweep(4.25)
        o, b = _pair(w.L, w.rc, w.eps, w.sigma, w.positions(), w.types(), precision)
        args, seed, n = (w.p_disp, w.p_ins, w.p_del, w.max_disp, w.beta, w.log_z), w.seed, 10_000
    else:
        # L = 5.6: M = 6 microcells per side but the cube needs 2D+1 = 7, so
        # every cell of an axis is visited once
        L = 5.6
        o, b = _pair(L, 2.5, [[1.0]], [[1.0]], _relaxed(80, L, 9), np.zeros(80, np.int32), precision)
        args, seed, n = (0.4, 0.3, 0.3, 0.5, 1 / 1.2, [-2.0]), 5, 20_000
    o.micro_build(1.0)
    b.build_microcells(1.0)
    sg, _ = _chain(o, b, seed, 0, n, args, precision)
    assert sg["accepted"][0] > 0
    _same_microcells(o, b)


def test_micro_empty_start_and_capacity_growth():
    """An ideal gas filled from empty at high activity: <N> = zV ~ 1.7 per unit
    cube, so microcells soon need more than 5 slots and the library grows them."""
    L = 9.0
    o, b = _pair(L, 2.5, [[0.0]], [[1.0]], np.zeros((0, 3)), np.zeros(0, np.int32))
    o.micro_build(1.0)
    b.build_microcells(1.0)
    assert b.microcells()[1] == 5
    args = (0.2, 0.5, 0.3, 0.5, 1.0, [float(np.log(1.7))])
    _chain(o, b, 3, 0, 30_000, args, "fp64")
    assert b.microcells()[1] > 5
    _same_microcells(o, b)


def test_micro_fixed_capacity_overflow_is_reported():
    L = 6.0
    rng = np.random.default_rng(2)
    pos = rng.random((400, 3)) * L  # ~1.85 per unit cell: some cells hold more than 5
    b = Box(L, 2.5, [[0.0]], [[1.0]])
    b.build_cells(torch.as_tensor(pos), torch.zeros(400, dtype=torch.int32))
    with pytest.raises(RuntimeError):
        b.build_microcells(1.0, 3)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_micro_and_cell_chains_alternate(precision):
    """Microcell chain, 27-cell chain, microcell chain again (the microcells
    are rebuilt from the particles): one continuous chain, equal to the
    oracle's, with the oracle's microcells rebuilt at the same point."""
    L = W.box_edge(1200, 0.5)
    o, b = _pair(L, 2.5, [[1.0]], [[1.0]], _relaxed(1200, L, 21, 0.8), np.zeros(1200, np.int32), precision)
    args = (1 / 3, 1 / 3, 1 / 3, 0.3, 1 / 1.2, [-2.786])
    o.micro_build(1.0)
    b.build_microcells(1.0)
    _chain(o, b, 9, 0, 8000, args, precision, micro=True)
    _chain(o, b, 9, 8000, 8000, args, precision, micro=False)
    o.micro_build(1.0)  # the GPU rebuilds its stale microcells the same way
    _chain(o, b, 9, 16000, 8000, args, precision, micro=True)
    _same_microcells(o, b)
    # the full-system energy in the context's precision (FP32 pair terms: ~1e-8 relative)
    rel = 1e-9 if precision == "fp64" else 1e-6
    assert b.total_energy() == pytest.approx(o.total_energy(), rel=rel, abs=1e-9)


def test_micro_chain_refuses_the_virial_flag():
    L = 8.0
    b = Box(L, 2.5, [[1.0]], [[1.0]])
    b.build_cells(torch.as_tensor(_relaxed(100, L, 4)), torch.zeros(100, dtype=torch.int32))
    b.build_microcells(1.0)
    with pytest.raises(RuntimeError):
        b.run_moves_micro(1, 0, 100, Mix(0.4, 0.3, 0.3, 0.3, 1.0, [-2.0], virial=True))
