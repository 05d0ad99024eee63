"""GPU: batched chains and the chain kernel's team shapes.

Every team shape and the batched launch must take exactly the decisions of
the sequential chain; each batched chain k is compared with the oracle
running chain index k (its Philox counter word) on its own."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_1408_3764_gb300 import workloads as W  # noqa: E402
from paper_1408_3764_gb300.gcmc import Batch, Box, Mix  # noqa: E402


def _relaxed(n, L, seed, dmin=0.8):
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


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_team_shapes_take_identical_moves(precision):
    L = W.box_edge(1500, 0.55)
    pos = _relaxed(1500, L, 3)
    mix = Mix(1 / 3, 1 / 3, 1 / 3, 0.3, 1 / 1.2, [-2.7])
    traces = []
    for cfg in range(4):
        b = Box(L, 2.5, [[1.0]], [[1.0]], precision=precision)
        b.set_chain_config(cfg)
        b.build_cells(torch.as_tensor(pos), torch.zeros(1500, dtype=torch.int32))
        _, tr = b.run_moves(21, 0, 8000, mix, trace=True)
        traces.append((tr, b.get_state()))
    tol = 1e-5 if precision == "fp32" else 1e-12
    t0 = traces[0][0]
    for tr, st in traces[1:]:
        # decisions and configurations are identical; the energies differ only
        # in the summation order of the pair terms
        for k in ("type", "species", "index", "accepted"):
            assert np.array_equal(tr[k], t0[k]), k
        ok = np.isfinite(t0["lnA"])
        assert np.all(np.abs(tr["dU"] - t0["dU"])[ok] <= tol * t0["uabs"][ok] + 1e-300)
        for x, y in zip(st[:4], traces[0][1][:4]):
            assert np.array_equal(np.asarray(x), np.asarray(y))


def test_autotuned_shape_takes_identical_moves():
    L = W.box_edge(1200, 0.5)
    pos = _relaxed(1200, L, 4)
    mix = Mix(1 / 3, 1 / 3, 1 / 3, 0.3, 1 / 1.2, [-2.7])
    ref = Box(L, 2.5, [[1.0]], [[1.0]])
    ref.set_chain_config(0)
    ref.build_cells(torch.as_tensor(pos), torch.zeros(1200, dtype=torch.int32))
    _, tr0 = ref.run_moves(5, 0, 60_000, mix, trace=True)
    auto = Box(L, 2.5, [[1.0]], [[1.0]])
    auto.set_chain_config(-1)
    auto.build_cells(torch.as_tensor(pos), torch.zeros(1200, dtype=torch.int32))
    _, tr1 = auto.run_moves(5, 0, 60_000, mix, trace=True)
    assert auto.chain_config() in (0, 1, 2, 3)
    for k in ("type", "species", "index", "accepted"):
        assert np.array_equal(tr0[k], tr1[k]), k
    ok = np.isfinite(tr0["lnA"])
    assert np.all(np.abs(tr0["dU"] - tr1["dU"])[ok] <= 1e-5 * tr0["uabs"][ok] + 1e-300)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_matches_oracle_per_chain(precision):
    """Six uneven chains (N 60-1500, rho 0.1-0.6) in one batched launch; chain
    k equals the oracle's chain k move for move (final state and counts)."""
    chains = []
    for k, (n, rho) in enumerate([(60, 0.1), (300, 0.2), (900, 0.6), (1500, 0.45), (200, 0.35), (700, 0.5)]):
        L = max(W.box_edge(n, rho), 5.01)
        pos = W.uniform_positions(n, L, 100 + k) if rho < 0.3 else _relaxed(n, L, 100 + k)
        chains.append((L, pos, float(np.log(rho) - 1.0)))
    boxes, oracles, mixes, seeds = [], [], [], []
    for k, (L, pos, lz) in enumerate(chains):
        n = len(pos)
        b = Box(L, 2.5, [[1.0]], [[1.0]], precision=precision)
        b.build_cells(torch.as_tensor(pos), torch.zeros(n, dtype=torch.int32))
        boxes.append(b)
        o = O.System(L, 2.5, [[1.0]], [[1.0]])
        o.build(pos, np.zeros(n, np.int32))
        o.set_energy(o.total_energy())
        oracles.append(o)
        mixes.append(Mix(0.4, 0.3, 0.3, 0.3, 1 / 1.2, [lz]))
        seeds.append(1000 + 17 * k)
    batch = Batch(boxes)
    stats = batch.run_moves(seeds, 0, 20_000, mixes)
    stats2 = batch.run_moves(seeds, 20_000, 5_000, mixes)  # a second round (graph replay)
    assert batch.launches() >= 2
    for k, o in enumerate(oracles):
        m = mixes[k]
        tol = 1e-12 if precision == "fp64" else 1e-5
        to, so = o.run_moves(seeds[k], 0, 25_000, m.p_disp, m.p_ins, m.p_del, m.max_disp, m.beta, m.log_z,
                             tol=tol, chain=k, trace=True)
        assert [a + b for a, b in zip(stats[k]["accepted"], stats2[k]["accepted"])] == list(so.accepted)
        st_o, st_g = o.state(), boxes[k].get_state()
        for x, y in zip(st_o, st_g[:4]):
            assert np.array_equal(x, y)
        # the running energy adds the accepted dU, each within tol * uabs
        drift = tol * to["uabs"][to["accepted"] == 1].sum() + 1e-9
        assert abs(stats2[k]["energy"] - so.energy) <= drift


def test_batch_rejects_mixed_precision():
    a = Box(10.0, 2.5, [[1.0]], [[1.0]], precision="fp32")
    b = Box(10.0, 2.5, [[1.0]], [[1.0]], precision="fp64")
    with pytest.raises(RuntimeError):
        Batch([a, b])


def test_batch_rejects_bad_mix():
    """Every chain's mix is checked: a non-finite ln z or beta is refused before
    any launch, and the chains keep their state."""
    a = Box(10.0, 2.5, [[1.0]], [[1.0]])
    b = Box(10.0, 2.5, [[1.0]], [[1.0]])
    pos = W.uniform_positions(100, 10.0, 3)
    for x in (a, b):
        x.build_cells(torch.as_tensor(pos), torch.zeros(100, dtype=torch.int32))
    batch = Batch([a, b])
    good = Mix(0.4, 0.3, 0.3, 0.3, 1 / 1.2, [-2.7])
    for bad in (Mix(0.4, 0.3, 0.3, 0.3, 1 / 1.2, [float("nan")]), Mix(0.4, 0.3, 0.3, 0.3, float("inf"), [-2.7])):
        with pytest.raises(RuntimeError):
            batch.run_moves([1, 2], 0, 100, [good, bad])
    assert a.counts()[0] == 100 and b.counts()[0] == 100


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batched_prepare_and_gradient_match_per_box_calls(precision):
    """gcmc_batch_prepare and gcmc_batch_energy_grad give what the per-box
    calls give (same kernels, fewer host synchronisations); the exported
    configuration rebuilds the same state."""
    chains = W.isotherm_chains(n_chains=6, n_max=3000)
    boxes, ref = [], []
    for w in chains:
        b = Box(w.L, w.rc, w.eps, w.sigma, precision=precision)
        boxes.append(b)
        r = Box(w.L, w.rc, w.eps, w.sigma, precision=precision)
        r.build_cells(torch.as_tensor(w.positions()), torch.as_tensor(w.types()))
        ref.append(r)
    batch = Batch(boxes)
    pos = [torch.as_tensor(w.positions()).cuda() for w in chains]
    typ = [torch.as_tensor(w.types()).cuda() for w in chains]
    e = batch.prepare(pos, typ)
    for k, r in enumerate(ref):
        assert e[k] == r.total_energy()
        for x, y in zip(boxes[k].get_state(), r.get_state()):
            assert np.array_equal(np.asarray(x), np.asarray(y))
    # moves, then the batched gradient against the per-box one
    mixes = [Mix(w.p_disp, w.p_ins, w.p_del, w.max_disp, w.beta, w.log_z) for w in chains]
    batch.run_moves([w.seed for w in chains], 0, 3000, mixes)
    dpos = [torch.empty((int(b.counts().sum()), 3), dtype=torch.float32, device="cuda") for b in boxes]
    eg, wg = batch.energy_grad(dpos)
    for k, b in enumerate(boxes):
        g = b.energy_grad()
        assert eg[k] == g["energy"] and wg[k] == g["virial"]
        assert torch.equal(dpos[k], g["dpos"])
    # the batched export writes what the per-box export writes (buffers may
    # be longer than N; a shorter one is refused before anything is written)
    n = [int(b.counts().sum()) for b in boxes]
    bp = [torch.empty((n[k] + 5, 3), dtype=torch.float64, device="cuda") for k in range(len(boxes))]
    bt = [torch.empty(n[k] + 5, dtype=torch.int32, device="cuda") for k in range(len(boxes))]
    assert list(batch.export_positions(bp, bt)) == n
    for k, b in enumerate(boxes):
        p, s = b.export_positions()
        assert torch.equal(bp[k][: n[k]], p) and torch.equal(bt[k][: n[k]], s)
    with pytest.raises(ValueError):
        batch.export_positions([x[:1] for x in bp], bt)
    # export and rebuild: the same configuration, particle for particle (the
    # order within a cell follows the ids after a build, the move history
    # before it)
    for b in boxes:
        st0 = b.get_state()
        p, s = b.export_positions()
        b.build_cells(p, s)
        st1 = b.get_state()
        for x, y in zip(st0[:3], st1[:3]):
            assert np.array_equal(np.asarray(x), np.asarray(y))
        bounds = np.concatenate([[0], np.cumsum(st0[2])])
        for c in range(len(st0[2])):
            a0 = np.sort(st0[3][bounds[c]:bounds[c + 1]])
            a1 = np.sort(st1[3][bounds[c]:bounds[c + 1]])
            assert np.array_equal(a0, a1)


def test_cycle_counters_only_when_asked_and_same_moves():
    """The per-role cycle counters are compiled in only for a profiled run;
    the profiled kernel takes the same moves and decisions."""
    L = W.box_edge(900, 0.45)
    pos = _relaxed(900, L, 7)
    mix = Mix(1 / 3, 1 / 3, 1 / 3, 0.3, 1 / 1.2, [-2.7])
    traces, profs = [], []
    for on in (False, True):
        b = Box(L, 2.5, [[1.0]], [[1.0]], precision="fp32")
        b.set_chain_config(0)
        b.set_chain_profile(on)
        b.build_cells(torch.as_tensor(pos), torch.zeros(900, dtype=torch.int32))
        _, tr = b.run_moves(13, 0, 6000, mix, trace=True)
        traces.append(tr)
        profs.append(b.chain_profile())
    off, on = profs
    assert all(off[k] == 0 for k in off if k != "evaluations")
    assert off["evaluations"] >= 6000
    assert on["commit_total"] > 0 and on["team_eval"] > 0
    assert on["commit_total"] >= on["commit_wait"] + on["commit_valid"] + on["commit_decide"]
    for k in ("type", "species", "index", "accepted"):
        assert np.array_equal(traces[0][k], traces[1][k]), k
    from paper_1408_3764_gb300 import _lib
    assert _lib.load().gcmc_set_chain_profile(b.handle, 2) == 1  # INVALID_ARG
