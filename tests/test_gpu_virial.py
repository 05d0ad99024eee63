"""GPU: the running virial W = sum_{i<j} r U'(r) kept by the chain kernel
(virial pressure P = rho k T - W / (3V), updated on each accepted move,
Sec. 3.1.2, and averaged on the GPU, Sec. 3.3.4), against the oracle's
running virial on the same seeded chain.

Each accepted trial adds its dW, the 27-cell sum of r U'(r) = -12 rep + 6 att
over the new and old positions.  A pair's |r U'(r)| is at most 12 (rep + att),
so the rounding error of one evaluation is below 12 * tol * uabs (uabs the
trial's sum of |rep| + |att|, tol = 1e-12 FP64, 1e-5 FP32) and the running
value drifts by at most the sum of that over the accepted moves, plus the
error of the initial full sum (12 * tol * the system's uabs).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_1408_3764_gb300 import workloads as W  # noqa: E402
from paper_1408_3764_gb300.gcmc import Batch, Box, Mix  # noqa: E402

TOL = {"fp64": 1e-12, "fp32": 1e-5}


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


def _system_uabs(o, L):
    """1/2 sum over the particles of their |rep| + |att| pair terms (oracle)."""
    cnt, X, _, _ = o.state()
    if len(X) == 0:
        return 0.0
    pos = X.astype(np.float64) * (L / 2.0 ** 32)
    spec = np.repeat(np.arange(len(cnt)), cnt).astype(np.int32)
    first = np.concatenate([[0], np.cumsum(cnt)])
    ex = [(int(s) << 32) | (i - int(first[s])) for i, s in enumerate(spec)]
    _, ua = o.trial_energy(pos, spec, exclude=ex, with_abs=True)
    return 0.5 * float(ua.sum())


def _setup(precision, n=1500, rho=0.55, S=2, seed=4):
    L = W.box_edge(n, rho)
    pos = _relaxed(n, L, seed)
    types = (np.arange(n) % 4 == 0).astype(np.int32) if S == 2 else np.zeros(n, np.int32)
    if S == 2:
        eps, sigma = W.lorentz_berthelot([1.0, 0.8], [1.0, 1.2])
    else:
        eps, sigma = [[1.0]], [[1.0]]
    o = O.System(L, 2.5, eps, sigma)
    o.build(pos, types)
    o.set_energy(o.total_energy())
    b = Box(L, 2.5, eps, sigma, precision=precision)
    b.set_chain_config(1)
    b.build_cells(torch.as_tensor(pos), torch.as_tensor(types))
    return L, o, b


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_running_virial_matches_oracle(precision):
    """Two-species mixture, 20,000 moves: identical decisions, and the running
    virial and its sum over the moves within the drift bound."""
    L, o, b = _setup(precision)
    tol = TOL[precision]
    u0 = _system_uabs(o, L)
    args = (0.4, 0.3, 0.3, 0.35, 1 / 1.3, [-2.2, -3.0])
    to, so = o.run_moves(77, 1000, 20_000, *args, tol=tol)
    sg, tg = b.run_moves(77, 1000, 20_000, Mix(*args, virial=True), trace=True)
    for k in ("type", "species", "index", "accepted"):
        assert np.array_equal(tg[k], to[k]), k
    acc = to["accepted"] == 1
    # per-move bound on the running value: initial sum + accepted trials so far
    bound_m = 12 * tol * (u0 + np.cumsum(np.where(acc, to["uabs"], 0.0))) + 1e-9
    assert abs(sg["virial"] - so.virial) <= bound_m[-1], (sg["virial"], so.virial, bound_m[-1])
    assert abs(sg["sum_virial"] - so.sum_virial) <= bound_m.sum(), (sg["sum_virial"], so.sum_virial)
    # the oracle's own running value equals its recomputed full sum
    assert so.virial == pytest.approx(o.energy_grad()["virial"], rel=1e-9, abs=1e-9)
    # and the GPU's equals the GPU's recomputed full sum
    u1 = _system_uabs(o, L)
    assert abs(sg["virial"] - b.energy_grad(want_pos=False)["virial"]) <= bound_m[-1] + 12 * tol * u1


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_virial_flag_changes_nothing_else(precision):
    """With and without the virial the chain takes the same moves and decisions,
    dU to rounding; without it the stats carry NaN."""
    L, _, a = _setup(precision, n=1200, rho=0.5, S=1, seed=21)
    _, _, c = _setup(precision, n=1200, rho=0.5, S=1, seed=21)
    mix = dict(p_disp=1 / 3, p_ins=1 / 3, p_del=1 / 3, max_disp=0.3, beta=1 / 1.2, log_z=[-2.786])
    sa, ta = a.run_moves(9, 0, 30_000, Mix(**mix), trace=True)
    sc, tc = c.run_moves(9, 0, 30_000, Mix(**mix, virial=True), trace=True)
    for k in ("type", "species", "index", "accepted"):
        assert np.array_equal(ta[k], tc[k]), k
    tol = TOL[precision]
    ok = np.isfinite(ta["lnA"])
    assert np.all(np.abs(ta["dU"] - tc["dU"])[ok] <= tol * ta["uabs"][ok] + 1e-300)
    assert np.isnan(sa["virial"]) and np.isnan(sa["sum_virial"])
    assert np.isfinite(sc["virial"]) and np.isfinite(sc["sum_virial"])
    drift = tol * ta["uabs"][ta["accepted"] == 1].sum() + 1e-9
    assert abs(sa["energy"] - sc["energy"]) <= 2 * drift
    for x, y in zip(a.get_state()[:4], c.get_state()[:4]):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_virial_restarts_after_a_run_without_it():
    """A run without the virial leaves it stale; the next virial run starts from
    a fresh full sum, and consecutive virial runs continue the running value."""
    L, o, b = _setup("fp64", n=900, rho=0.45, S=1, seed=8)
    args = (0.5, 0.25, 0.25, 0.3, 1 / 1.2, [-2.5])
    o.run_moves(3, 0, 5000, *args)
    b.run_moves(3, 0, 5000, Mix(*args))
    _, s1 = o.run_moves(3, 5000, 5000, *args)
    g1 = b.run_moves(3, 5000, 5000, Mix(*args, virial=True))
    _, s2 = o.run_moves(3, 10_000, 5000, *args)
    g2 = b.run_moves(3, 10_000, 5000, Mix(*args, virial=True))
    u = _system_uabs(o, L)
    for g, s in ((g1, s1), (g2, s2)):
        assert abs(g["virial"] - s.virial) <= 12 * 1e-12 * 20 * u + 1e-9
        assert abs(g["sum_virial"] - s.sum_virial) <= 5000 * (12 * 1e-12 * 20 * u + 1e-9)


def test_ideal_gas_virial_is_zero():
    """eps = 0: every pair term vanishes, so W and its sum stay exactly 0."""
    L = 8.0
    b = Box(L, 2.5, [[0.0]], [[1.0]])
    b.build_cells(torch.as_tensor(W.uniform_positions(200, L, 5)), torch.zeros(200, dtype=torch.int32))
    st = b.run_moves(1, 0, 20_000, Mix(0.4, 0.3, 0.3, 0.5, 1.0, [float(np.log(200 / L ** 3))], virial=True))
    assert st["virial"] == 0.0 and st["sum_virial"] == 0.0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_virial_per_chain(precision):
    """Batched chains, the virial on for some: each equals its oracle chain."""
    tol = TOL[precision]
    specs = [(300, 0.2, True), (900, 0.6, False), (700, 0.5, True)]
    boxes, oracles, mixes, seeds, u0 = [], [], [], [], []
    for k, (n, rho, vir) in enumerate(specs):
        L = max(W.box_edge(n, rho), 5.01)
        pos = _relaxed(n, L, 200 + k)
        b = Box(L, 2.5, [[1.0]], [[1.0]], precision=precision)
        b.build_cells(torch.as_tensor(pos), torch.zeros(n, dtype=torch.int32))
        o = O.System(L, 2.5, [[1.0]], [[1.0]])
        o.build(pos, np.zeros(n, np.int32))
        o.set_energy(o.total_energy())
        boxes.append(b)
        oracles.append((o, L))
        mixes.append(Mix(0.4, 0.3, 0.3, 0.3, 1 / 1.2, [float(np.log(rho) - 1.0)], virial=vir))
        seeds.append(500 + k)
        u0.append(_system_uabs(o, L))
    stats = Batch(boxes).run_moves(seeds, 0, 15_000, mixes)
    for k, (o, L) in enumerate(oracles):
        m = mixes[k]
        to, so = o.run_moves(seeds[k], 0, 15_000, m.p_disp, m.p_ins, m.p_del, m.max_disp, m.beta, m.log_z,
                             tol=tol, chain=k)
        assert list(so.accepted) == stats[k]["accepted"]
        if not m.virial:
            assert np.isnan(stats[k]["virial"])
            continue
        acc = to["accepted"] == 1
        bound_m = 12 * tol * (u0[k] + np.cumsum(np.where(acc, to["uabs"], 0.0))) + 1e-9
        assert abs(stats[k]["virial"] - so.virial) <= bound_m[-1]
        assert abs(stats[k]["sum_virial"] - so.sum_virial) <= bound_m.sum()
