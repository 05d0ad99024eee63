"""GPU: failure detection without a GPU fault.

* A bounded wait that runs out: the committer, at a chosen move, waits on a
  flag that nothing sets (the diagnostic hook gcmc_set_wait_limit, 10 ms
  limit).  The kernel returns a timeout status, gcmc_run_moves reports
  TIMEOUT with every committed move applied and booked, the configuration
  passes the host consistency check, and the same context then continues the
  chain -- move for move the oracle's.
* A corrupted checkpoint is refused by gcmc_set_state and the context keeps
  its configuration.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_1408_3764_gb300 import _lib  # noqa: E402
from paper_1408_3764_gb300 import workloads as W  # noqa: E402
from paper_1408_3764_gb300.gcmc import Box, Mix  # noqa: E402

TOL = {"fp64": 1e-12, "fp32": 1e-5}
TIMEOUT = 5  # GCMC_ERR_TIMEOUT


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


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_stalled_committer_times_out_and_context_stays_usable(precision):
    L = W.box_edge(800, 0.5)
    pos = _relaxed(800, L, 7)
    args = (1 / 3, 1 / 3, 1 / 3, 0.3, 1 / 1.2, [-2.7])
    o = O.System(L, 2.5, [[1.0]], [[1.0]])
    o.build(pos, np.zeros(800, np.int32))
    o.set_energy(o.total_energy())
    b = Box(L, 2.5, [[1.0]], [[1.0]], precision=precision)
    b.set_chain_config(0)
    b.build_cells(torch.as_tensor(pos), torch.zeros(800, dtype=torch.int32))
    b.set_wait_limit(10_000_000, stall_move=1500)
    st = b.run_moves(5, 0, 5000, Mix(*args), check_status=False)
    assert st["status"] == TIMEOUT
    assert st["moves_done"] == 1500
    assert "bounded wait" in _lib.load().gcmc_last_error(b.handle).decode()
    b.check_state()
    # the running energy covers exactly the applied moves
    to1, _ = o.run_moves(5, 0, 1500, *args, tol=TOL[precision])
    drift = TOL[precision] * to1["uabs"][to1["accepted"] == 1].sum() + 1e-9
    assert abs(st["energy"] - b.total_energy()) <= 2 * drift
    for x, y in zip(o.state(), b.get_state()[:4]):
        assert np.array_equal(x, y)
    # the context carries on: the rest of the chain is the oracle's
    b.set_wait_limit(0, -1)
    st2, tr2 = b.run_moves(5, 1500, 3500, Mix(*args), trace=True)
    assert st2["status"] == 0 and st2["moves_done"] == 3500
    to2, _ = o.run_moves(5, 1500, 3500, *args, tol=TOL[precision])
    for k in ("type", "species", "index", "accepted"):
        assert np.array_equal(tr2[k], to2[k]), k
    for x, y in zip(o.state(), b.get_state()[:4]):
        assert np.array_equal(x, y)
    b.check_state()


def test_corrupted_checkpoint_is_refused():
    L = W.box_edge(600, 0.5)
    b = Box(L, 2.5, [[1.0]], [[1.0]])
    b.build_cells(torch.as_tensor(_relaxed(600, L, 8)), torch.zeros(600, dtype=torch.int32))
    b.run_moves(2, 0, 3000, Mix(1 / 3, 1 / 3, 1 / 3, 0.3, 1 / 1.2, [-2.7]))
    n, X, cc, refs, E = b.get_state()
    nz = np.flatnonzero(cc)
    bad = []
    r = refs.copy()
    r[0], r[-1] = r[-1], r[0]  # two particles listed in each other's cells
    bad.append((n, X, cc, r))
    r = refs.copy()
    r[1] = r[0]  # a particle listed twice, another not at all
    bad.append((n, X, cc, r))
    c = cc.copy()
    c[nz[0]] += 1
    c[nz[1]] -= 1  # counts that no longer match the positions
    bad.append((n, X, c, refs))
    for args in bad:
        with pytest.raises(RuntimeError):
            b.restore(*args, energy=E)
    # the configuration is the one before the refused restores
    after = b.get_state()
    for x, y in zip((n, X, cc, refs), after[:4]):
        assert np.array_equal(np.asarray(x), np.asarray(y))
    b.check_state()
    b.restore(n, X, cc, refs, energy=E)
    b.check_state()
