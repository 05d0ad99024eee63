"""GPU: the cutoff sweep (Sec. 4, performance against the cutoff: 87,296
particles in 131,072 sigma^3, rc from 2.5 to 4.25 sigma) at full size.

At each tested cutoff the cell build is bit-exact, the full-system energy is
within tol * uabs of the oracle's, and a chain of 20,000 moves takes the
oracle's decisions move by move with dU within tol * uabs and ends in the
oracle's configuration (tol = 1e-12 FP64, 1e-5 FP32; uabs the sum of |rep| +
|att| over the evaluated pair terms).
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


def _pair(w, precision):
    pos, types = w.positions(), w.types()
    o = O.System(w.L, w.rc, w.eps, w.sigma)
    cl = o.build(pos, types)
    b = Box(w.L, w.rc, w.eps, w.sigma, precision=precision)
    b.build_cells(torch.as_tensor(pos), torch.as_tensor(types))
    return o, cl, b


@pytest.mark.parametrize("rc", [2.5, 3.25, 4.25])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sweep_chain_parity(rc, precision):
    w = W.cutoff_sweep(rc)
    o, cl, b = _pair(w, precision)
    g = b.geometry()
    assert g["T"] == int(w.L // rc)
    cs, cc, order = b.cell_list()
    assert np.array_equal(cc.cpu().numpy(), cl.cell_count)
    assert np.array_equal(cs.cpu().numpy(), cl.cell_start)
    assert np.array_equal(order.cpu().numpy(), cl.order)
    # full-system energy against the oracle, scaled by the system's uabs
    E = o.total_energy()
    cnt, X, _, _ = o.state()
    pos = X.astype(np.float64) * (w.L / 2.0 ** 32)
    ex = np.arange(len(pos), dtype=np.int64)  # single species: id = index
    _, ua = o.trial_energy(pos, np.zeros(len(pos), np.int32), exclude=ex, with_abs=True)
    assert abs(b.total_energy() - E) <= TOL[precision] * 0.5 * ua.sum()
    # the chain, move by move
    o.set_energy(E)
    m = 20_000
    to, so = o.run_moves(w.seed, 0, m, w.p_disp, w.p_ins, w.p_del, w.max_disp, w.beta, w.log_z,
                         tol=TOL[precision])
    sg, tg = b.run_moves(w.seed, 0, m, Mix(w.p_disp, w.p_ins, w.p_del, w.max_disp, w.beta, w.log_z),
                         trace=True)
    for k in ("type", "species", "index", "accepted"):
        assert np.array_equal(tg[k], to[k]), k
    ok = np.isfinite(to["lnA"])
    err = np.abs(tg["dU"] - to["dU"])[ok]
    assert np.all(err <= TOL[precision] * to["uabs"][ok] + 1e-300)
    for x, y in zip(o.state(), b.get_state()[:4]):
        assert np.array_equal(x, y)
