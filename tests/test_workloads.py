"""CPU: the seeded input generators (they hold none of the method's
arithmetic, only the shapes of the paper's workloads)."""
import numpy as np
import pytest

from paper_1408_3764_gb300 import workloads as W


def _min_periodic_distance(p, L):
    scipy = pytest.importorskip("scipy.spatial")
    d, _ = scipy.cKDTree(p, boxsize=L).query(p, k=2)
    return float(d[:, 1].min())


@pytest.mark.parametrize("n,L,dmin,seed", [(3000, 16.0, 0.9, 1), (800, 10.0, 0.85, 2), (50, 6.0, 1.0, 3)])
def test_separated_positions_keep_their_distance(n, L, dmin, seed):
    p = W.separated_positions(n, L, dmin, seed)
    assert p.shape == (n, 3) and p.dtype == np.float64
    assert (p >= 0.0).all() and (p < L).all()
    assert _min_periodic_distance(p, L) >= dmin
    # the same arguments give the same positions; another seed others
    assert np.array_equal(p, W.separated_positions(n, L, dmin, seed))
    assert not np.array_equal(p, W.separated_positions(n, L, dmin, seed + 1))


def test_separated_positions_refuses_an_impossible_packing():
    with pytest.raises(ValueError):
        W.separated_positions(50, 4.0, 1.2, 3)  # packing fraction 0.7


def test_cutoff_sweep_workloads():
    assert len(W.SWEEP_RC) == len(W.SWEEP_LOGZ) == 8
    for rc in W.SWEEP_RC:
        w = W.cutoff_sweep(rc, moves=10)
        assert w.n == 87296 and w.L == pytest.approx(131072.0 ** (1 / 3))
        assert w.rho == pytest.approx(87296 / 131072.0)
        assert w.L >= 2 * rc and w.dmin == 0.9 and w.temperature == 1.5


def test_isotherm_chains_span_the_isotherm():
    ch = W.isotherm_chains()
    assert len(ch) == 64
    rho = np.array([w.rho for w in ch])
    assert rho.min() == pytest.approx(0.1) and rho.max() == pytest.approx(0.7)
    n = np.array([w.n for w in ch])
    assert n.min() >= 500 and n.max() <= 20000
    assert all(w.L >= 2 * w.rc for w in ch)
