"""GPU: the allocation-free full-system energy (gcmc_total_energy_noalloc)
against the ordinary entry point (gcmc_total_energy) and the CPU oracle,
through the C ABI.

Both run on the same context after moves have reordered the cells; the
variant reads the padded cell layout and sums into the library's static
device array.  It is called twice in a row (the second call reuses the
array) and each result must equal gcmc_total_energy within the tolerance of
the energy parity tests: tol * uabs, uabs = 1/2 sum over the pair terms of
|4 eps s^12| + |4 eps s^6|, tol = 1e-12 (FP64) or 1e-5 (FP32).
"""
import ctypes as C

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


def _noalloc(box, out):
    L = _lib.load()
    st = L.gcmc_total_energy_noalloc(box._h, C.c_void_p(out.data_ptr()))
    _lib.check(st, box._h, "gcmc_total_energy_noalloc")
    box.stream.synchronize()
    return out.item()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_energy_matches_total_energy_twice(precision):
    n, L, S = 1800, 15.0, 2
    pos = _relaxed(n, L, 31)
    types = (np.arange(n) % 3 == 0).astype(np.int32)
    eps, sigma = W.lorentz_berthelot([1.0, 0.8], [1.0, 1.15])
    b = Box(L, 2.5, eps, sigma, precision=precision)
    b.build_cells(torch.as_tensor(pos), torch.as_tensor(types))
    # moves reorder the cells (swap-with-last, appends) and change N
    b.run_moves(9, 0, 5000, Mix(0.5, 0.25, 0.25, 0.3, 1 / 1.2, [-2.4, -3.0]))
    ref = b.total_energy()
    # scale of the rounding error: 1/2 sum of the per-particle |terms|
    cnt, X, _, _, _ = b.get_state()
    pos_now = X.astype(np.float64) * (L / 2.0 ** 32)
    spec = np.repeat(np.arange(S), cnt[:S]).astype(np.int32)
    first = np.concatenate([[0], np.cumsum(cnt[:S])])
    ex = [(int(s) << 32) | (i - int(first[s])) for i, s in enumerate(spec)]
    _, uabs = b.trial_energy(pos_now, spec, exclude=ex, with_abs=True)
    scale = 0.5 * float(uabs.cpu().numpy().sum())
    out = torch.full((1,), float("nan"), dtype=torch.float64, device=b.device)
    for _ in range(2):
        got = _noalloc(b, out)
        assert abs(got - ref) <= TOL[precision] * scale, (got, ref, scale)
        out.fill_(float("nan"))
    # the running energy of the chain is not touched
    assert b.get_state()[4] == ref


def test_noalloc_rejects_host_pointer_and_empty_box_is_zero():
    b = Box(10.0, 2.5, [[1.0]], [[1.0]])
    b.build_cells(torch.zeros((0, 3), dtype=torch.float64), torch.zeros(0, dtype=torch.int32))
    out = torch.full((1,), float("nan"), dtype=torch.float64, device=b.device)
    assert _noalloc(b, out) == 0.0
    host = np.zeros(1)
    st = _lib.load().gcmc_total_energy_noalloc(b._h, C.c_void_p(host.ctypes.data))
    assert st == 1  # INVALID_ARG


def test_noalloc_energy_matches_oracle():
    """FP64 mode against the oracle's full-system energy of the same
    configuration (after moves), within 1e-12 of the pair terms' scale."""
    n, L = 1500, 14.0
    pos = _relaxed(n, L, 41)
    b = Box(L, 2.5, [[1.0]], [[1.0]], precision="fp64")
    b.build_cells(torch.as_tensor(pos), torch.zeros(n, dtype=torch.int32))
    b.run_moves(3, 0, 4000, Mix(0.5, 0.25, 0.25, 0.3, 1 / 1.2, [-2.6]))
    cnt, X, _, _, _ = b.get_state()
    o = O.System(L, 2.5, [[1.0]], [[1.0]])
    # the centres of the grid cells quantise back to the same grid points
    o.build((X.astype(np.float64) + 0.5) * (L / 2.0 ** 32), np.zeros(len(X), np.int32))
    ref = o.total_energy()
    _, uabs = o.trial_energy(*_self_points(o, X, L), with_abs=True)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device=b.device)
    got = _noalloc(b, out)
    assert abs(got - ref) <= 1e-12 * 0.5 * uabs.sum(), (got, ref)


def _self_points(o, X, L):
    pos = (X.astype(np.float64) + 0.5) * (L / 2.0 ** 32)
    return pos, np.zeros(len(X), np.int32), np.arange(len(X), dtype=np.int64)


def test_noalloc_rejects_oversize_box_and_pinned_host_memory():
    """A box of 51^3 = 132,651 cells exceeds the static array of
    GCMC_NOALLOC_MAX_CELLS and is refused; so is pinned host memory."""
    b = Box(128.0, 2.5, [[1.0]], [[1.0]])
    assert b.geometry()["n_cells"] == 51 ** 3 > _lib.NOALLOC_MAX_CELLS
    b.build_cells(torch.zeros((0, 3), dtype=torch.float64), torch.zeros(0, dtype=torch.int32))
    out = torch.full((1,), float("nan"), dtype=torch.float64, device=b.device)
    st = _lib.load().gcmc_total_energy_noalloc(b._h, C.c_void_p(out.data_ptr()))
    assert st == 1  # INVALID_ARG
    assert "cells exceed" in _lib.load().gcmc_last_error(b._h).decode()
    small = Box(10.0, 2.5, [[1.0]], [[1.0]])
    small.build_cells(torch.as_tensor(W.uniform_positions(50, 10.0, 2)), torch.zeros(50, dtype=torch.int32))
    pinned = torch.zeros(1, dtype=torch.float64).pin_memory()
    st = _lib.load().gcmc_total_energy_noalloc(small._h, C.c_void_p(pinned.data_ptr()))
    assert st == 1  # INVALID_ARG
