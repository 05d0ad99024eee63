"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports
every symbol include/gcmc.h declares.  No compute call is made (no GPU here)."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gcmc.h")).read()
    src += open(os.path.join(ROOT, "include", "gcmc_probe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gcmc_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ["gcmc_create", "gcmc_destroy", "gcmc_build_cells", "gcmc_trial_energy", "gcmc_run_moves",
                 "gcmc_total_energy", "gcmc_energy_grad", "gcmc_get_state", "gcmc_set_state",
                 "gcmc_last_error"]:
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_1408_3764_gb300 import _lib
    L = _lib.load()
    for name in _declared():
        assert hasattr(L, name), name
    assert set(_declared()) <= set(_lib.SIGNATURES)
    assert b"sm_103a" in L.gcmc_version()


def test_library_is_independent_of_the_oracle():
    """The product library neither defines nor imports any oracle symbol."""
    from paper_1408_3764_gb300 import _lib
    path = _lib.load()._name
    out = subprocess.run(["nm", "-D", path], capture_output=True, text=True).stdout
    assert "orc_" not in out
    assert "gcmc_oracle" not in out


def test_library_built_for_sm_103a():
    from paper_1408_3764_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    from paper_1408_3764_gb300 import _lib
    path = _lib.load()._name
    out = subprocess.run(["cuobjdump", "--list-elf", path], capture_output=True, text=True)
    if out.returncode == 0:
        assert "sm_103a" in out.stdout


def test_null_and_bad_arguments_without_gpu():
    """Argument checks happen on the host before any device work."""
    from paper_1408_3764_gb300 import _lib
    L = _lib.load()
    h = C.c_void_p()
    assert L.gcmc_create(None, None, C.byref(h)) == 1
    p = _lib.Params()
    eps = np.array([1.0])
    sig = np.array([1.0])
    p.L, p.rc, p.n_species, p.precision = 5.0, 3.0, 1, 0  # 2 rc > L
    p.eps = eps.ctypes.data_as(C.POINTER(C.c_double))
    p.sigma = sig.ctypes.data_as(C.POINTER(C.c_double))
    assert L.gcmc_create(C.byref(p), None, C.byref(h)) == 1
    p.rc, p.n_species = 2.5, 9
    assert L.gcmc_create(C.byref(p), None, C.byref(h)) == 1
    assert L.gcmc_destroy(None) == 0
    assert L.gcmc_last_error(None) == b"null context"
    assert L.gcmc_set_chain_profile(None, 1) == 1


def test_species_major_order():
    from paper_1408_3764_gb300.gcmc import species_major_order
    s = np.array([1, 0, 1, 0, 0, 1])
    assert list(species_major_order(s)) == [1, 3, 4, 0, 2, 5]


def test_workloads_are_seeded_and_shaped():
    from paper_1408_3764_gb300 import workloads as W
    a = W.c1_plain_fp64()
    assert a.L == pytest.approx(16.0)
    assert np.array_equal(a.positions(), W.c1_plain_fp64().positions())
    c2 = W.c2_fp32_vs_fp64()
    assert c2.L == pytest.approx(60.226, abs=1e-3)
    c3 = W.c3_mixture_1m()
    t = c3.types()
    assert abs(t.mean() - 0.2) < 0.01
    iso = W.isotherm_chains()
    assert len(iso) == 64
    ns = np.array([w.n for w in iso])
    assert ns.min() >= 500 and ns.max() <= 20000
