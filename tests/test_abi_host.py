"""CPU-only checks of the C ABI library: it loads, exports every function
that include/cgdem.h declares, and its host-only helpers agree with the
oracle and the paper.  No GPU is touched."""
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2211_06142_gb300 import build as B
from paper_2211_06142_gb300 import cgdem
from paper_2211_06142_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return cgdem.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cgdem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cgdem_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_function(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(cgdem.EXPORTS)


def test_rayleigh_dt_matches_oracle_and_paper(lib, printed):
    for Rbar in [5e-5, 1.15e-4, 3e-4]:
        for E, nu in [(1e8, 0.3), (2e10, 0.3), (5e9, 0.25)]:
            assert cgdem.cgdem_rayleigh_dt(Rbar, 2605.0, E, nu) == O.rayleigh_dt(Rbar, 2605.0, E, nu)
    t2 = printed["table2"]
    w = np.array(t2["mass_fraction"])
    d = np.array(t2["d_original_mm"]) * 1e-3
    dbar = (w.sum() / (w / d ** 3).sum()) ** (1 / 3)
    frac = 1e-8 / cgdem.cgdem_rayleigh_dt(dbar / 2, 2605.0, 2e10, 0.3)
    assert round(100 * frac, 1) == 4.4


@pytest.mark.parametrize("scheme,name", [(cgdem.CG_SSW, "ssw"), (cgdem.CG_SSP, "ssp")])
@pytest.mark.parametrize("k", [2, 3])
def test_cg_scaling_matches_oracle(lib, scheme, name, k):
    d = I.table2_diameters(270000, np.random.default_rng(4))
    g = cgdem.cgdem_cg_scale_diameters(d, k, scheme)
    o, gam = O.cg_scale(d, k, name, 30.0)
    assert len(g) == len(o) == 270000 // k ** 3
    np.testing.assert_allclose(g, o, rtol=1e-13)
    assert gam == k * 30.0


def test_workspace_size_and_invalid_arguments(lib):
    s = I.cached(I.small_periodic, 600, 11)
    p = cgdem.sample_params(s, 1e-7, 2e-5)
    import ctypes as C
    cfg = cgdem.Config(cgdem.MIXED, 1, 48, 128, 0.0, 32)
    arr = (cgdem.SampleParams * 1)(p)
    counts = np.array([600], np.int64)
    nb = C.c_size_t(0)
    assert lib.cgdem_workspace_size(C.byref(cfg), arr, counts.ctypes.data, C.byref(nb)) == 0
    assert nb.value > 600 * 1000
    # bond-break separation larger than the skin -> rejected before any GPU work
    p2 = cgdem.sample_params(s, 1e-7, 1e-12)
    arr2 = (cgdem.SampleParams * 1)(p2)
    assert lib.cgdem_workspace_size(C.byref(cfg), arr2, counts.ctypes.data, C.byref(nb)) == cgdem.CGDEM_E_INVALID
    # non-cubic periodic box -> rejected
    p3 = cgdem.sample_params(s, 1e-7, 2e-5)
    p3.L[2] = 2 * p3.L[2]
    arr3 = (cgdem.SampleParams * 1)(p3)
    assert lib.cgdem_workspace_size(C.byref(cfg), arr3, counts.ctypes.data, C.byref(nb)) == cgdem.CGDEM_E_INVALID
    # too many neighbours per sphere
    cfg2 = cgdem.Config(cgdem.MIXED, 1, 4096, 128, 0.0, 32)
    assert lib.cgdem_workspace_size(C.byref(cfg2), arr, counts.ctypes.data, C.byref(nb)) == cgdem.CGDEM_E_INVALID
    # spheres per warp of the force kernel: 0, 16 or 32
    for ppw, rc in ((16, 0), (32, 0), (0, 0), (8, cgdem.CGDEM_E_INVALID)):
        cfg3 = cgdem.Config(cgdem.MIXED, 1, 48, 128, 0.0, 32, 0, ppw)
        assert lib.cgdem_workspace_size(C.byref(cfg3), arr, counts.ctypes.data, C.byref(nb)) == rc
    # form of the Darcy solve: 0 (one cooperative launch) or 1 (a kernel per phase)
    for fk, rc in ((0, 0), (1, 0), (2, cgdem.CGDEM_E_INVALID)):
        cfg4 = cgdem.Config(cgdem.MIXED, 1, 48, 128, 0.0, 32, 0, 32, 0, 0.0, fk)
        assert lib.cgdem_workspace_size(C.byref(cfg4), arr, counts.ctypes.data, C.byref(nb)) == rc


def test_noalloc_rejects_oversize_without_gpu(lib):
    with pytest.raises(cgdem.CgdemError) as e:
        cgdem.cgdem_touching_pairs_noalloc(1, 1, 262145, np.zeros(3), np.ones(3), 0, 0.1, 0.0, 1, 1, 1)
    assert e.value.code == cgdem.CGDEM_E_CAPACITY


def test_context_refuses_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    s = I.cached(I.small_periodic, 600, 11)
    p = cgdem.sample_params(s, 1e-7, 2e-5)
    with pytest.raises(RuntimeError):
        cgdem.Context([p], [600])
