"""CPU checks of the C-ABI library: it loads, exports every declared symbol,
and its host-side small dense routines (Hessenberg QR, implicit shifts)
agree with the mathematics.  No GPU compute is called."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1704_08521_gb300._lib import lib
    return lib


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return set(re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", txt)) - {"if", "sizeof"}


def test_exports_every_declared_symbol(lib):
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            names |= _declared(h)
    assert {"fv_grid_create", "ns_residual", "ns_jacvec", "simple_krylov_solve",
            "newton_steady", "arnoldi_leading"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_invalid_arguments_rejected_without_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.fv_grid_create(3, 8, 8, 1, 0.0, 100.0, None, ctypes.byref(h)) == 1   # FV_EINVAL
    assert b"[4, 1024]" in lib.fv_last_error()
    assert lib.fv_grid_create(8, 8, 8, 7, 0.0, 100.0, None, ctypes.byref(h)) == 1
    assert lib.fv_grid_create(8, 8, 8, 1, 0.0, -1.0, None, ctypes.byref(h)) == 1
    assert lib.ns_jacvec(None, None, None, None, 0) == 1


def _hess(m, seed):
    rng = np.random.default_rng(seed)
    return np.triu(rng.standard_normal((m, m)), -1)


@pytest.mark.parametrize("m", [3, 7, 30, 60])
def test_hessenberg_eigenvalues_match_lapack(lib, m):
    H = _hess(m, m)
    wr = np.zeros(m); wi = np.zeros(m)
    Hc = np.ascontiguousarray(H)
    assert lib.fv_host_hess_eigenvalues(m, Hc.ctypes.data, wr.ctypes.data, wi.ctypes.data) == 0
    got = np.sort_complex(wr + 1j * wi)
    ref = np.sort_complex(np.linalg.eigvals(H))
    np.testing.assert_allclose(got, ref, atol=1e-10 * np.abs(ref).max())


def test_exact_shifts_deflate_and_preserve_similarity(lib):
    # implicit restart step: applying the p unwanted eigenvalues as shifts
    # leaves a similar Hessenberg matrix whose leading k x k block carries the
    # wanted eigenvalues and whose Q has a zero last row in its first k-1 columns
    m, k = 20, 8
    H = _hess(m, 5)
    lam = np.linalg.eigvals(H)
    lam = lam[np.lexsort((-lam.imag, -lam.real))]
    if abs(lam[k - 1].imag) > 0 and abs(lam[k - 1] - np.conj(lam[k])) < 1e-12:
        k += 1
    sh = lam[k:]
    Hs = np.ascontiguousarray(H.copy()); Q = np.ascontiguousarray(np.eye(m))
    sr = np.ascontiguousarray(sh.real); si = np.ascontiguousarray(sh.imag)
    assert lib.fv_host_shift_steps(m, Hs.ctypes.data, Q.ctypes.data, len(sh), sr.ctypes.data, si.ctypes.data) == 0
    np.testing.assert_allclose(Q.T @ Q, np.eye(m), atol=1e-12)
    np.testing.assert_allclose(Q.T @ H @ Q, Hs, atol=1e-9)
    assert np.abs(np.tril(Hs, -2)).max() == 0
    assert np.abs(Q[m - 1, :k - 1]).max() < 1e-12
    assert abs(Hs[k, k - 1]) < 1e-6 * np.abs(H).max()
    np.testing.assert_allclose(np.sort_complex(np.linalg.eigvals(Hs[:k, :k])), np.sort_complex(lam[:k]), atol=1e-7)
