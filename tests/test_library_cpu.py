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


def test_ff_conversions_match_ieee(lib):
    # integer-only double <-> float-float conversions of the mixed path
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-30, 30, 20000),
                        [0.0, -0.0, 1.0, -1.0, 1e-40, 3.4e38, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24,
                         np.pi, -np.e, 1e-30, 2.0 ** -126]])
    n = x.size
    hi = np.zeros(n, np.float32); lo = np.zeros(n, np.float32)
    jo = np.zeros(n); ro = np.zeros(n, np.float32)
    assert lib.fv_host_ff_convert(n, x.ctypes.data, hi.ctypes.data, lo.ctypes.data,
                                  jo.ctypes.data, ro.ctypes.data) == 0
    normal = np.abs(x) >= 2.0 ** -126
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32)
    assert np.array_equal(ro[normal], ref[normal])                  # round to nearest even
    assert np.array_equal(hi, ro)
    big = np.abs(x) > 1e-20
    np.testing.assert_allclose(lo[big].astype(np.float64), (x - hi.astype(np.float64))[big],
                               rtol=2.0 ** -23, atol=0)
    np.testing.assert_allclose(jo[big], x[big], rtol=2.0 ** -47, atol=0)
    # joining the pair reproduces hi + lo exactly when it is representable
    pair = hi.astype(np.float64) + lo.astype(np.float64)
    np.testing.assert_array_equal(jo[big], pair[big])


def test_ff_arithmetic_48_bits(lib):
    rng = np.random.default_rng(12)
    n = 5000
    def ffpair(v):
        h = v.astype(np.float32)
        l = (v - h.astype(np.float64)).astype(np.float32)
        return np.ascontiguousarray(np.stack([h, l], 1).ravel()), h.astype(np.float64) + l
    a, av = ffpair(rng.standard_normal(n))
    b, bv = ffpair(rng.standard_normal(n) * 0.999)
    c, cv = ffpair(rng.standard_normal(n) * 3.0)
    out = np.zeros(2 * n, np.float32)
    lib.fv_host_ff_arith(n, a.ctypes.data, b.ctypes.data, c.ctypes.data, out.ctypes.data)
    got = out[0::2].astype(np.float64) + out[1::2]
    ref = (av + bv) * cv
    scale = (np.abs(av) + np.abs(bv)) * np.abs(cv)
    assert np.all(np.abs(got - ref) <= 2.0 ** -44 * scale)
