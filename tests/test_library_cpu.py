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


@pytest.mark.parametrize("seed", [5, 6, 7, 8])
def test_exact_shifts_filter_and_preserve_similarity(lib, seed):
    # implicit restart step: applying the p unwanted eigenvalues mu_i as
    # shifts is an orthogonal similarity to a Hessenberg matrix whose Q has
    # a zero last row in its first k-1 columns and whose first column is
    # psi(H) e1 / |psi(H) e1| with psi(x) = prod (x - mu_i) (implicit Q
    # theorem).  Whether H_s[k, k-1] also comes out small depends on the
    # size of H's subdiagonal (exact shifts are forward unstable), so that
    # is not asserted.
    m, k = 20, 8
    H = _hess(m, seed)
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
    x = np.zeros(m, complex)
    x[0] = 1.0
    for mu in sh:
        x = H @ x - mu * x
        x /= np.linalg.norm(x)
    assert np.linalg.norm(x.imag) < 1e-8          # conjugate pairs: a real polynomial
    x = x.real / np.linalg.norm(x.real)
    assert min(np.linalg.norm(Q[:, 0] - x), np.linalg.norm(Q[:, 0] + x)) < 1e-9


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


def _ff_dot(lib, a, b):
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = np.zeros(1)
    assert lib.fv_host_ff_dot(a.size, a.ctypes.data, b.ctypes.data, out.ctypes.data) == 0
    return float(out[0])


def test_ff_split_truncation_bound(lib):
    # one term times 1.0 returns hi + lo of the truncating split
    rng = np.random.default_rng(13)
    d = rng.choice([-1.0, 1.0], 4000) * rng.uniform(1, 2, 4000) * 2.0 ** rng.integers(-80, 100, 4000)
    got = np.array([_ff_dot(lib, [x], [1.0]) for x in d])
    assert np.all(np.abs(got - d) < 2.0 ** -46 * np.abs(d))
    assert np.all(np.abs(got) <= np.abs(d))               # truncation toward zero
    # below 2^-80 only the leading float is kept; below 2^-126 nothing
    tiny = np.array([2.0 ** -81 * 1.7, 2.0 ** -110, -3.0 * 2.0 ** -120, 2.0 ** -127, 0.0, -0.0])
    got = np.array([_ff_dot(lib, [x], [1.0]) for x in tiny])
    assert np.all(np.abs(got - tiny) <= np.maximum(2.0 ** -23 * np.abs(tiny), 2.0 ** -126))


@pytest.mark.parametrize("scale", [1.0, 1e-12, 1e12])
def test_ff_dot_against_exact_sum(lib, scale):
    from fractions import Fraction
    rng = np.random.default_rng(14)
    n = 3000
    a = rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 3, n) * scale
    b = rng.standard_normal(n)
    exact = float(sum(Fraction(x) * Fraction(y) for x, y in zip(a, b)))
    mag = float(np.sum(np.abs(a * b)))
    got = _ff_dot(lib, a, b)
    # per term: split (2 x 2^-46) + dropped lo*lo + one renormalised add
    assert abs(got - exact) <= 2.0 ** -43 * mag
    # a sum that cancels to ~1e-10 of its terms keeps its absolute accuracy
    c = np.concatenate([a, -a[::-1]])
    d = np.concatenate([b, b[::-1] * (1 + 1e-10)])
    exact = float(sum(Fraction(x) * Fraction(y) for x, y in zip(c, d)))
    got = _ff_dot(lib, c, d)
    assert abs(got - exact) <= 2.0 ** -43 * float(np.sum(np.abs(c * d)))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_hessenberg_qr_near_a_multiple_of_the_identity(lib, seed):
    # H = lambda0 I + E with |E| ~ 1e-8 |lambda0| (a cluster of unwanted Ritz
    # values met by the Arnoldi method at 100^3): the Francis step must form
    # its first column from h_ii - shift, or rounding of h_ii^2 hides E
    import scipy.linalg
    rng = np.random.default_rng(seed)
    n = 12
    E = scipy.linalg.hessenberg(rng.standard_normal((n, n)) * 1e-3)
    H = np.ascontiguousarray(-47898.2 * np.eye(n) + E)
    wr = np.zeros(n); wi = np.zeros(n)
    assert lib.fv_host_hess_eigenvalues(n, H.ctypes.data, wr.ctypes.data, wi.ctypes.data) == 0
    got = np.sort_complex(wr + 1j * wi) + 47898.2
    ref = np.sort_complex(np.linalg.eigvals(E))
    lapack = np.sort_complex(np.linalg.eigvals(H)) + 47898.2
    # the eigenvalues of H are those of E shifted; forming H rounds E's
    # diagonal to 7e-12, which moves these (non-normal) eigenvalues by up to
    # a few 1e-9 for LAPACK too
    err_lapack = np.abs(lapack - ref).max()
    assert np.abs(got - ref).max() <= 2 * err_lapack + 1e-10, (np.abs(got - ref).max(), err_lapack)
