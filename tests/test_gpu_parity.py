"""GPU parity: every C-ABI entry point against the FP64 oracle on the same
seeded inputs (element by element).  Sizes span several 64-wide tiles of the
pressure-correction transforms with ragged tails, odd and non-cubic shapes,
and the minimum grid; the 100^3 benchmark grid and the 150^3 / 256^3 grids
are in test_gpu_fullsize.py.

Tolerances (max |gpu - oracle| / max |oracle|):
  FP64 stencils and residual          1e-12  (round-off of ~10^2 terms)
  FP64 pressure solve / Krylov vector 1e-10  (tensor transforms, K ~ N)
  mixed (FP32 sweeps in FP64 loop)    2e-5   (FP32 J.v, ~1e-7 per term,
                                              amplified by the stencil's
                                              cancellation on stretched grids)
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
import layout  # noqa: E402
from oracle import fv as ofv, grid as og, poisson, simple, krylov, dense, arnoldi  # noqa: E402

SHAPES = [(4, 4, 4, "uniform"), (7, 6, 5, "cosine"), (9, 11, 13, "sine0975"),
          (66, 67, 65, "cosine"), (20, 130, 24, "cosine")]


@pytest.fixture(scope="module")
def fv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1704_08521_gb300 as m
    return m


def relerr(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def setup(fv, nz, ny, nx, kind, alpha=0.3, re=700.0, seed=1):
    shape = (nz, ny, nx)
    g = fv.Grid(nx, ny, nz, kind, alpha=alpha, re=re)
    og_grid = og.Grid(nx, ny, nz, kind)
    U = synth.vortex_base_flow(shape, kind, alpha)
    v = synth.gaussian_velocity(shape, seed)
    return g, og_grid, shape, U, v


@pytest.mark.parametrize("nz,ny,nx,kind", SHAPES)
def test_jacvec(fv, nz, ny, nx, kind):
    g, G, shape, U, v = setup(fv, nz, ny, nx, kind)
    ref = layout.from_oracle(ofv.jacvec(G, layout.to_oracle(U, shape), layout.to_oracle(v, shape), 700.0))
    out = torch.empty(g.n_vel, dtype=torch.float64, device="cuda")
    fv.ns_jacvec(g, dev(U), dev(v), out, "fp64")
    assert relerr(host(out), ref) < 1e-12
    fv.ns_jacvec(g, dev(U), dev(v), out, "mixed")
    assert relerr(host(out), ref) < 2e-5
    fv.ns_jacvec(g, dev(U), dev(v), out, "ff")           # float-float on the FP32 pipes
    assert relerr(host(out), ref) < 1e-11


@pytest.mark.parametrize("nz,ny,nx,kind", SHAPES)
def test_residual(fv, nz, ny, nx, kind):
    g, G, shape, U, v = setup(fv, nz, ny, nx, kind)
    P = synth.gaussian_cells(shape, 5)
    rm, rd = ofv.residual(G, layout.to_oracle(U, shape), P.reshape(shape), 700.0, ofv.lid_velocity(0.3))
    Fm = torch.empty(g.n_vel, dtype=torch.float64, device="cuda")
    Fd = torch.empty(g.n_cell, dtype=torch.float64, device="cuda")
    fv.ns_residual(g, dev(U), dev(P), Fm, Fd)
    assert relerr(host(Fm), layout.from_oracle(rm)) < 1e-12
    # D U cancels to ~1e-14 for this nearly solenoidal field: compare against
    # the size of its terms |U| / dx, not against its own tiny maximum
    scale = np.abs(U).max() / min(a.dx.min() for a in G.ax)
    assert np.abs(host(Fd) - rd.ravel()).max() < 1e-14 * scale


@pytest.mark.parametrize("nz,ny,nx,kind", SHAPES)
def test_pressure_solve(fv, nz, ny, nx, kind):
    g, G, shape, U, v = setup(fv, nz, ny, nx, kind)
    r = ofv.divergence(G, layout.to_oracle(v, shape))       # compatible rhs
    ref = poisson.TPF(G).solve(r).ravel()
    phi = torch.empty(g.n_cell, dtype=torch.float64, device="cuda")
    fv.fv_pressure_solve(g, dev(r.ravel()), phi, "fp64")
    assert relerr(host(phi), ref) < 1e-10
    fv.fv_pressure_solve(g, dev(r.ravel()), phi, "mixed")
    assert relerr(host(phi), ref) < 1e-4


# the largest planes the fused tensor-core transforms take (112 x 112), and a
# plane just beyond (x = 120: shared memory too small), which falls back to the
# unfused transforms
@pytest.mark.parametrize("nz,ny,nx", [(8, 112, 112), (16, 24, 120)])
def test_simple_krylov_vector_fused_limits(fv, nz, ny, nx):
    g, G, shape, U, v = setup(fv, nz, ny, nx, "cosine")
    ref_v, _ = simple.krylov_vector(G, poisson.TPF(G), layout.to_oracle(U, shape),
                                    layout.to_oracle(v, shape), 700.0)
    out = torch.empty(g.n_vel, dtype=torch.float64, device="cuda")
    st = fv.simple_krylov_solve(g, dev(U), dev(v), out, None, eps=1e-12, prec="mixed")
    assert relerr(host(out), layout.from_oracle(ref_v)) < 2e-5
    assert st["passes"] <= 4


@pytest.mark.parametrize("nz,ny,nx,kind", SHAPES)
@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_simple_krylov_vector(fv, nz, ny, nx, kind, prec):
    g, G, shape, U, v = setup(fv, nz, ny, nx, kind)
    T = poisson.TPF(G)
    ref_v, ref_p = simple.krylov_vector(G, T, layout.to_oracle(U, shape), layout.to_oracle(v, shape), 700.0)
    out = torch.empty(g.n_vel, dtype=torch.float64, device="cuda")
    p = torch.empty(g.n_cell, dtype=torch.float64, device="cuda")
    st = fv.simple_krylov_solve(g, dev(U), dev(v), out, p, eps=1e-12, prec=prec)
    got = host(out)
    tol = {"fp64": 1e-10, "ff": 1e-10, "mixed": 2e-5}[prec]
    assert relerr(got, layout.from_oracle(ref_v)) < tol
    assert relerr(host(p), ref_p.ravel()) < {"fp64": 1e-9, "ff": 1e-6, "mixed": 1e-4}[prec]
    # the divergence of the result vanishes to round-off (Eq. 9)
    div = ofv.divergence(G, layout.to_oracle(got, shape))
    scale = np.abs(got).max() / min(a.dx.min() for a in G.ax)
    assert np.abs(div).max() < 1e-12 * scale
    assert st["passes"] <= (2 if prec == "fp64" else 4)
    for c, (a, b) in enumerate(((0, 0), (1, 0), (2, 0))):       # walls stay zero
        q = got.reshape(3, *shape)[c]
        assert np.all(np.take(q, 0, axis=2 - c) == 0)


def test_shifted_operator_and_relaxation(fv):
    g, G, shape, U, v = setup(fv, 10, 9, 12, "cosine")
    T = poisson.TPF(G)
    ref, _ = simple.shifted_operator(G, T, layout.to_oracle(U, shape), layout.to_oracle(v, shape), 700.0, 10.0)
    out = torch.empty(g.n_vel, dtype=torch.float64, device="cuda")
    st = fv.simple_krylov_solve(g, dev(U), dev(v), out, None, eps=1e-12, sigma=10.0)
    assert relerr(host(out), layout.from_oracle(ref)) < 1e-10
    # under-relaxed loop: same fixed point, more passes (omega only scales phi)
    ref2, _ = simple.krylov_vector(G, T, layout.to_oracle(U, shape), layout.to_oracle(v, shape), 700.0)
    st = fv.simple_krylov_solve(g, dev(U), dev(v), out, None, eps=1e-12, omega=0.6, prec="mixed")
    assert relerr(host(out), layout.from_oracle(ref2)) < 2e-5
    assert st["passes"] > 5


def test_weighted_dot(fv):
    g, G, shape, U, v = setup(fv, 8, 9, 10, "cosine")
    W = ofv.pack(ofv.weights(G))
    ref = float(np.sum(W * ofv.pack(layout.to_oracle(U, shape)) * ofv.pack(layout.to_oracle(v, shape))))
    assert abs(fv.fv_dot_w(g, dev(U), dev(v)) - ref) < 1e-12 * abs(ref) + 1e-14


def test_invalid_arguments(fv):
    g, G, shape, U, v = setup(fv, 5, 5, 5, "cosine")
    out = torch.empty(g.n_vel, dtype=torch.float64, device="cuda")
    t = dev(U)
    with pytest.raises(fv.FvError):
        fv.simple_krylov_solve(g, t, t, t)                 # v_in aliases v_out
    with pytest.raises(fv.FvError):
        fv.simple_krylov_solve(g, t, dev(v), out, omega=1.5)
    with pytest.raises(fv.FvError):
        fv.arnoldi_leading(g, t, dev(v), m=5, nev=5)
    with pytest.raises(ValueError):
        fv.ns_jacvec(g, t, dev(v[:-1]), out)


def _oracle_newton(n, re, alpha, kind="cosine"):
    G = og.Grid(n, n, n, kind)
    T = poisson.TPF(G)
    U, P, h = krylov.newton(G, T, re, ofv.lid_velocity(alpha))
    return G, T, U, P


@pytest.mark.parametrize("n,re,alpha", [(6, 100.0, 0.0), (8, 300.0, np.pi / 4)])
def test_newton_small(fv, n, re, alpha):
    G, T, Uo, Po = _oracle_newton(n, re, alpha)
    g = fv.Grid(n, n, n, "cosine", alpha=alpha, re=re)
    U = torch.zeros(g.n_vel, dtype=torch.float64, device="cuda")
    P = torch.zeros(g.n_cell, dtype=torch.float64, device="cuda")
    st = fv.newton_steady(g, U, P, tol=1e-10)
    ref = layout.from_oracle(Uo)
    assert relerr(host(U), ref) < 1e-9          # steady velocity, max-rel 1e-9
    assert relerr(host(P), Po.ravel()) < 1e-8
    assert st["res_final"] < 1e-10


@pytest.mark.parametrize("n,re,alpha", [(6, 100.0, 0.0), (7, 300.0, np.pi / 4)])
@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_arnoldi_small_vs_dense(fv, n, re, alpha, prec):
    G, T, Uo, Po = _oracle_newton(n, re, alpha)
    ref = dense.reduced_spectrum(G, Uo, re)[:5]
    g = fv.Grid(n, n, n, "cosine", alpha=alpha, re=re)
    U = dev(layout.from_oracle(Uo))
    v0 = dev(synth.gaussian_velocity((n, n, n), 1))
    evec = torch.empty(2 * g.n_vel, dtype=torch.float64, device="cuda")
    lam, info = fv.arnoldi_leading(g, U, v0, m=30, nev=5, evec=evec, prec=prec)
    lam = np.array(lam)
    tol = 1e-4 if prec == "mixed" else 1e-7
    np.testing.assert_allclose(lam.real, ref.real, atol=tol * abs(ref[0]))
    np.testing.assert_allclose(np.abs(lam.imag), np.abs(ref.imag), atol=tol * abs(ref[0]))
    # leading eigenvector: eigen-residual through the oracle operator
    e = host(evec)
    x = layout.to_oracle(e[:g.n_vel], (n, n, n)), layout.to_oracle(e[g.n_vel:], (n, n, n))
    Ar = ofv.pack(simple.krylov_vector(G, T, Uo, x[0], re)[0])
    Ai = ofv.pack(simple.krylov_vector(G, T, Uo, x[1], re)[0])
    z = ofv.pack(x[0]) + 1j * ofv.pack(x[1])
    W = ofv.pack(ofv.weights(G))
    res = np.sqrt(np.sum(W * np.abs(Ar + 1j * Ai - lam[0] * z) ** 2))
    assert res < (1e-3 if prec == "mixed" else 1e-7) * abs(lam[0])
    assert abs(np.sum(W * np.abs(z) ** 2) - 1.0) < 1e-10


def test_mixed_async_graph_matches_sync(fv):
    # the graph path without host synchronisation gives the same fields
    g, G, shape, U, v = setup(fv, 24, 26, 28, "cosine")
    a = torch.empty(g.n_vel, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    tU, tv = dev(U), dev(v)
    st = fv.simple_krylov_solve(g, tU, tv, a, None, eps=1e-8, prec="mixed")
    for _ in range(3):
        fv.simple_krylov_solve(g, tU, tv, b, None, eps=1e-8, prec="mixed", async_=True)
    assert np.array_equal(host(a), host(b))
    assert 2 <= st["passes"] <= 4
    # a different right-hand side through the same captured graph
    v2 = dev(synth.gaussian_velocity(shape, 9))
    fv.simple_krylov_solve(g, tU, v2, b, None, eps=1e-8, prec="mixed", async_=True)
    T = poisson.TPF(G)
    ref, _ = simple.krylov_vector(G, T, layout.to_oracle(U, shape), layout.to_oracle(host(v2), shape), 700.0)
    assert relerr(host(b), layout.from_oracle(ref)) < 2e-5


def test_host_driven_loop_matches_graph(fv, monkeypatch):
    # FVNS_NO_GRAPH=1 selects the host-driven mixed loop (same kernels, one
    # synchronisation per pass); both must give the same fields, also when
    # called without statistics
    g1, G, shape, U, v = setup(fv, 12, 10, 14, "cosine")
    monkeypatch.setenv("FVNS_NO_GRAPH", "1")
    g2 = fv.Grid(14, 10, 12, "cosine", alpha=0.3, re=700.0)
    a = torch.empty(g1.n_vel, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    fv.simple_krylov_solve(g1, dev(U), dev(v), a, None, eps=1e-10, prec="mixed")
    fv.simple_krylov_solve(g2, dev(U), dev(v), b, None, eps=1e-10, prec="mixed", async_=True)
    assert relerr(host(b), host(a)) < 1e-9


@pytest.mark.parametrize("prec", ["mixed", "ff"])
def test_set_re_reaches_the_captured_graph(fv, prec):
    """An evaluation after fv_grid_set_re uses the new Re: the same as a grid
    created at that Re (the captured graph held 1/Re as a kernel argument)."""
    n = 12
    U = dev(synth.vortex_base_flow((n, n, n), "cosine", 0.0))
    v = dev(synth.gaussian_velocity((n, n, n), 3))
    g1 = fv.Grid(n, n, n, "cosine", alpha=0.0, re=200.0)
    o1 = torch.empty_like(v)
    fv.simple_krylov_solve(g1, U, v, o1, eps=1e-8, prec=prec, sigma=10.0)   # captures at Re 200
    g1.set_re(1000.0)
    fv.simple_krylov_solve(g1, U, v, o1, eps=1e-8, prec=prec, sigma=10.0)
    g2 = fv.Grid(n, n, n, "cosine", alpha=0.0, re=1000.0)
    o2 = torch.empty_like(v)
    fv.simple_krylov_solve(g2, U, v, o2, eps=1e-8, prec=prec, sigma=10.0)
    torch.cuda.synchronize()
    assert relerr(host(o1), host(o2)) < 1e-12


def test_ff_newton_continuation_is_quadratic(fv):
    """Newton with float-float Krylov vectors along Re 200 -> 600 on 12^3:
    every Re converges to 1e-10 within 8 steps (a stale 1/Re in the captured
    evaluation graph made it linear, ratio ~0.5 per step)."""
    n = 12
    g = fv.Grid(n, n, n, "cosine", alpha=0.0, re=200.0)
    U = torch.zeros(g.n_vel, dtype=torch.float64, device="cuda")
    P = torch.zeros(g.n_cell, dtype=torch.float64, device="cuda")
    for re in (200.0, 400.0, 600.0):
        g.set_re(re)
        st = fv.newton_steady(g, U, P, tol=1e-10, prec="ff", max_newton=8)
        assert st["res_final"] < 1e-10, (re, st["res_hist"])


@pytest.mark.parametrize("prec", ["mixed", "ff"])
def test_nan_in_operator_is_reported(fv, prec):
    """Krylov drivers launch the evaluation graphs without reading their status
    back; a NaN in the base flow must still end Arnoldi and Newton with an
    error (the graph's sticky status, or the NaN reaching a dot product)."""
    n = 8
    g = fv.Grid(n, n, n, "cosine", alpha=0.0, re=300.0)
    U = dev(synth.vortex_base_flow((n, n, n), "cosine", 0.0))
    U[g.n_vel // 2] = float("nan")
    v0 = dev(synth.gaussian_velocity((n, n, n), 1))
    with pytest.raises(fv.FvError):
        fv.arnoldi_leading(g, U, v0, m=10, nev=2, prec=prec, max_restarts=2)
    P = torch.zeros(g.n_cell, dtype=torch.float64, device="cuda")
    with pytest.raises(fv.FvError):
        fv.newton_steady(g, U, P, tol=1e-10, prec=prec, max_newton=2)
    # the grid stays usable
    U2 = dev(synth.vortex_base_flow((n, n, n), "cosine", 0.0))
    lam, _ = fv.arnoldi_leading(g, U2, v0, m=20, nev=2, prec=prec, tol=1e-6)
    assert np.isfinite(np.array(lam)).all()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_registered_base_flow(fv, prec):
    """fv_grid_set_base: evaluations with U = NULL use the registered base
    flow and give the same vector as passing U (the same rounding / split of
    U, made once instead of per evaluation)."""
    g, G, shape, U, v = setup(fv, 14, 13, 15, "cosine")
    tU, tv = dev(U), dev(v)
    a = torch.empty(g.n_vel, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    fv.simple_krylov_solve(g, tU, tv, a, None, eps=1e-10, prec=prec, sigma=10.0)
    g.set_base(tU)
    fv.simple_krylov_solve(g, None, tv, b, None, eps=1e-10, prec=prec, sigma=10.0)
    assert np.array_equal(host(a), host(b))
    # no registered base on a fresh grid: U = NULL is refused
    g2 = fv.Grid(15, 13, 14, "cosine", alpha=0.3, re=700.0)
    with pytest.raises(fv.FvError):
        fv.simple_krylov_solve(g2, None, tv, b, None, eps=1e-10, prec=prec)
