"""Error paths on the GPU, made on the host (no device fault is caused).

* Timeout: a tensor-core pressure transform whose bounded mbarrier wait gives
  up sets the grid's sticky timeout word.  fv_debug_inject_status sets that
  word from the host exactly as such a kernel would; the next synchronised
  mixed / float-float evaluation, and a Krylov driver at its next status
  check, must report FV_ETIMEOUT (distinct from FV_ENAN), and the grid must
  work again afterwards.
* Iteration caps: a SIMPLE loop capped at one pass, and Newton capped at one
  step, return FV_ENOCONV with their statistics filled in."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402

FV_ENOCONV, FV_ENAN, FV_ETIMEOUT = 4, 5, 6


@pytest.fixture(scope="module")
def fv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1704_08521_gb300 as m
    return m


def fields(n, alpha=0.0):
    U = torch.tensor(synth.vortex_base_flow((n, n, n), "cosine", alpha), device="cuda")
    v = torch.tensor(synth.gaussian_velocity((n, n, n), 2), device="cuda")
    return U, v


@pytest.mark.parametrize("prec", ["mixed", "ff"])
def test_injected_timeout_is_reported_by_an_evaluation(fv, prec):
    n = 16
    g = fv.Grid(n, n, n, "cosine", alpha=0.0, re=500.0)
    U, v = fields(n)
    out = torch.empty_like(v)
    fv.simple_krylov_solve(g, U, v, out, eps=1e-8, prec=prec)        # captures the graph
    ref = out.clone()
    fv.fv_debug_inject_status(g, FV_ETIMEOUT)
    with pytest.raises(fv.FvError) as e:
        fv.simple_krylov_solve(g, U, v, out, eps=1e-8, prec=prec)
    assert e.value.status == FV_ETIMEOUT
    # reported once: the grid works again and gives the same vector
    st = fv.simple_krylov_solve(g, U, v, out, eps=1e-8, prec=prec)
    assert 2 <= st["passes"] <= 4
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


def test_injected_timeout_ends_arnoldi(fv):
    n = 10
    g = fv.Grid(n, n, n, "cosine", alpha=0.0, re=300.0)
    U, v = fields(n)
    fv.fv_debug_inject_status(g, FV_ETIMEOUT)
    with pytest.raises(fv.FvError) as e:
        fv.arnoldi_leading(g, U, v, m=12, nev=2, prec="mixed", max_restarts=3)
    assert e.value.status == FV_ETIMEOUT
    lam, _ = fv.arnoldi_leading(g, U, v, m=20, nev=2, prec="mixed", tol=1e-6)
    assert np.isfinite(np.array(lam)).all()


def test_injected_timeout_host_driven_loop(fv, monkeypatch):
    monkeypatch.setenv("FVNS_NO_GRAPH", "1")
    n = 12
    g = fv.Grid(n, n, n, "cosine", alpha=0.0, re=500.0)
    U, v = fields(n)
    out = torch.empty_like(v)
    fv.fv_debug_inject_status(g, FV_ETIMEOUT)
    with pytest.raises(fv.FvError) as e:
        fv.simple_krylov_solve(g, U, v, out, eps=1e-8, prec="mixed")
    assert e.value.status == FV_ETIMEOUT


def test_only_timeouts_can_be_injected(fv):
    g = fv.Grid(6, 6, 6, "cosine")
    with pytest.raises(fv.FvError) as e:
        fv.fv_debug_inject_status(g, FV_ENAN)
    assert e.value.status == 1


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_pass_cap_reports_enoconv_with_stats(fv, prec):
    n = 12
    g = fv.Grid(n, n, n, "cosine", alpha=0.0, re=500.0)
    U, v = fields(n)
    out = torch.empty_like(v)
    o = fv.fv_simple_opts(1e-14, 1, fv.PRECS[prec], 1.0, 0.0, 0)
    s = fv.fv_simple_stats()
    st = fv.lib.simple_krylov_solve(g.handle, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), None, ctypes.byref(o), ctypes.byref(s))
    assert st == FV_ENOCONV
    assert s.passes == 1 and s.phi_first > 0 and s.phi_last == s.phi_first
    assert b"max_pass" in fv.lib.fv_last_error()


def test_newton_step_cap_reports_enoconv_with_stats(fv):
    n = 8
    g = fv.Grid(n, n, n, "cosine", alpha=0.0, re=300.0)
    U = torch.zeros(g.n_vel, dtype=torch.float64, device="cuda")
    P = torch.zeros(g.n_cell, dtype=torch.float64, device="cuda")
    st = fv.newton_steady(g, U, P, tol=1e-12, max_newton=1, raise_on_fail=False)
    assert st["status"] == FV_ENOCONV
    assert st["iterations"] == 1 and st["res_hist"][0] > 0 and st["res_final"] < st["res_hist"][0]
