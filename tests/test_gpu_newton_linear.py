"""Newton corrections by BiCGstab(2) and by Section 3's hand-off (GMRES(m)
restarted until it saturates, then BiCGstab(2) from its last approximation)
on the device, against the oracle's Newton with the same linear solver.

Tolerances: steady velocity max-rel 1e-9 and pressure 1e-8 (as for the
GMRES Newton); in FP64 the device follows the oracle's Newton path, so the
step count is the same and the residual after the first correction agrees
to 1e-5 relative (both linear solves stop at 1e-8 of ||F||, possibly one
BiCGstab cycle apart)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import layout  # noqa: E402
from oracle import fv as ofv, grid as og, poisson, krylov  # noqa: E402

GOLD = os.path.join(os.path.dirname(__file__), "golden", "config1_16.npz")


@pytest.fixture(scope="module")
def fv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1704_08521_gb300 as m
    return m


def relerr(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


# gmres_sat = 1e-12 with m = 10: every GMRES(10) cycle that does not
# converge counts as saturated, so each correction hands off after two cycles
CASES = [("bicgstab", 100, 0.5), ("gmres+bicgstab", 10, 1e-12)]


@pytest.mark.parametrize("linear,m,sat", CASES)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_newton_small_matches_oracle(fv, linear, m, sat, prec):
    n, re, alpha = 8, 300.0, np.pi / 4
    G = og.Grid(n, n, n, "cosine")
    Uo, Po, ho = krylov.newton(G, poisson.TPF(G), re, ofv.lid_velocity(alpha), tol=1e-10,
                               m=m, linear=linear, gmres_sat=sat)
    g = fv.Grid(n, n, n, "cosine", alpha=alpha, re=re)
    U = torch.zeros(g.n_vel, dtype=torch.float64, device="cuda")
    P = torch.zeros(g.n_cell, dtype=torch.float64, device="cuda")
    st = fv.newton_steady(g, U, P, tol=1e-10, gmres_m=m, prec=prec, linear=linear, gmres_sat=sat)
    torch.cuda.synchronize()
    assert relerr(U.cpu().numpy(), layout.from_oracle(Uo)) < 1e-9
    assert relerr(P.cpu().numpy(), Po.ravel()) < 1e-8
    assert st["res_final"] < 1e-10
    assert st["bicgstab_total"] > 0
    if linear == "bicgstab":
        assert st["gmres_total"] == 0
    else:
        assert st["gmres_total"] > 0
    if prec == "fp64":
        assert st["iterations"] == len(ho) - 1, (st["res_hist"], ho)
        np.testing.assert_allclose(st["res_hist"][:2], ho[:2], rtol=1e-5)


@pytest.mark.parametrize("linear", ["bicgstab", "gmres+bicgstab"])
def test_config1_continuation(fv, linear):
    """16^3, Re 200 -> 1000 from rest (the stored oracle steady state)."""
    gold = np.load(GOLD)
    g = fv.Grid(16, 16, 16, "cosine", alpha=0.0, re=200.0)
    U = torch.zeros(g.n_vel, dtype=torch.float64, device="cuda")
    P = torch.zeros(g.n_cell, dtype=torch.float64, device="cuda")
    tot = [0, 0]
    for re in (200.0, 400.0, 600.0, 800.0, 1000.0):
        g.set_re(re)
        st = fv.newton_steady(g, U, P, tol=1e-10, prec="mixed", linear=linear, gmres_m=30)
        tot[0] += st["gmres_total"]
        tot[1] += st["bicgstab_total"]
    torch.cuda.synchronize()
    ref = gold["U"]
    assert np.abs(U.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-9
    print(f"\n16^3 continuation, {linear}: GMRES {tot[0]}, BiCGstab(2) {tot[1]} products")


def test_bad_linear_option(fv):
    g = fv.Grid(6, 6, 6, "cosine", re=100.0)
    U = torch.zeros(g.n_vel, dtype=torch.float64, device="cuda")
    P = torch.zeros(g.n_cell, dtype=torch.float64, device="cuda")
    with pytest.raises(fv.FvError):
        fv.newton_steady(g, U, P, linear=3)


@pytest.mark.parametrize("prec", ["ff", "mixed"])
def test_preconditioned_newton_same_steady_state(fv, prec):
    """Newton with the Stokes-type right preconditioner (flexible GMRES):
    the 16^3 continuation Re 200 -> 1000 from rest reaches the stored oracle
    steady state to the same 1e-9, with fewer operator products than the
    unpreconditioned GMRES(30) Newton (the correction does not depend on how
    the linear system is solved)."""
    gold = np.load(GOLD)
    res = {}
    for pre in (0, 1):
        g = fv.Grid(16, 16, 16, "cosine", alpha=0.0, re=200.0)
        U = torch.zeros(g.n_vel, dtype=torch.float64, device="cuda")
        P = torch.zeros(g.n_cell, dtype=torch.float64, device="cuda")
        tot = 0
        for re in (200.0, 400.0, 600.0, 800.0, 1000.0):
            g.set_re(re)
            st = fv.newton_steady(g, U, P, tol=1e-10, prec=prec, linear="gmres", gmres_m=30,
                                  precond=pre)
            tot += st["gmres_total"]
        torch.cuda.synchronize()
        ref = gold["U"]
        assert np.abs(U.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-9, pre
        res[pre] = tot
    print(f"\n16^3 continuation, {prec}: GMRES(30) products {res[0]}, preconditioned {res[1]}")
    assert res[1] < res[0] / 2


@pytest.mark.parametrize("linear", ["bicgstab", "gmres+bicgstab"])
def test_preconditioned_bicgstab_same_steady_state(fv, linear):
    """The right-preconditioned BiCGstab(2) (alone, and as the hand-off
    after a saturated flexible GMRES(10), which may not saturate on this
    small grid) reaches the stored oracle steady state of the 16^3
    continuation Re 200 -> 1000 to 1e-9."""
    gold = np.load(GOLD)
    g = fv.Grid(16, 16, 16, "cosine", alpha=0.0, re=200.0)
    U = torch.zeros(g.n_vel, dtype=torch.float64, device="cuda")
    P = torch.zeros(g.n_cell, dtype=torch.float64, device="cuda")
    tot = [0, 0]
    for re in (200.0, 400.0, 600.0, 800.0, 1000.0):
        g.set_re(re)
        st = fv.newton_steady(g, U, P, tol=1e-10, prec="ff", linear=linear, gmres_m=10,
                              gmres_sat=0.9, precond=1)
        tot[0] += st["gmres_total"]
        tot[1] += st["bicgstab_total"]
    torch.cuda.synchronize()
    ref = gold["U"]
    assert np.abs(U.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-9
    if linear == "bicgstab":
        assert tot[0] == 0 and tot[1] > 0
    print(f"\n16^3 continuation, preconditioned {linear}: GMRES {tot[0]}, BiCGstab(2) {tot[1]}")


def test_bad_precond_option(fv):
    g = fv.Grid(6, 6, 6, "cosine", re=100.0)
    U = torch.zeros(g.n_vel, dtype=torch.float64, device="cuda")
    P = torch.zeros(g.n_cell, dtype=torch.float64, device="cuda")
    with pytest.raises(fv.FvError):
        fv.newton_steady(g, U, P, precond=2)
    with pytest.raises(fv.FvError):
        fv.newton_steady(g, U, P, precond=1, precond_sigma=-1.0)


def test_augmented_flexible_gmres_same_steady_state(fv):
    """Flexible GMRES(10) whose last two steps per cycle take the previous
    cycles' corrections (LGMRES augmentation) reaches the stored oracle
    steady state of the 16^3 continuation to 1e-9; the option is refused
    without the preconditioner or beyond 4 vectors."""
    gold = np.load(GOLD)
    g = fv.Grid(16, 16, 16, "cosine", alpha=0.0, re=200.0)
    U = torch.zeros(g.n_vel, dtype=torch.float64, device="cuda")
    P = torch.zeros(g.n_cell, dtype=torch.float64, device="cuda")
    for re in (200.0, 400.0, 600.0, 800.0, 1000.0):
        g.set_re(re)
        fv.newton_steady(g, U, P, tol=1e-10, prec="ff", linear="gmres", gmres_m=10, precond=1,
                         gmres_aug=2)
    torch.cuda.synchronize()
    ref = gold["U"]
    assert np.abs(U.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-9
    with pytest.raises(fv.FvError):
        fv.newton_steady(g, U, P, gmres_aug=2)
    with pytest.raises(fv.FvError):
        fv.newton_steady(g, U, P, precond=1, gmres_aug=5)


def test_shifted_newton_same_steady_state(fv):
    """Corrections from (A - tau I) du = F (tau = 0.1) converge to the same
    stored oracle steady state of the 16^3 continuation, to 1e-9: the shift
    changes the path, not the fixed point."""
    gold = np.load(GOLD)
    g = fv.Grid(16, 16, 16, "cosine", alpha=0.0, re=200.0)
    U = torch.zeros(g.n_vel, dtype=torch.float64, device="cuda")
    P = torch.zeros(g.n_cell, dtype=torch.float64, device="cuda")
    steps = 0
    for re in (200.0, 400.0, 600.0, 800.0, 1000.0):
        g.set_re(re)
        st = fv.newton_steady(g, U, P, tol=1e-10, prec="ff", precond=1, precond_sigma=1.0,
                              tau=0.1, max_newton=60)
        steps += st["iterations"]
    torch.cuda.synchronize()
    ref = gold["U"]
    assert np.abs(U.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-9
    with pytest.raises(fv.FvError):
        fv.newton_steady(g, U, P, tau=-1.0)
    print(f"\n16^3 continuation with tau = 0.1: {steps} Newton steps")
