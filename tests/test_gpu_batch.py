"""Batched instances (one graph launch, persistent work-queue J.v, concurrent
SIMPLE loops) against the single-instance evaluation and the oracle.

Configuration 4 shape: 12 instances, grids {48, 64, 80, 96}^3 x Re {1700,
1900, 2100}, lid parallel to the x sidewall for even instance index and to
the diagonal plane for odd; Philox Gaussian right-hand sides of seed
100 + instance."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
import layout  # noqa: E402
from oracle import grid as og, poisson, simple  # noqa: E402


@pytest.fixture(scope="module")
def fv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1704_08521_gb300 as m
    return m


def _instances(sizes, res):
    out = []
    for n in sizes:
        for re in res:
            i = len(out)
            out.append((n, re, 0.0 if i % 2 == 0 else math.pi / 4, 100 + i))
    return out


def _run(fv, inst, sigma, tmp_path):
    grids, U, X, O, R = [], [], [], [], []
    for n, re, alpha, seed in inst:
        shape = (n, n, n) if isinstance(n, int) else n
        nz, ny, nx = shape
        g = fv.Grid(nx, ny, nz, "cosine", alpha=alpha, re=re)
        grids.append(g)
        U.append(torch.tensor(synth.vortex_base_flow(shape, "cosine", alpha), device="cuda"))
        X.append(torch.tensor(synth.gaussian_velocity(shape, seed), device="cuda"))
        O.append(torch.empty(g.n_vel, dtype=torch.float64, device="cuda"))
        R.append(torch.empty(g.n_vel, dtype=torch.float64, device="cuda"))
    b = fv.Batch(grids)
    tune = b.autotune(cache=str(tmp_path / "tune.json"))
    assert tune["planes"] in (1, 2, 4, 8)
    for _ in range(2):                                    # twice: graph reuse
        passes = b.krylov(U, X, O, eps=1e-8, sigma=sigma)
    assert all(2 <= p <= 4 for p in passes)
    for i, g in enumerate(grids):                         # single-instance reference
        fv.simple_krylov_solve(g, U[i], X[i], R[i], None, eps=1e-8, prec="mixed", sigma=sigma)
    torch.cuda.synchronize()
    return grids, U, X, O, R


def test_batch_small_uneven(fv, tmp_path):
    inst = [((8, 8, 8), 500.0, 0.0, 1), ((11, 9, 10), 700.0, math.pi / 4, 2),
            ((12, 12, 12), 900.0, 0.0, 3), ((8, 7, 6), 1100.0, math.pi / 4, 4)]
    grids, U, X, O, R = _run(fv, inst, 10.0, tmp_path)
    for i, (shape, re, alpha, seed) in enumerate(inst):
        a, r = O[i].cpu().numpy(), R[i].cpu().numpy()
        assert np.abs(a - r).max() <= 1e-6 * np.abs(r).max()
        nz, ny, nx = shape
        G = og.Grid(nx, ny, nz, "cosine")
        ref, _ = simple.shifted_operator(G, poisson.TPF(G), layout.to_oracle(U[i].cpu().numpy(), shape),
                                         layout.to_oracle(X[i].cpu().numpy(), shape), re, 10.0)
        ref = layout.from_oracle(ref)
        assert np.abs(a - ref).max() <= 2e-5 * np.abs(ref).max()


def test_batch_config4(fv, tmp_path):
    inst = _instances([48, 64, 80, 96], [1700.0, 1900.0, 2100.0])
    grids, U, X, O, R = _run(fv, inst, 0.0, tmp_path)
    for i in range(len(inst)):
        a, r = O[i].cpu().numpy(), R[i].cpu().numpy()
        assert np.abs(a - r).max() <= 1e-6 * np.abs(r).max(), i
    # one full instance against the oracle (96^3, Re 1900, diagonal lid)
    n, re, alpha, seed = inst[10]
    G = og.Grid(n, n, n, "cosine")
    shape = (n, n, n)
    ref, _ = simple.krylov_vector(G, poisson.TPF(G), layout.to_oracle(U[10].cpu().numpy(), shape),
                                  layout.to_oracle(X[10].cpu().numpy(), shape), re)
    ref = layout.from_oracle(ref)
    a = O[10].cpu().numpy()
    assert np.abs(a - ref).max() <= 2e-5 * np.abs(ref).max()


def test_batch_follows_set_re(fv):
    """fv_grid_set_re between batch calls reaches the batched J.v: after the
    change the batch matches single-instance evaluations at the new Re."""
    shapes = [(12, 12, 12), (16, 12, 8)]
    grids, U, X, O, R = [], [], [], [], []
    for i, shape in enumerate(shapes):
        nz, ny, nx = shape
        g = fv.Grid(nx, ny, nz, "cosine", alpha=0.0, re=300.0)
        grids.append(g)
        U.append(torch.tensor(synth.vortex_base_flow(shape, "cosine", 0.0), device="cuda"))
        X.append(torch.tensor(synth.gaussian_velocity(shape, 7 + i), device="cuda"))
        O.append(torch.empty(g.n_vel, dtype=torch.float64, device="cuda"))
        R.append(torch.empty(g.n_vel, dtype=torch.float64, device="cuda"))
    b = fv.Batch(grids)
    b.krylov(U, X, O, eps=1e-8, sigma=0.0)                # captured at Re 300
    for g in grids:
        g.set_re(1500.0)
    b.krylov(U, X, O, eps=1e-8, sigma=0.0)
    for i, shape in enumerate(shapes):
        nz, ny, nx = shape
        g2 = fv.Grid(nx, ny, nz, "cosine", alpha=0.0, re=1500.0)
        fv.simple_krylov_solve(g2, U[i], X[i], R[i], None, eps=1e-8, prec="mixed")
    torch.cuda.synchronize()
    for o, r in zip(O, R):
        o, r = o.cpu().numpy(), r.cpu().numpy()
        assert np.abs(o - r).max() <= 1e-6 * np.abs(r).max()
