"""GPU parity at the full sizes of the benchmark configurations, element by
element against the FP64 oracle's plain definition of the Krylov vector
(Eqs. 8-10: J.v of Eq. 10, then one exact projection).

* 100^3 cosine grid, lid parallel to the x sidewall, Re 1900: the benchmark
  workload, in the launch configuration bench.py times (asynchronous graph
  evaluation, stop test 1e-8) -- the fused tensor-core pressure transforms;
* 150^3 cosine grid, diagonal lid, Re 2300 (the 150^3 configuration) and
  256^3 cosine grid, lid parallel to the x sidewall, Re 1900 (the largest
  grid of the learned-guess configuration) -- planes too large for one
  block's shared memory, so the unfused transforms.

Tolerances (max |gpu - oracle| / max |oracle|): mixed form 2e-5 (float32
J.v; the loop itself converges to float-float accuracy), float-float form
1e-10; pressure 1e-4 / 1e-6.  The divergence of every result vanishes to
round-off (Eq. 9)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
import layout  # noqa: E402
from oracle import fv as ofv, grid as og, poisson, simple  # noqa: E402

CASES = [(100, 0.0, 1900.0), (150, np.pi / 4, 2300.0), (256, 0.0, 1900.0)]
TOL_V = {"mixed": 2e-5, "ff": 1e-10}
TOL_P = {"mixed": 1e-4, "ff": 1e-6}


@pytest.fixture(scope="module")
def fv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1704_08521_gb300 as m
    return m


def relerr(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


_ORACLE = {}


def oracle_case(n, alpha, re, seed):
    key = (n, alpha, re, seed)
    if key not in _ORACLE:
        _ORACLE.clear()                      # one large case held at a time
        shape = (n, n, n)
        G = og.Grid(n, n, n, "cosine")
        U = synth.vortex_base_flow(shape, "cosine", alpha)
        v = synth.gaussian_velocity(shape, seed)
        ref_v, ref_p = simple.krylov_vector(G, poisson.TPF(G), layout.to_oracle(U, shape),
                                            layout.to_oracle(v, shape), re)
        _ORACLE[key] = (G, U, v, layout.from_oracle(ref_v), ref_p.ravel())
    return _ORACLE[key]


@pytest.mark.parametrize("n,alpha,re", CASES)
@pytest.mark.parametrize("prec", ["mixed", "ff"])
def test_krylov_vector_full_size(fv, n, alpha, re, prec):
    G, U, v, ref_v, ref_p = oracle_case(n, alpha, re, 1)
    g = fv.Grid(n, n, n, "cosine", alpha=alpha, re=re)
    tU = torch.tensor(U, device="cuda")
    tv = torch.tensor(v, device="cuda")
    out = torch.empty(g.n_vel, dtype=torch.float64, device="cuda")
    p = torch.empty(g.n_cell, dtype=torch.float64, device="cuda")
    st = fv.simple_krylov_solve(g, tU, tv, out, p, eps=1e-8, prec=prec)   # statistics
    assert 2 <= st["passes"] <= 4
    out.zero_()
    fv.simple_krylov_solve(g, tU, tv, out, p, eps=1e-8, prec=prec, async_=True)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert relerr(got, ref_v) < TOL_V[prec]
    assert relerr(p.cpu().numpy(), ref_p) < TOL_P[prec]
    shape = (n, n, n)
    div = ofv.divergence(G, layout.to_oracle(got, shape))
    scale = np.abs(got).max() / min(a.dx.min() for a in G.ax)
    assert np.abs(div).max() < 1e-12 * scale
    g.close()
