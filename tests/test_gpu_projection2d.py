"""Divergence-free projections onto coordinate planes and their vector
potentials (Section 4, Eqs. 11-17) on the GPU against the oracle, element by
element, on ragged grids of all three maps and on the stored 16^3 steady
state of configuration 1 (the flow Section 4 visualises).  Tolerance 1e-10
of the largest entry (float64 transforms)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
import layout  # noqa: E402
from oracle import grid as og, projection2d as pr  # noqa: E402

GOLD = os.path.join(os.path.dirname(__file__), "golden", "config1_16.npz")


@pytest.fixture(scope="module")
def fv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1704_08521_gb300 as m
    return m


def _check(fv, g, G, v, shape, plane):
    tv = torch.tensor(v, device="cuda")
    vp = torch.empty_like(tv)
    a, c, b = pr.PLANES[plane]
    dims = [shape[2], shape[1], shape[0]]
    dims[a] += 1
    dims[c] += 1
    psi = torch.empty(dims[0] * dims[1] * dims[2], dtype=torch.float64, device="cuda")
    fv.fv_plane_projection(g, tv, plane, vp, psi)
    torch.cuda.synchronize()
    ref_v, _ = pr.project(G, layout.to_oracle(v, shape), plane)
    ref_psi = pr.potential(G, ref_v, plane)
    got = vp.cpu().numpy()
    ref = layout.from_oracle(ref_v)
    assert np.abs(got - ref).max() < 1e-10 * np.abs(ref).max()
    gp = psi.cpu().numpy().reshape(dims[2], dims[1], dims[0])
    assert np.abs(gp - ref_psi).max() < 1e-10 * np.abs(ref_psi).max()


@pytest.mark.parametrize("plane", ["xz", "yz", "xy"])
@pytest.mark.parametrize("nz,ny,nx,kind", [(5, 6, 7, "cosine"), (9, 11, 13, "sine0975"),
                                          (33, 20, 17, "cosine")])
def test_plane_projection_matches_oracle(fv, nz, ny, nx, kind, plane):
    shape = (nz, ny, nx)
    g = fv.Grid(nx, ny, nz, kind, alpha=0.0, re=100.0)
    G = og.Grid(nx, ny, nz, kind)
    _check(fv, g, G, synth.gaussian_velocity(shape, 4), shape, plane)


@pytest.mark.parametrize("plane", ["xz", "yz", "xy"])
def test_plane_projection_of_the_config1_steady_state(fv, plane):
    gold = np.load(GOLD)
    n = 16
    g = fv.Grid(n, n, n, "cosine", alpha=0.0, re=1000.0)
    G = og.Grid(n, n, n, "cosine")
    _check(fv, g, G, gold["U"], (n, n, n), plane)


def test_plane_projection_rejects_bad_arguments(fv):
    g = fv.Grid(6, 6, 6, "cosine")
    v = torch.zeros(g.n_vel, dtype=torch.float64, device="cuda")
    with pytest.raises(fv.FvError):
        fv.fv_plane_projection(g, v, 3, torch.empty_like(v))
    with pytest.raises(fv.FvError):
        fv.fv_plane_projection(g, v, "xz", v)
