"""Pins of the oracle's divergence-free projections onto coordinate planes
and their vector potentials (Section 4, Eqs. 11-17)."""
import numpy as np
import pytest

import synth
import layout
from oracle import fv, grid as og, projection2d as pr


def _field(shape, seed, kind="cosine"):
    nz, ny, nx = shape
    G = og.Grid(nx, ny, nz, kind)
    return G, layout.to_oracle(synth.gaussian_velocity(shape, seed), shape)


def _wdot(G, a, b):
    W = fv.weights(G)
    return sum(float(np.sum(W[d] * a[d] * b[d])) for d in range(3))


@pytest.mark.parametrize("plane", ["xz", "yz", "xy"])
@pytest.mark.parametrize("shape,kind", [((5, 6, 7), "cosine"), ((8, 7, 9), "sine0975"), ((6, 6, 6), "uniform")])
def test_projection_is_divergence_free_idempotent_orthogonal(plane, shape, kind):
    G, v = _field(shape, 3, kind)
    a, c, b = pr.PLANES[plane]
    vb, phi = pr.project(G, v, plane)
    scale = max(np.abs(x).max() for x in vb) / min(G.ax[d].dx.min() for d in range(3))
    assert np.abs(pr.divergence_2d(G, vb, a, c)).max() < 1e-12 * scale          # Eqs. 12-14
    assert np.abs(vb[b]).max() == 0.0                                          # Eq. 11
    vb2, _ = pr.project(G, vb, plane)
    assert max(np.abs(vb2[d] - vb[d]).max() for d in range(3)) < 1e-12 * max(np.abs(x).max() for x in vb)
    # the removed part (in-plane part of v minus vb) is W-orthogonal to vb
    q = [np.zeros_like(x) for x in v]
    for d in (a, c):
        q[d] = fv._zero_walls(v[d].copy(), d)
    rem = [q[d] - vb[d] for d in range(3)]
    assert abs(_wdot(G, rem, vb)) < 1e-12 * _wdot(G, q, q)
    # and the projection lowers the W-norm (Pythagoras)
    assert abs(_wdot(G, q, q) - _wdot(G, vb, vb) - _wdot(G, rem, rem)) < 1e-10 * _wdot(G, q, q)


def _rot_of_potential(G, psi, plane):
    """The field of Eqs. 15-17 from a corner potential (the definition written out)."""
    a, c, b = pr.PLANES[plane]
    sign = {"xz": 1.0, "yz": -1.0, "xy": -1.0}[plane]
    out = [np.zeros(G.shape_vel(d)) for d in range(3)]
    # component c: sign * d psi / d a  at c-faces, a-centres
    P = np.moveaxis(psi, [2 - a, 2 - c], [-1, -2])
    dc_ = sign * (P[..., :, 1:] - P[..., :, :-1]) / G.ax[a].dx
    oc = np.moveaxis(out[c], [2 - a, 2 - c], [-1, -2])
    oc[...] = dc_
    # component a: -sign * d psi / d c at a-faces, c-centres
    da_ = -sign * (P[..., 1:, :] - P[..., :-1, :]) / G.ax[c].dx[:, None]
    oa = np.moveaxis(out[a], [2 - a, 2 - c], [-1, -2])
    oa[...] = da_
    return [fv._zero_walls(out[d], d) for d in range(3)]


@pytest.mark.parametrize("plane", ["xz", "yz", "xy"])
def test_potential_reproduces_projection(plane):
    G, v = _field((6, 7, 8), 5)
    vb, _ = pr.project(G, v, plane)
    psi = pr.potential(G, vb, plane)
    back = _rot_of_potential(G, psi, plane)
    ref = max(np.abs(x).max() for x in vb)
    assert max(np.abs(back[d] - vb[d]).max() for d in range(3)) < 1e-12 * ref
    # the potential vanishes on the walls of every plane
    a, c, b = pr.PLANES[plane]
    P = np.moveaxis(psi, [2 - a, 2 - c], [-1, -2])
    pmax = np.abs(P).max()
    for edge in (P[..., 0, :], P[..., -1, :], P[..., :, 0], P[..., :, -1]):
        assert np.abs(edge).max() < 1e-12 * pmax


@pytest.mark.parametrize("plane", ["xz", "yz", "xy"])
def test_field_from_a_potential_is_kept(plane):
    """A field built from a random corner potential (zero on the walls) is
    already divergence-free in the planes: the projection keeps it and the
    potential is recovered."""
    G = og.Grid(7, 6, 5, "cosine")
    a, c, b = pr.PLANES[plane]
    n = [G.ax[d].n for d in range(3)]
    shp = [n[2], n[1], n[0]]
    shp[2 - a] += 1
    shp[2 - c] += 1
    rng = np.random.default_rng(11)
    psi = rng.standard_normal(shp)
    P = np.moveaxis(psi, [2 - a, 2 - c], [-1, -2])
    P[..., 0, :] = P[..., -1, :] = P[..., :, 0] = P[..., :, -1] = 0.0
    v = _rot_of_potential(G, psi, plane)
    vb, _ = pr.project(G, v, plane)
    ref = max(np.abs(x).max() for x in v)
    assert max(np.abs(vb[d] - v[d]).max() for d in range(3)) < 1e-12 * ref
    assert np.abs(pr.potential(G, vb, plane) - psi).max() < 1e-12 * np.abs(psi).max()


def test_two_dimensional_flow_is_its_own_xz_projection():
    """A flow with no y-dependence and no y-velocity, divergence-free in 3-D,
    is divergence-free in every (x, z) plane: v_1 = v."""
    G = og.Grid(8, 5, 7, "sine0975")
    a, c, b = pr.PLANES["xz"]
    n = [G.ax[d].n for d in range(3)]
    rng = np.random.default_rng(2)
    p2 = rng.standard_normal((n[2] + 1, n[0] + 1))
    p2[0, :] = p2[-1, :] = p2[:, 0] = p2[:, -1] = 0.0
    psi = np.repeat(p2[:, None, :], n[1], axis=1)
    v = _rot_of_potential(G, psi, "xz")
    assert np.abs(fv.divergence(G, v)).max() < 1e-12 * max(np.abs(x).max() for x in v) / G.ax[0].dx.min()
    vb, _ = pr.project(G, v, "xz")
    assert max(np.abs(vb[d] - v[d]).max() for d in range(3)) < 1e-12 * max(np.abs(x).max() for x in v)
