"""Manufactured solution for the steady Navier-Stokes residual (test helper).

U_e = curl(psi a) with psi = sin^2(pi x) sin^2(pi y) sin^2(pi z) and a fixed
vector a, so U_e is divergence-free and vanishes (all components) on every
wall; P_e is a smooth pressure.  The body force that makes (U_e, P_e) an
exact steady solution of Eq. 2 is
    f = -[(1/Re) Lap U_e - (U_e . grad) U_e - grad P_e],
derived symbolically with sympy and sampled at the staggered face points.
"""
import numpy as np


def build(re, a=(1.0, 2.0, -1.5)):
    sp = __import__("sympy")
    x, y, z = sp.symbols("x y z", real=True)
    psi = sp.sin(sp.pi * x) ** 2 * sp.sin(sp.pi * y) ** 2 * sp.sin(sp.pi * z) ** 2
    A = [a[0] * psi, a[1] * psi, a[2] * psi]
    U = [sp.diff(A[2], y) - sp.diff(A[1], z),
         sp.diff(A[0], z) - sp.diff(A[2], x),
         sp.diff(A[1], x) - sp.diff(A[0], y)]
    P = sp.cos(sp.pi * x) * sp.sin(sp.pi * y) * sp.cos(2 * sp.pi * z)
    X = (x, y, z)
    f = []
    for c in range(3):
        lap = sum(sp.diff(U[c], X[d], 2) for d in range(3))
        adv = sum(U[d] * sp.diff(U[c], X[d]) for d in range(3))
        f.append(-(lap / re - adv - sp.diff(P, X[c])))
    lam = lambda e: sp.lambdify((x, y, z), e, "numpy")
    return [lam(e) for e in U], lam(P), [lam(e) for e in f]


def face_points(grid, c):
    """Coordinates (Z, Y, X) broadcast to the shape of component c (walls included)."""
    X, Y, Z = grid.ax
    xs = X.x if c == 0 else X.xc
    ys = Y.x if c == 1 else Y.xc
    zs = Z.x if c == 2 else Z.xc
    return np.meshgrid(zs, ys, xs, indexing="ij")


def sample(grid, funcs):
    out = []
    for c in range(3):
        Zg, Yg, Xg = face_points(grid, c)
        out.append(np.broadcast_to(funcs[c](Xg, Yg, Zg), Xg.shape).astype(np.float64).copy())
    return out
