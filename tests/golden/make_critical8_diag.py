"""Writes tests/golden/critical8_diag.npz with the oracle only.

Workload: 8^3 cosine grid, lid parallel to the diagonal plane (alpha = pi/4,
u = v = 1/sqrt(2) at z = 1, Eq. 4).  On this coarse grid the leading complex
pair (omega ~ 4.22) crosses the imaginary axis between Re = 1500 and 1550
(a second pair, omega ~ 1.73, stays below it there).  Steady states by Newton
continuation from rest (Re = 500, 1000, 1500), then the secant iteration on
sigma(Re) = Re(Lambda) from Re = 1500 and 1550, each evaluation = Newton
from the previous steady state + Arnoldi (Krylov dimension 30, 4
eigenvalues, Philox Gaussian start vector of seed 1).  Stops at
|dRe| <= 1e-8 Re.

Run:  python tests/golden/make_critical8_diag.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

import synth                                    # noqa: E402
import layout                                   # noqa: E402
from oracle import arnoldi, critical, fv, grid as G, krylov, poisson, simple   # noqa: E402

N = 8


def main():
    g = G.Grid(N, N, N, "cosine")
    tpf = poisson.TPF(g)
    lid = fv.lid_velocity(np.pi / 4)
    wts = fv.pack(fv.weights(g))
    state = {}
    U, P, _ = krylov.newton_continuation(g, tpf, [500.0, 1000.0, 1500.0], lid)
    state["U"] = U
    x0 = layout.to_oracle(synth.gaussian_velocity((N, N, N), 1), (N, N, N))

    def sigma(re):
        U, P, _ = krylov.newton(g, tpf, re, lid, U0=state["U"], tol=1e-10)
        state["U"] = U
        v0 = fv.pack(simple.project(g, tpf, x0)[0])
        A = lambda x: fv.pack(simple.shifted_operator(g, tpf, U, fv.unpack(g, x), re, 10.0)[0])
        lam, X, info = arnoldi.arnoldi_leading(A, v0, wts, nev=4, m=30, tol=1e-10)
        print(re, lam[0], flush=True)
        return float(lam[0].real), float(abs(lam[0].imag))

    re_cr, omega, hist = critical.secant(sigma, 1500.0, 1550.0, rtol=1e-8)
    print("Re_cr", re_cr, "omega", omega)
    np.savez(os.path.join(HERE, "critical8_diag.npz"), re_cr=re_cr, omega_cr=omega,
             hist=np.array(hist))


if __name__ == "__main__":
    main()
