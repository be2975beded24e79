"""Writes tests/golden/config1_16.npz with the oracle only.

Workload: unit cube, lid parallel to the x sidewall (alpha = 0), Re = 1000,
16^3 cosine-stretched grid.  Newton steady state to ||F|| < 1e-10, reached
from rest by continuation in Re (200, 400, 600, 800, 1000), then implicitly
restarted Arnoldi (Krylov dimension 30) for the 5 leading eigenvalues from
the Philox Gaussian start vector of seed 1.

Run:  python tests/golden/make_config1.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

import synth                                    # noqa: E402
import layout                                   # noqa: E402
from oracle import arnoldi, fv, grid as G, krylov, poisson, simple   # noqa: E402

N, RE, ALPHA = 16, 1000.0, 0.0


def main():
    g = G.Grid(N, N, N, "cosine")
    tpf = poisson.TPF(g)
    lid = fv.lid_velocity(ALPHA)
    U, P, hist = krylov.newton_continuation(g, tpf, [200.0, 400.0, 600.0, 800.0, RE], lid, tol=1e-10)
    print("newton", hist[-1])
    wts = fv.pack(fv.weights(g))
    x0 = layout.to_oracle(synth.gaussian_velocity((N, N, N), 1), (N, N, N))
    x0 = fv.pack(simple.project(g, tpf, x0)[0])
    A = lambda x: fv.pack(simple.shifted_operator(g, tpf, U, fv.unpack(g, x), RE, 10.0)[0])
    lam, X, info = arnoldi.arnoldi_leading(A, x0, wts, nev=5, m=30, tol=1e-10)
    print("eigenvalues", lam, info["restarts"], info["matvecs"])
    np.savez(os.path.join(HERE, "config1_16.npz"),
             U=layout.from_oracle(U), P=P.ravel(), lam=lam,
             evec0=layout.from_oracle(fv.unpack(g, X[:, 0].real)),
             evec0_imag=layout.from_oracle(fv.unpack(g, X[:, 0].imag)),
             newton_hist=np.array(hist[-1][1]))


if __name__ == "__main__":
    main()
