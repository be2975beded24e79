"""Conversions between the library's cell-indexed MAC layout and the oracle's
component arrays (test helper; no arithmetic of the method)."""
import numpy as np


def to_oracle(vel, shape):
    nz, ny, nx = shape
    q = np.asarray(vel, dtype=np.float64).reshape(3, nz, ny, nx)
    u = np.zeros((nz, ny, nx + 1)); u[:, :, :nx] = q[0]; u[:, :, 0] = 0
    v = np.zeros((nz, ny + 1, nx)); v[:, :ny, :] = q[1]; v[:, 0, :] = 0
    w = np.zeros((nz + 1, ny, nx)); w[:nz] = q[2]; w[0] = 0
    return [u, v, w]


def from_oracle(q):
    u, v, w = q
    nz, ny, nx = u.shape[0], u.shape[1], u.shape[2] - 1
    return np.concatenate([u[:, :, :nx].ravel(), v[:, :ny, :].ravel(), w[:nz].ravel()])
