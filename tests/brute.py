"""Brute-force references used to pin the oracle (textbook definitions, O(N_nodes * N_p)).

Nothing here copies the oracle's arithmetic: the shape functions are written
from the textbook piecewise B-spline definitions in terms of the signed
distance s = x_node - x (with the periodic minimum image), and every node of
the grid is visited.
"""
from __future__ import annotations

import numpy as np


def W_cic(s):
    """Linear B-spline (cloud-in-cell): max(0, 1 - |s|)."""
    s = np.abs(s)
    return np.where(s < 1.0, 1.0 - s, 0.0)


def W_tsc(s):
    """Quadratic B-spline (triangular-shaped cloud)."""
    s = np.abs(s)
    inner = 0.75 - s * s
    outer = 0.5 * (1.5 - s) ** 2
    return np.where(s <= 0.5, inner, np.where(s < 1.5, outer, 0.0))


def W(shape):
    return W_cic if shape == 1 else W_tsc


def min_image(d, n):
    """Periodic minimum-image distance on an axis of n nodes (unit spacing)."""
    return (d + 0.5 * n) % n - 0.5 * n


def axis_weights(shape, n, x):
    """Weights of every node k = 0..n-1 of one axis for particles at x (array)."""
    k = np.arange(n, dtype=np.float64)[:, None]
    return W(shape)(min_image(k - x[None, :], n))  # (n, N)


def deposit(shape, grid, pos, Q):
    """G[q, z, y, x] = sum_j W(x_node - x_j) Q[q, j] over all nodes (dx = 1)."""
    nx, ny, nz = grid
    wx = axis_weights(shape, nx, pos[0])
    wy = axis_weights(shape, ny, pos[1])
    wz = axis_weights(shape, nz, pos[2])
    return np.einsum("zj,yj,xj,qj->qzyx", wz, wy, wx, Q)


def gather(shape, grid, pos, F):
    """F at particles: sum over all nodes W(x_node - x_j) F[q, node]; returns (q, N)."""
    nx, ny, nz = grid
    wx = axis_weights(shape, nx, pos[0])
    wy = axis_weights(shape, ny, pos[1])
    wz = axis_weights(shape, nz, pos[2])
    return np.einsum("zj,yj,xj,qzyx->qj", wz, wy, wx, F)


def positions(parts):
    return parts["cell"].astype(np.float64) + parts["off"]


def unwrap_track(track, n):
    """Unwrap a (steps, N) periodic coordinate track of a box of n cells."""
    d = np.diff(track, axis=0)
    d = (d + 0.5 * n) % n - 0.5 * n
    return np.concatenate([track[:1], track[:1] + np.cumsum(d, axis=0)], axis=0)
