"""Seeded synthetic inputs for the RSOL cosmic-ray push.

This module is the one place both sides of every comparison take their inputs
from: the CUDA library's tests and benchmark, and the FP64 oracle.  It holds
random draws and the analytic field source that stands in for the MHD solver
(which is out of scope), and nothing of the particle method itself (no shape
functions, no push, no deposit).

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw ``i`` of stream ``s`` under seed ``seed`` is the SplitMix64
output for the state ``key(seed, s) + i``.  Every draw is therefore addressable
on its own, which lets a sample of particles be regenerated by index.

Workload shapes follow the paper's problem statement (Sec. 2: packets with
weight N_j, position, momentum; Eq. momentum with E = -(u/c) x B from the MHD
fluid) with the readings listed in the design notes:

* positions uniform in a periodic box, held as an integer cell per axis plus
  an in-cell offset in [0, 1) drawn on a 2^-24 lattice (exact in FP32 and FP64);
* |u| = |p|/(m c) from a power law dN/dp ~ p^-slope on [p1, p2] by inverse CDF,
  isotropic directions; optionally a Lorentz boost along x (a beam);
* equal weights N_j = 1;
* fields: uniform B0 x-hat plus a superposition of Alfven modes, with
  E = -(u/c) x B.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream ids of the particle draws
S_CELL = (0, 1, 2)
S_OFF = (3, 4, 5)
S_PMAG = 6
S_MU = 7
S_PHI = 8
S_MODE = 100


def splitmix64(state: np.ndarray) -> np.ndarray:
    """SplitMix64 output for the given states (state advanced by one golden step)."""
    with np.errstate(over="ignore"):
        z = state.astype(np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    """Base state of one stream: the 64-bit key (seed << 48) | (stream << 32)."""
    return np.uint64(((seed & 0xFFFF) << 48) | ((stream & 0xFFFF) << 32))


def raw(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """64-bit draws ``idx`` of stream ``stream``; ``idx`` < 2^32."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return splitmix64(stream_key(seed, stream) + idx)


def uniform(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each draw."""
    return (raw(seed, stream, idx) >> np.uint64(11)).astype(np.float64) * 2.0**-53


def uniform24(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Uniform values in [0, 1) on the 2^-24 lattice (exact in float32)."""
    return (raw(seed, stream, idx) >> np.uint64(40)).astype(np.float64) * 2.0**-24


def power_law_momentum(U: np.ndarray, p1: float, p2: float, slope: float) -> np.ndarray:
    """Inverse CDF of dN/dp ~ p^-slope on [p1, p2] (slope > 1)."""
    e = 1.0 - slope
    return (p1**e + U * (p2**e - p1**e)) ** (1.0 / e)


def make_particles(n: int, grid: tuple[int, int, int], seed: int, *,
                   p_range: tuple[float, float] = (1.0, 100.0), slope: float = 4.5,
                   beam_beta: float = 0.0, fp32: bool = True,
                   first: int = 0) -> dict:
    """Seeded macroparticles in SoA form.

    Returns a dict of float64/int32 numpy arrays:
    ``cell`` (3, n) int32 cell per axis, ``off`` (3, n) offsets in [0, 1),
    ``u`` (3, n) dimensionless momentum gamma*beta, ``w`` (n,) weights N_j.
    With ``fp32`` the momenta are rounded to float32 (offsets already are), so
    an FP32 run and an FP64 run can start from identical values.
    ``first`` selects particles first .. first+n-1 of the same seeded set.
    """
    nx, ny, nz = grid
    idx = np.arange(first, first + n, dtype=np.uint64)
    cell = np.empty((3, n), dtype=np.int32)
    for a, nn in enumerate((nx, ny, nz)):
        cell[a] = np.minimum((uniform(seed, S_CELL[a], idx) * nn).astype(np.int64), nn - 1)
    off = np.stack([uniform24(seed, S_OFF[a], idx) for a in range(3)])
    pmag = power_law_momentum(uniform(seed, S_PMAG, idx), p_range[0], p_range[1], slope)
    mu = 2.0 * uniform(seed, S_MU, idx) - 1.0
    phi = 2.0 * math.pi * uniform(seed, S_PHI, idx)
    st = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    u = np.stack([pmag * mu, pmag * st * np.cos(phi), pmag * st * np.sin(phi)])
    if beam_beta:
        # Lorentz boost of the four-momentum (gamma, u) by beam_beta along x.
        gd = 1.0 / math.sqrt(1.0 - beam_beta * beam_beta)
        g = np.sqrt(1.0 + (u * u).sum(0))
        u[0] = gd * (u[0] + beam_beta * g)
    if fp32:
        u = u.astype(np.float32).astype(np.float64)
    w = np.ones(n, dtype=np.float64)
    return {"cell": cell, "off": off, "u": u, "w": w}


def alfven_modes(n_modes: int, seed: int, *, L: tuple[float, float, float],
                 kmax: int = 16, dB_rms: float = 0.1, B0: float = 1.0) -> dict:
    """Seeded Alfven-mode parameters.

    Integer wave vectors n with 0 < |n| <= kmax (k = 2 pi n / L, periodic),
    phases uniform in [0, 2 pi), propagation sign sigma = +-1, and equal
    amplitudes A = dB_rms * B0 * sqrt(2 / n_modes) so that the rms of
    |dB| / B0 is dB_rms.
    """
    ns = []
    i = 0
    span = 2 * kmax + 1
    while len(ns) < n_modes:
        cand = [int(raw(seed, S_MODE + a, np.array([i]))[0] % np.uint64(span)) - kmax
                for a in range(3)]
        i += 1
        r2 = sum(c * c for c in cand)
        if 0 < r2 <= kmax * kmax:
            ns.append(cand)
    nvec = np.array(ns, dtype=np.float64)
    k = 2.0 * math.pi * nvec / np.array(L, dtype=np.float64)
    j = np.arange(n_modes, dtype=np.uint64)
    phase = 2.0 * math.pi * uniform(seed, S_MODE + 3, j)
    sigma = np.where(raw(seed, S_MODE + 4, j) >> np.uint64(63), -1.0, 1.0)
    amp = np.full(n_modes, dB_rms * B0 * math.sqrt(2.0 / n_modes))
    # polarisation e = (k_hat x x_hat) / |k_hat x x_hat|, y_hat when k || x_hat
    e = np.zeros((n_modes, 3))
    for m in range(n_modes):
        kx, ky, kz = k[m]
        cx = np.array([0.0, kz, -ky])
        nrm = math.sqrt(cx[1] ** 2 + cx[2] ** 2)
        e[m] = cx / nrm if nrm > 0 else np.array([0.0, 1.0, 0.0])
    return {"n": nvec, "k": k, "phase": phase, "sigma": sigma, "amp": amp, "e": e}


def field_grid(grid: tuple[int, int, int], *, t: float = 0.0, B0: float = 1.0,
               modes: dict | None = None, vA: float = 0.0,
               u_gas: tuple[float, float, float] = (0.0, 0.0, 0.0),
               c: float = 1.0, dx: float = 1.0) -> np.ndarray:
    """E and B on the periodic node grid: array (6, nz, ny, nx) = Ex, Ey, Ez, Bx, By, Bz.

    B = B0 x_hat + sum_m A_m e_m cos(k_m . r - w_m t + phi_m), w_m = sigma_m k_x vA,
    gas velocity u = u_gas + sum_m (-sigma_m vA dB_m / B0), and the ideal-MHD
    electric field E = -(u / c) x B.  Nodes sit at r = (ix, iy, iz) * dx.
    """
    nx, ny, nz = grid
    z, y, x = np.meshgrid(np.arange(nz) * dx, np.arange(ny) * dx, np.arange(nx) * dx,
                          indexing="ij")
    B = np.zeros((3, nz, ny, nx))
    B[0] += B0
    u = np.zeros((3, nz, ny, nx))
    for a in range(3):
        u[a] += u_gas[a]
    if modes is not None:
        for m in range(len(modes["amp"])):
            kx, ky, kz = modes["k"][m]
            om = modes["sigma"][m] * kx * vA
            cphi = modes["amp"][m] * np.cos(kx * x + ky * y + kz * z - om * t + modes["phase"][m])
            for a in range(3):
                dBa = modes["e"][m, a] * cphi
                B[a] += dBa
                u[a] += -modes["sigma"][m] * vA * dBa / B0
    E = -np.cross(u, B, axis=0) / c
    return np.concatenate([E, B], axis=0)


def log_uniform_int(seed: int, stream: int, idx: np.ndarray, lo: float, hi: float) -> np.ndarray:
    """round(exp(U[ln lo, ln hi])) for seeded batch shapes."""
    U = uniform(seed, stream, idx)
    return np.rint(np.exp(math.log(lo) + U * (math.log(hi) - math.log(lo)))).astype(np.int64)


def batch_boxes(n_boxes: int, seed: int, *, n_lo: float = 16, n_hi: float = 64,
                p_lo: float = 2 ** 12, p_hi: float = 2 ** 18, r_lo: float = 1.0,
                r_hi: float = 100.0, db_lo: float = 0.01, db_hi: float = 0.3) -> dict:
    """Seeded shapes of a batch of independent boxes: cubic grid edge and packet
    count log-uniform in [n_lo, n_hi] and [p_lo, p_hi], c/c~ log-uniform in
    [r_lo, r_hi], rms dB/B0 uniform in [db_lo, db_hi]."""
    b = np.arange(n_boxes, dtype=np.uint64)
    edge = log_uniform_int(seed, 200, b, n_lo, n_hi)
    count = log_uniform_int(seed, 201, b, p_lo, p_hi)
    ratio = np.exp(math.log(r_lo) + uniform(seed, 202, b) * (math.log(r_hi) - math.log(r_lo)))
    db = db_lo + uniform(seed, 203, b) * (db_hi - db_lo)
    return {"edge": edge, "count": count, "c_over_c_tilde": ratio, "dB_rms": db}
