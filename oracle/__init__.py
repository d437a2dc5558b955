"""Python access to the FP64 C oracle (``oracle/rsol_oracle.c``).

TEST INFRASTRUCTURE.  Only the tests, the package smoke check and the
benchmark's CPU-baseline leg may import this module.  It compiles the C file
with gcc on first use (``-O2 -ffp-contract=off``), and wraps its functions for
numpy arrays in the oracle's own layout:

* particles: dict with ``cell`` (3, n) int32, ``off`` (3, n), ``u`` (3, n),
  ``w`` (n,) float64 -- the layout ``rsol_inputs.make_particles`` returns;
* fields: float64 (6, nz, ny, nx) = Ex, Ey, Ez, Bx, By, Bz planes;
* deposits: float64 (8, nz, ny, nx) planes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rsol_oracle.c")
_SO = os.path.join(_HERE, "librsol_oracle.so")
_lock = threading.Lock()
_lib = None
_override = []


class OrcParams(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("shape", C.c_int32), ("dx", C.c_double), ("c", C.c_double),
                ("c_tilde", C.c_double), ("q_over_m", C.c_double), ("q", C.c_double),
                ("dt", C.c_double)]


class OrcParticles(C.Structure):
    _fields_ = [("n", C.c_int64)] + \
        [(k, C.POINTER(C.c_int32)) for k in ("ix", "iy", "iz")] + \
        [(k, C.POINTER(C.c_double)) for k in ("ox", "oy", "oz", "ux", "uy", "uz", "w")]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _SO)
    return _SO


def _declare(L):
    """Declare the C signatures on a loaded oracle library."""
    D = C.POINTER(C.c_double)
    P = C.POINTER(OrcParams)
    L.orc_weights_1d.argtypes = [C.c_int, C.c_double, D]
    L.orc_weights_1d.restype = C.c_int
    L.orc_gather.argtypes = [P, D, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                             C.c_double, D, D]
    L.orc_boris.argtypes = [C.c_double, D, D, D, D, D, D, D]
    L.orc_boris_h.argtypes = [P]
    L.orc_boris_h.restype = C.c_double
    L.orc_feedback.argtypes = [P, C.c_double, D, D, D, D, C.c_double, D, C.c_double,
                               C.c_double, D]
    L.orc_step.argtypes = [P, D, C.POINTER(OrcParticles), D]
    L.orc_state_moments.argtypes = [P, C.POINTER(OrcParticles), D]
    L.orc_totals.argtypes = [P, C.POINTER(OrcParticles), D]
    L.orc_anchor_node.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_int32]
    L.orc_anchor_node.restype = C.c_int32
    L.orc_cell_key.argtypes = [C.c_int32] * 7
    L.orc_cell_key.restype = C.c_int64
    L.orc_stable_sort.argtypes = [C.POINTER(C.c_int64), C.c_int64, C.c_int64,
                                  C.POINTER(C.c_int64)]
    L.orc_stable_sort.restype = C.c_int
    L.orc_losses.argtypes = [P, C.POINTER(OrcParticles), D, C.c_double, C.c_double]
    L.orc_tangent_run.argtypes = [P, C.c_int, D, D, C.c_int64, C.POINTER(OrcParticles), D]
    L.orc_dt_limit.argtypes = [P, D, C.POINTER(OrcParticles), C.c_int64, C.c_double, C.c_double]
    L.orc_dt_limit.restype = C.c_double
    L.orc_subcycle_level.argtypes = [C.c_double, C.c_double, C.c_int]
    L.orc_subcycle_level.restype = C.c_int
    L.orc_step_subcycled.argtypes = [P, D, C.POINTER(OrcParticles), D, C.c_double, C.c_double,
                                     C.c_int, C.POINTER(C.c_int32)]
    return L


def lib():
    global _lib
    if _override:
        return _override[-1]
    with _lock:
        if _lib is None:
            _lib = _declare(C.CDLL(build()))
    return _lib


class use_library:
    """Context manager: route every call to another build of the oracle source
    (used by the mutation test, which compiles copies with planted mistakes)."""

    def __init__(self, so_path: str):
        self.L = _declare(C.CDLL(so_path))

    def __enter__(self):
        _override.append(self.L)
        return self.L

    def __exit__(self, *exc):
        _override.pop()
        return False


def compile_source(src_text: str, so_path: str) -> str:
    """Compile C source text with the oracle's flags into so_path."""
    c_path = so_path[:-3] + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared",
                    "-o", so_path, c_path, "-lm"], check=True)
    return so_path


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def params(grid, *, shape: int, dt: float, c: float = 1.0, c_tilde: float = 1.0,
           q_over_m: float = 1.0, q: float = 1.0, dx: float = 1.0) -> OrcParams:
    nx, ny, nz = grid
    return OrcParams(nx, ny, nz, shape, dx, c, c_tilde, q_over_m, q, dt)


class Particles:
    """Oracle-owned contiguous copy of a particle set (mutated in place by step)."""

    def __init__(self, parts: dict):
        n = parts["w"].shape[0]
        self.cell = np.ascontiguousarray(parts["cell"], dtype=np.int32).copy()
        self.off = np.ascontiguousarray(parts["off"], dtype=np.float64).copy()
        self.u = np.ascontiguousarray(parts["u"], dtype=np.float64).copy()
        self.w = np.ascontiguousarray(parts["w"], dtype=np.float64).copy()
        ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
        self.s = OrcParticles(n, ip(self.cell[0]), ip(self.cell[1]), ip(self.cell[2]),
                              _dp(self.off[0]), _dp(self.off[1]), _dp(self.off[2]),
                              _dp(self.u[0]), _dp(self.u[1]), _dp(self.u[2]), _dp(self.w))
        self.n = n

    def as_dict(self) -> dict:
        return {"cell": self.cell.copy(), "off": self.off.copy(), "u": self.u.copy(),
                "w": self.w.copy()}


def _grid_planes(p: OrcParams, nplanes: int) -> np.ndarray:
    return np.zeros((nplanes, p.nz, p.ny, p.nx), dtype=np.float64)


def step(p: OrcParams, fields: np.ndarray, P: Particles, deposit: bool = True):
    """One RSOL step in place; returns the 8 feedback planes (or None)."""
    F = np.ascontiguousarray(fields, dtype=np.float64)
    assert F.shape == (6, p.nz, p.ny, p.nx)
    G = _grid_planes(p, 8) if deposit else None
    lib().orc_step(C.byref(p), _dp(F), C.byref(P.s), _dp(G) if G is not None else None)
    return G


def state_moments(p: OrcParams, P: Particles) -> np.ndarray:
    G = _grid_planes(p, 8)
    lib().orc_state_moments(C.byref(p), C.byref(P.s), _dp(G))
    return G


def totals(p: OrcParams, P: Particles) -> np.ndarray:
    out = np.zeros(8)
    lib().orc_totals(C.byref(p), C.byref(P.s), _dp(out))
    return out


def weights_1d(shape: int, f: float):
    w = np.zeros(3)
    off = lib().orc_weights_1d(shape, f, _dp(w))
    return off, w


def gather(p: OrcParams, fields: np.ndarray, cell, off):
    F = np.ascontiguousarray(fields, dtype=np.float64)
    E = np.zeros(3)
    B = np.zeros(3)
    lib().orc_gather(C.byref(p), _dp(F), int(cell[0]), int(cell[1]), int(cell[2]),
                     float(off[0]), float(off[1]), float(off[2]), _dp(E), _dp(B))
    return E, B


def boris(h: float, E, B, u0):
    E = np.ascontiguousarray(E, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    um, up, u1, gm = np.zeros(3), np.zeros(3), np.zeros(3), np.zeros(1)
    lib().orc_boris(h, _dp(E), _dp(B), _dp(u0), _dp(um), _dp(up), _dp(u1), _dp(gm))
    return um, up, u1, float(gm[0])


def boris_h(p: OrcParams) -> float:
    return lib().orc_boris_h(C.byref(p))


def anchor_nodes(shape: int, grid, cell: np.ndarray, off: np.ndarray) -> np.ndarray:
    """Per-axis anchor node of every packet (CIC: its cell; TSC: nearest node)."""
    L = lib()
    out = np.empty_like(cell, dtype=np.int32)
    for a in range(3):
        for j in range(cell.shape[1]):
            out[a, j] = L.orc_anchor_node(shape, int(cell[a, j]), float(off[a, j]), grid[a])
    return out


def cell_keys(grid, bin_: int, cell: np.ndarray) -> np.ndarray:
    nx, ny, nz = grid
    L = lib()
    return np.array([L.orc_cell_key(nx, ny, nz, bin_, int(cell[0, j]), int(cell[1, j]),
                                    int(cell[2, j])) for j in range(cell.shape[1])],
                    dtype=np.int64)


def sort_keys(grid, bin_: int, shape: int, cell: np.ndarray, off: np.ndarray) -> np.ndarray:
    """Sort key of every packet: the bin-major key of its anchor node."""
    return cell_keys(grid, bin_, anchor_nodes(shape, grid, cell, off))


def n_keys(grid, bin_: int) -> int:
    nx, ny, nz = grid
    nb = [(n + bin_ - 1) // bin_ for n in (nx, ny, nz)]
    return nb[0] * nb[1] * nb[2] * bin_ ** 3


def stable_sort(keys: np.ndarray, nkeys: int) -> np.ndarray:
    keys = np.ascontiguousarray(keys, dtype=np.int64)
    perm = np.zeros(keys.shape[0], dtype=np.int64)
    rc = lib().orc_stable_sort(keys.ctypes.data_as(C.POINTER(C.c_int64)), keys.shape[0],
                               nkeys, perm.ctypes.data_as(C.POINTER(C.c_int64)))
    if rc != 0:
        raise ValueError("oracle sort: key out of range")
    return perm


def sort_particles(P: Particles, grid, bin_: int, shape: int) -> np.ndarray:
    """Stable sort of the particle set by anchor-node key, in place; returns the permutation."""
    keys = sort_keys(grid, bin_, shape, P.cell, P.off)
    perm = stable_sort(keys, n_keys(grid, bin_))
    P.cell[...] = P.cell[:, perm]
    P.off[...] = P.off[:, perm]
    P.u[...] = P.u[:, perm]
    P.w[...] = P.w[perm]
    return perm


def losses(p: OrcParams, P: Particles, sigma: float, nn_uniform: float = 0.0, nn=None):
    """Catastrophic-loss decay of the packet weights over one step p.dt, in place."""
    g = None
    if nn is not None:
        g = np.ascontiguousarray(nn, dtype=np.float64)
        assert g.shape == (p.nz, p.ny, p.nx)
    lib().orc_losses(C.byref(p), C.byref(P.s), _dp(g) if g is not None else None,
                     float(nn_uniform), float(sigma))


def tangent(p: OrcParams, fields: np.ndarray, dfields: np.ndarray, P: Particles, steps: int = 0):
    """(L, dL/d eps) for L = ||sum_n S^n||_2 over `steps` steps (static fields,
    arrays (6, nz, ny, nx)) or len(fields) steps (arrays (n, 6, nz, ny, nx))."""
    F = np.ascontiguousarray(fields, dtype=np.float64)
    dF = np.ascontiguousarray(dfields, dtype=np.float64)
    assert F.shape == dF.shape
    if F.ndim == 4:
        n, stride = steps, 0
    else:
        n, stride = F.shape[0], int(np.prod(F.shape[1:]))
    out = np.zeros(2)
    lib().orc_tangent_run(C.byref(p), int(n), _dp(F), _dp(dF), stride, C.byref(P.s), _dp(out))
    return float(out[0]), float(out[1])


def momentum_source_loss(p: OrcParams, fields: np.ndarray, P: Particles, steps: int = 0) -> float:
    """L = ||sum_n S^n||_2 (S = deposited momentum source, planes 4..6) over a run."""
    F = np.asarray(fields, dtype=np.float64)
    seq = [F] * steps if F.ndim == 4 else list(F)
    G = None
    for Fn in seq:
        g = step(p, Fn, P)[4:7]
        G = g if G is None else G + g
    return float(np.sqrt((G * G).sum()))


def dt_limits(p: OrcParams, fields: np.ndarray, P: Particles, courant: float,
              sigma_nn: float = 0.0) -> np.ndarray:
    """Per-packet timestep limits C min(1/Omega~, dx/|v_eff|, N/|dN/dt|) (Sec. 3)."""
    F = np.ascontiguousarray(fields, dtype=np.float64)
    return np.array([lib().orc_dt_limit(C.byref(p), _dp(F), C.byref(P.s), j, float(courant),
                                        float(sigma_nn)) for j in range(P.n)])


def subcycle_level(dt: float, limit: float, max_level: int) -> int:
    return int(lib().orc_subcycle_level(float(dt), float(limit), int(max_level)))


def step_subcycled(p: OrcParams, fields: np.ndarray, P: Particles, courant: float,
                   sigma_nn: float = 0.0, max_level: int = 8, deposit: bool = True):
    """One global step with per-packet sub-cycling, in place.
    Returns (8 feedback planes or None, levels)."""
    F = np.ascontiguousarray(fields, dtype=np.float64)
    assert F.shape == (6, p.nz, p.ny, p.nx)
    G = _grid_planes(p, 8) if deposit else None
    lev = np.zeros(P.n, dtype=np.int32)
    lib().orc_step_subcycled(C.byref(p), _dp(F), C.byref(P.s), _dp(G) if G is not None else None,
                             float(courant), float(sigma_nn), int(max_level),
                             lev.ctypes.data_as(C.POINTER(C.c_int32)))
    return G, lev
