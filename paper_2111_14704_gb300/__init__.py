"""Python binding of librsol (the C ABI in include/rsol.h).

Argument marshalling only: every step of the packet push runs in librsol's
CUDA kernels.  PyTorch supplies device memory and the current stream.  There
is no CPU fallback: if librsol.so is missing or no CUDA device is present the
calls raise.

Names follow the C ABI: ``rsol_init`` -> :class:`Context`, and the context
methods ``push_gather``, ``deposit``, ``sort``, ``moments``, ``alfven_fields``,
``check``.  Packets live in a :class:`Particles` structure of arrays.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librsol.so")

STATUS = {0: "RSOL_OK", 1: "RSOL_ERR_INVALID_ARG", 2: "RSOL_ERR_CUDA", 3: "RSOL_ERR_OOM",
          4: "RSOL_ERR_NONFINITE", 5: "RSOL_ERR_COURANT", 6: "RSOL_ERR_UNSORTED",
          7: "RSOL_ERR_TIMEOUT"}
EXPORTS = ["rsol_init", "rsol_destroy", "rsol_last_error", "rsol_push_gather", "rsol_deposit",
           "rsol_sort", "rsol_moments", "rsol_alfven_fields", "rsol_check", "rsol_kernel_launches",
           "rsol_losses", "rsol_batch_init", "rsol_batch_destroy", "rsol_batch_last_error",
           "rsol_batch_total_nodes", "rsol_batch_sort", "rsol_batch_push_gather",
           "rsol_batch_alfven_fields", "rsol_batch_check", "rsol_loss_norm", "rsol_adjoint_step",
           "rsol_alfven_adjoint", "rsol_gradient", "rsol_push_subcycled",
           "rsol_sort_push_subcycled"]
CELL_BITS = 10


class RsolError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class CParams(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("shape", C.c_int32),
                ("precision", C.c_int32), ("deterministic", C.c_int32), ("bin", C.c_int32),
                ("warps", C.c_int32), ("dx", C.c_double), ("c", C.c_double),
                ("c_tilde", C.c_double), ("q_over_m", C.c_double), ("q", C.c_double)]


class CBatchDesc(C.Structure):
    _fields_ = [("n_boxes", C.c_int32), ("warps", C.c_int32), ("h_dims", C.c_void_p),
                ("h_c_tilde", C.c_void_p), ("h_dt", C.c_void_p), ("h_offsets", C.c_void_p)]


class CGradDesc(C.Structure):
    _fields_ = [("steps", C.c_int32), ("checkpoint_every", C.c_int32), ("dt", C.c_double),
                ("d_fields", C.c_void_p), ("h_modes", C.POINTER(C.c_double)),
                ("h_sigma", C.POINTER(C.c_double)), ("n_modes", C.c_int32), ("reserved", C.c_int32),
                ("t0", C.c_double), ("B0", C.c_double), ("vA", C.c_double),
                ("h_u_gas", C.POINTER(C.c_double))]


class CSubcycleDesc(C.Structure):
    _fields_ = [("courant", C.c_double), ("sigma_nn", C.c_double), ("max_level", C.c_int32),
                ("reserved", C.c_int32)]


class CParticles(C.Structure):
    _fields_ = [("n", C.c_int64), ("cell", C.c_void_p), ("off", C.c_void_p * 3),
                ("u", C.c_void_p * 3), ("w", C.c_void_p)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load librsol.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2111_14704_gb300.build`"
                           " (or __graft_entry__.build())")
    L = C.CDLL(path)
    vp = C.c_void_p
    L.rsol_init.argtypes = [C.POINTER(CParams), C.POINTER(vp)]
    L.rsol_destroy.argtypes = [vp]
    L.rsol_last_error.argtypes = [vp]
    L.rsol_last_error.restype = C.c_char_p
    L.rsol_push_gather.argtypes = [vp, C.POINTER(CParticles), vp, C.c_double, vp, vp]
    L.rsol_deposit.argtypes = [vp, C.POINTER(CParticles), vp, vp]
    L.rsol_sort.argtypes = [vp, C.POINTER(CParticles), C.POINTER(CParticles), vp]
    L.rsol_moments.argtypes = [vp, C.POINTER(CParticles), vp, C.POINTER(C.c_double), vp]
    L.rsol_alfven_fields.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int32,
                                     C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double),
                                     vp, vp]
    L.rsol_check.argtypes = [vp, vp]
    L.rsol_losses.argtypes = [vp, C.POINTER(CParticles), vp, C.c_double, C.c_double, C.c_double, vp]
    L.rsol_kernel_launches.argtypes = [vp]
    L.rsol_kernel_launches.restype = C.c_int64
    L.rsol_batch_init.argtypes = [C.POINTER(CParams), C.POINTER(CBatchDesc), C.POINTER(vp)]
    L.rsol_batch_destroy.argtypes = [vp]
    L.rsol_batch_last_error.argtypes = [vp]
    L.rsol_batch_last_error.restype = C.c_char_p
    L.rsol_batch_total_nodes.argtypes = [vp]
    L.rsol_batch_total_nodes.restype = C.c_int64
    L.rsol_batch_sort.argtypes = [vp, C.POINTER(CParticles), C.POINTER(CParticles), vp]
    L.rsol_batch_push_gather.argtypes = [vp, C.POINTER(CParticles), vp, vp, vp]
    L.rsol_batch_alfven_fields.argtypes = [vp, C.c_int32, C.POINTER(C.c_double),
                                           C.POINTER(C.c_double), C.c_int32, C.c_double,
                                           C.c_double, C.c_double, C.POINTER(C.c_double), vp, vp]
    L.rsol_batch_check.argtypes = [vp, vp]
    D = C.POINTER(C.c_double)
    L.rsol_loss_norm.argtypes = [vp, vp, vp, vp]
    L.rsol_adjoint_step.argtypes = [vp, C.POINTER(CParticles), vp, C.c_double, vp, vp,
                                    C.c_void_p * 3, C.c_void_p * 3, vp, vp]
    L.rsol_alfven_adjoint.argtypes = [vp, D, D, C.c_int32, C.c_double, C.c_double, C.c_double, D,
                                      vp, vp, vp, vp]
    L.rsol_gradient.argtypes = [vp, C.POINTER(CParticles), C.POINTER(CGradDesc), vp, vp, vp, vp, vp]
    L.rsol_push_subcycled.argtypes = [vp, C.POINTER(CParticles), vp, C.c_double,
                                      C.POINTER(CSubcycleDesc), vp, vp, vp]
    L.rsol_sort_push_subcycled.argtypes = [vp, C.POINTER(CParticles), C.POINTER(CParticles), vp,
                                           C.c_double, C.POINTER(CSubcycleDesc), vp,
                                           C.POINTER(C.c_int64), vp]
    for name in EXPORTS:
        fn = getattr(L, name)
        if name not in ("rsol_last_error", "rsol_kernel_launches", "rsol_batch_last_error",
                        "rsol_batch_total_nodes"):
            fn.restype = C.c_int
    _lib = L
    return L


@dataclass
class Params:
    """Mirror of rsol_params (see include/rsol.h)."""
    nx: int
    ny: int
    nz: int
    shape: int = 2
    precision: int = 32
    deterministic: int = 0
    bin: int = 0
    warps: int = 0
    dx: float = 1.0
    c: float = 1.0
    c_tilde: float = 1.0
    q_over_m: float = 1.0
    q: float = 1.0

    def to_c(self) -> CParams:
        return CParams(self.nx, self.ny, self.nz, self.shape, self.precision, self.deterministic,
                       self.bin, self.warps, self.dx, self.c, self.c_tilde, self.q_over_m, self.q)

    @property
    def grid(self):
        return (self.nx, self.ny, self.nz)


def _torch():
    import torch
    return torch


def _ptr(t) -> int:
    return int(t.data_ptr())


def _stream_handle(stream) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def pack_cells(cell: np.ndarray) -> np.ndarray:
    """(3, n) integer cells -> packed ix | iy << 10 | iz << 20 (int32 storage)."""
    c = cell.astype(np.int64)
    return (c[0] | (c[1] << CELL_BITS) | (c[2] << 2 * CELL_BITS)).astype(np.int32)


def unpack_cells(packed: np.ndarray) -> np.ndarray:
    p = packed.astype(np.int64) & 0xFFFFFFFF
    m = (1 << CELL_BITS) - 1
    return np.stack([p & m, (p >> CELL_BITS) & m, p >> 2 * CELL_BITS]).astype(np.int32)


class Particles:
    """Structure-of-arrays packets on the device (rsol_particles).

    ``cell`` int32 (packed cell), ``off`` / ``u`` lists of 3 tensors, ``w``.
    """

    def __init__(self, cell, off, u, w):
        self.cell, self.off, self.u, self.w = cell, list(off), list(u), w
        self.n = int(w.shape[0])

    @classmethod
    def empty(cls, n: int, precision: int = 32, device="cuda"):
        torch = _torch()
        dt = torch.float32 if precision == 32 else torch.float64
        mk = lambda: torch.empty(n, dtype=dt, device=device)
        return cls(torch.empty(n, dtype=torch.int32, device=device), [mk(), mk(), mk()],
                   [mk(), mk(), mk()], mk())

    @classmethod
    def from_numpy(cls, parts: dict, precision: int = 32, device="cuda"):
        """From the layout of rsol_inputs.make_particles (cell (3,n), off, u (3,n), w)."""
        torch = _torch()
        dt = torch.float32 if precision == 32 else torch.float64
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device=device, dtype=dt)
        cell = torch.from_numpy(pack_cells(parts["cell"])).to(device)
        return cls(cell, [t(parts["off"][a]) for a in range(3)], [t(parts["u"][a]) for a in range(3)],
                   t(parts["w"]))

    def to_numpy(self) -> dict:
        f = lambda x: x.detach().double().cpu().numpy()
        return {"cell": unpack_cells(self.cell.cpu().numpy()),
                "off": np.stack([f(x) for x in self.off]), "u": np.stack([f(x) for x in self.u]),
                "w": f(self.w)}

    def c_struct(self) -> CParticles:
        s = CParticles()
        s.n = self.n
        s.cell = _ptr(self.cell)
        for a in range(3):
            s.off[a] = _ptr(self.off[a])
            s.u[a] = _ptr(self.u[a])
        s.w = _ptr(self.w)
        return s

    def tensors(self):
        return [self.cell, *self.off, *self.u, self.w]


def fields_to_device(planes: np.ndarray, precision: int = 32, device="cuda"):
    """(6, nz, ny, nx) E, B planes -> node-major (nz, ny, nx, 8) device grid."""
    torch = _torch()
    nz, ny, nx = planes.shape[1:]
    g = np.zeros((nz, ny, nx, 8))
    g[..., :6] = np.moveaxis(planes, 0, -1)
    dt = torch.float32 if precision == 32 else torch.float64
    return torch.from_numpy(g).to(device=device, dtype=dt)


def grid_to_planes(grid) -> np.ndarray:
    """Node-major (nz, ny, nx, 8) device grid -> (8, nz, ny, nx) float64 planes."""
    return np.moveaxis(grid.detach().double().cpu().numpy(), -1, 0).copy()


class Context:
    """An rsol_ctx: parameters plus the library's scratch on the current device."""

    def __init__(self, params: Params):
        self.params = params
        self.L = load_library()
        h = C.c_void_p()
        self._cp = params.to_c()
        st = self.L.rsol_init(C.byref(self._cp), C.byref(h))
        if st != 0:
            raise RsolError(st, "rsol_init rejected the parameters or could not set up the device")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.L.rsol_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ok(self, st: int):
        if st != 0:
            raise RsolError(st, self.L.rsol_last_error(self.h).decode())

    def grid_tensor(self, zero: bool = True):
        torch = _torch()
        p = self.params
        dt = torch.float32 if p.precision == 32 else torch.float64
        mk = torch.zeros if zero else torch.empty
        return mk((p.nz, p.ny, p.nx, 8), dtype=dt, device="cuda")

    def push_gather(self, parts: Particles, fields, dt: float, feedback=None, stream=None):
        s = parts.c_struct()
        self._ok(self.L.rsol_push_gather(self.h, C.byref(s), _ptr(fields), float(dt),
                                         _ptr(feedback) if feedback is not None else None,
                                         _stream_handle(stream)))

    def deposit(self, parts: Particles, moments, stream=None):
        s = parts.c_struct()
        self._ok(self.L.rsol_deposit(self.h, C.byref(s), _ptr(moments), _stream_handle(stream)))

    def sort(self, parts_in: Particles, parts_out: Particles, stream=None):
        a, b = parts_in.c_struct(), parts_out.c_struct()
        self._ok(self.L.rsol_sort(self.h, C.byref(a), C.byref(b), _stream_handle(stream)))

    def moments(self, parts: Particles, feedback=None, stream=None) -> np.ndarray:
        s = parts.c_struct()
        out = np.zeros(16)
        self._ok(self.L.rsol_moments(self.h, C.byref(s),
                                     _ptr(feedback) if feedback is not None else None,
                                     out.ctypes.data_as(C.POINTER(C.c_double)),
                                     _stream_handle(stream)))
        return out

    def alfven_fields(self, modes: dict | None, t: float, B0: float, vA: float, u_gas, fields,
                      stream=None):
        if modes is None:
            rec = np.zeros((1, 8))
            sig = np.ones(1)
            nm = 0
        else:
            nm = len(modes["amp"])
            rec = np.zeros((nm, 8))
            rec[:, 0:3] = modes["n"]
            rec[:, 3:6] = modes["e"]
            rec[:, 6] = modes["amp"]
            rec[:, 7] = modes["phase"]
            sig = np.ascontiguousarray(modes["sigma"], dtype=np.float64)
        rec = np.ascontiguousarray(rec)
        ug = np.ascontiguousarray(np.asarray(u_gas, dtype=np.float64))
        D = C.POINTER(C.c_double)
        self._ok(self.L.rsol_alfven_fields(self.h, rec.ctypes.data_as(D), sig.ctypes.data_as(D), nm,
                                           float(t), float(B0), float(vA), ug.ctypes.data_as(D),
                                           _ptr(fields), _stream_handle(stream)))

    def losses(self, parts: Particles, sigma: float, dt: float, nn_uniform: float = 0.0,
               nn=None, stream=None):
        """Catastrophic-loss decay of the packet weights over one step (rsol_losses)."""
        s = parts.c_struct()
        self._ok(self.L.rsol_losses(self.h, C.byref(s), _ptr(nn) if nn is not None else None,
                                    float(nn_uniform), float(sigma), float(dt),
                                    _stream_handle(stream)))

    def check(self, stream=None):
        self._ok(self.L.rsol_check(self.h, _stream_handle(stream)))

    def kernel_launches(self) -> int:
        return int(self.L.rsol_kernel_launches(self.h))

    def push_subcycled(self, parts: Particles, fields, dt: float, courant: float,
                       feedback=None, levels=None, sigma_nn: float = 0.0, max_level: int = 8,
                       stream=None):
        """One global step with per-packet sub-cycling (rsol_push_subcycled);
        levels: optional uint8 device tensor receiving each packet's level."""
        d = CSubcycleDesc(float(courant), float(sigma_nn), int(max_level), 0)
        s = parts.c_struct()
        self._ok(self.L.rsol_push_subcycled(self.h, C.byref(s), _ptr(fields), float(dt), C.byref(d),
                                            _ptr(feedback) if feedback is not None else None,
                                            _ptr(levels) if levels is not None else None,
                                            _stream_handle(stream)))

    def sort_push_subcycled(self, parts_in: Particles, parts_out: Particles, fields, dt: float,
                            courant: float, feedback, sigma_nn: float = 0.0, max_level: int = 8,
                            stream=None) -> np.ndarray:
        """Level sort into parts_out, then the sub-cycled step on the tiled kernel
        (rsol_sort_push_subcycled).  Returns the packets per level."""
        d = CSubcycleDesc(float(courant), float(sigma_nn), int(max_level), 0)
        a, b = parts_in.c_struct(), parts_out.c_struct()
        counts = np.zeros(int(max_level) + 1, dtype=np.int64)
        self._ok(self.L.rsol_sort_push_subcycled(self.h, C.byref(a), C.byref(b), _ptr(fields), float(dt),
                                                 C.byref(d), _ptr(feedback),
                                                 counts.ctypes.data_as(C.POINTER(C.c_int64)),
                                                 _stream_handle(stream)))
        return counts

    # -- differentiable run (reverse mode) ------------------------------------
    def loss_norm(self, feedback, loss=None, stream=None):
        """Device tensor (L, 1/L) of L = ||sum_n S^n|| (rsol_loss_norm)."""
        torch = _torch()
        if loss is None:
            loss = torch.zeros(2, dtype=torch.float64, device="cuda")
        self._ok(self.L.rsol_loss_norm(self.h, _ptr(feedback), _ptr(loss), _stream_handle(stream)))
        return loss

    def adjoint_step(self, parts: Particles, fields, dt: float, feedback, loss, xbar, ubar,
                     field_bar, stream=None):
        """Reverse of one step (rsol_adjoint_step); xbar, ubar: (3, n) tensors, updated."""
        s = parts.c_struct()
        xb = (C.c_void_p * 3)(*[_ptr(xbar[a]) for a in range(3)])
        ub = (C.c_void_p * 3)(*[_ptr(ubar[a]) for a in range(3)])
        self._ok(self.L.rsol_adjoint_step(self.h, C.byref(s), _ptr(fields), float(dt), _ptr(feedback),
                                          _ptr(loss), xb, ub, _ptr(field_bar), _stream_handle(stream)))

    def alfven_adjoint(self, modes: dict, t: float, B0: float, vA: float, u_gas, field_bar,
                       amp_bar, field_bar_total=None, stream=None):
        """Adds dL/dA_m to amp_bar (device float64) from dL/dF (rsol_alfven_adjoint)."""
        rec, sig, nm = _mode_records(modes)
        ug = np.ascontiguousarray(np.asarray(u_gas, dtype=np.float64))
        D = C.POINTER(C.c_double)
        self._ok(self.L.rsol_alfven_adjoint(
            self.h, rec.ctypes.data_as(D), sig.ctypes.data_as(D), nm, float(t), float(B0), float(vA),
            ug.ctypes.data_as(D), _ptr(field_bar),
            _ptr(field_bar_total) if field_bar_total is not None else None, _ptr(amp_bar),
            _stream_handle(stream)))

    def gradient(self, parts: Particles, steps: int, dt: float, checkpoint_every: int = 8,
                 fields=None, modes: dict | None = None, t0: float = 0.0, B0: float = 1.0,
                 vA: float = 0.0, u_gas=(0.0, 0.0, 0.0), out: dict | None = None, stream=None) -> dict:
        """Checkpointed forward + reverse run (rsol_gradient) with a static field
        grid `fields` or the Alfven `modes` evaluated each step.  Returns device
        tensors: feedback (sum over steps), loss (L, 1/L), field_bar (dL/dF) and,
        for modes, amp_bar (dL/dA).  Reuses the tensors of `out` when given."""
        torch = _torch()
        if (fields is None) == (modes is None):
            raise ValueError("give exactly one of fields, modes")
        o = out if out is not None else {}
        if "feedback" not in o:
            o["feedback"] = self.grid_tensor(zero=False)
            o["field_bar"] = self.grid_tensor(zero=True)
            o["loss"] = torch.zeros(2, dtype=torch.float64, device="cuda")
            if modes is not None:
                o["amp_bar"] = torch.zeros(len(modes["amp"]), dtype=torch.float64, device="cuda")
        d = CGradDesc()
        d.steps = int(steps)
        d.checkpoint_every = int(checkpoint_every)
        d.dt = float(dt)
        keep = []
        D = C.POINTER(C.c_double)
        if modes is not None:
            rec, sig, nm = _mode_records(modes)
            ug = np.ascontiguousarray(np.asarray(u_gas, dtype=np.float64))
            keep += [rec, sig, ug]
            d.d_fields = None
            d.h_modes = rec.ctypes.data_as(D)
            d.h_sigma = sig.ctypes.data_as(D)
            d.n_modes = nm
            d.h_u_gas = ug.ctypes.data_as(D)
        else:
            d.d_fields = _ptr(fields)
            d.n_modes = 0
        d.t0, d.B0, d.vA = float(t0), float(B0), float(vA)
        s = parts.c_struct()
        self._ok(self.L.rsol_gradient(self.h, C.byref(s), C.byref(d), _ptr(o["feedback"]),
                                      _ptr(o["loss"]), _ptr(o["field_bar"]),
                                      _ptr(o["amp_bar"]) if "amp_bar" in o else None,
                                      _stream_handle(stream)))
        del keep
        return o


def _mode_records(modes):
    if modes is None:
        return np.zeros((1, 8)), np.ones(1), 0
    nm = len(modes["amp"])
    rec = np.zeros((nm, 8))
    rec[:, 0:3] = modes["n"]
    rec[:, 3:6] = modes["e"]
    rec[:, 6] = modes["amp"]
    rec[:, 7] = modes["phase"]
    return np.ascontiguousarray(rec), np.ascontiguousarray(modes["sigma"], dtype=np.float64), nm


class BatchContext:
    """An rsol_batch_ctx: many independent boxes sharing one packet array and
    one concatenated set of grids (see rsol_batch_init in include/rsol.h)."""

    def __init__(self, common: Params, dims, c_tilde, dt, offsets, warps: int = 0):
        self.params = common
        self.L = load_library()
        self.dims = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(-1, 3))
        self.c_tilde = np.ascontiguousarray(np.asarray(c_tilde, dtype=np.float64))
        self.dt = np.ascontiguousarray(np.asarray(dt, dtype=np.float64))
        self.offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        self.n_boxes = self.dims.shape[0]
        desc = CBatchDesc(self.n_boxes, warps, self.dims.ctypes.data, self.c_tilde.ctypes.data,
                          self.dt.ctypes.data, self.offsets.ctypes.data)
        self._cp = common.to_c()
        h = C.c_void_p()
        st = self.L.rsol_batch_init(C.byref(self._cp), C.byref(desc), C.byref(h))
        if st != 0:
            raise RsolError(st, "rsol_batch_init rejected the batch description")
        self.h = h
        self.total_nodes = int(self.L.rsol_batch_total_nodes(self.h))
        self.node_offsets = np.concatenate([[0], np.cumsum(np.prod(self.dims, axis=1))])

    def close(self):
        if getattr(self, "h", None):
            self.L.rsol_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ok(self, st: int):
        if st != 0:
            raise RsolError(st, self.L.rsol_batch_last_error(self.h).decode())

    def grid_tensor(self, zero: bool = True):
        torch = _torch()
        dt = torch.float32 if self.params.precision == 32 else torch.float64
        mk = torch.zeros if zero else torch.empty
        return mk((self.total_nodes, 8), dtype=dt, device="cuda")

    def box_view(self, grid, b: int):
        """Box b's slice of a concatenated grid as (nz, ny, nx, 8)."""
        nx, ny, nz = (int(v) for v in self.dims[b])
        lo = int(self.node_offsets[b])
        return grid[lo:lo + nx * ny * nz].view(nz, ny, nx, 8)

    def sort(self, parts_in: Particles, parts_out: Particles, stream=None):
        a, b = parts_in.c_struct(), parts_out.c_struct()
        self._ok(self.L.rsol_batch_sort(self.h, C.byref(a), C.byref(b), _stream_handle(stream)))

    def push_gather(self, parts: Particles, fields, feedback, stream=None):
        s = parts.c_struct()
        self._ok(self.L.rsol_batch_push_gather(self.h, C.byref(s), _ptr(fields), _ptr(feedback),
                                               _stream_handle(stream)))

    def alfven_fields(self, box: int, modes, t: float, B0: float, vA: float, u_gas, fields,
                      stream=None):
        rec, sig, nm = _mode_records(modes)
        ug = np.ascontiguousarray(np.asarray(u_gas, dtype=np.float64))
        D = C.POINTER(C.c_double)
        self._ok(self.L.rsol_batch_alfven_fields(self.h, int(box), rec.ctypes.data_as(D),
                                                 sig.ctypes.data_as(D), nm, float(t), float(B0),
                                                 float(vA), ug.ctypes.data_as(D), _ptr(fields),
                                                 _stream_handle(stream)))

    def check(self, stream=None):
        self._ok(self.L.rsol_batch_check(self.h, _stream_handle(stream)))
