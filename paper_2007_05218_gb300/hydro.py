"""Thin ctypes binding of include/hydro.h (argument marshalling only).

Functions keep the C names (hydro_alloc, hydro_step, ...).  Device buffers are
torch CUDA tensors (PyTorch supplies memory and streams); every step of the
update runs in the CUDA library.  There is no CPU fallback: if the library is
missing or was built for another machine, loading it raises.

`Boxes` is a small convenience owner of the state/scratch tensors and handle.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

HYDRO_OK = 0
HYDRO_PENDING = 1
HYDRO_ERR_INVALID = -1
HYDRO_ERR_NOMEM = -2
HYDRO_ERR_NONPHYSICAL = -3
HYDRO_ERR_TIMEOUT = -4
HYDRO_ERR_CUDA = -5
HYDRO_BC = {"periodic": 0, "outflow": 1, "reflect": 2}
HYDRO_FP64 = 0
HYDRO_MIXED = 1
HYDRO_NG = 4
HYDRO_LIMITER_CW84, HYDRO_LIMITER_CS08 = 0, 1
HYDRO_RIEMANN_HLLC, HYDRO_RIEMANN_TWO_SHOCK = 0, 1

EXPORTED = ("hydro_workspace_size", "hydro_box_layout", "hydro_alloc", "hydro_free", "hydro_fill_ghosts",
            "hydro_compute_dt", "hydro_step", "hydro_sync", "hydro_get_time", "hydro_upload",
            "hydro_download", "hydro_debug_fields", "hydro_kernel_launches", "hydro_profile_begin",
            "hydro_profile_end", "hydro_compute_dt_noalloc", "hydro_autotune", "hydro_use_graphs",
            "hydro_server_create", "hydro_server_destroy", "hydro_submit", "hydro_poll",
            "hydro_server_get_stats", "hydro_set_neighbors", "hydro_set_shared_dt", "hydro_set_method",
            "hydro_fuse_lines", "hydro_fuse_tiles", "hydro_set_tile_shape", "hydro_measure_peaks",
            "hydro_persistent", "hydro_set_spin_limit", "hydro_last_error")


class HydroError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class hydro_box_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("ng", ctypes.c_int32), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dz", ctypes.c_double), ("gamma", ctypes.c_double), ("cfl", ctypes.c_double),
                ("bc", ctypes.c_int32 * 6), ("precision", ctypes.c_int32)]


class hydro_layout(ctypes.Structure):
    _fields_ = [("offset", ctypes.c_int64), ("pitch", ctypes.c_int64), ("plane", ctypes.c_int64),
                ("var_stride", ctypes.c_int64)]


class hydro_tuning(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("precision", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("order", ctypes.c_int32), ("ms", ctypes.c_float), ("tile_rows", ctypes.c_int32),
                ("tile_seg", ctypes.c_int32)]


class hydro_server_config(ctypes.Structure):
    _fields_ = [("pool_dev", ctypes.c_void_p), ("pool_bytes", ctypes.c_size_t), ("max_active", ctypes.c_int32),
                ("dry_run", ctypes.c_int32)]


class hydro_request(ctypes.Structure):
    _fields_ = [("desc", hydro_box_desc), ("ic_host", ctypes.c_void_p), ("nsteps", ctypes.c_int32)]


class hydro_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("steps", ctypes.c_int32), ("time", ctypes.c_double),
                ("queued_s", ctypes.c_double), ("latency_s", ctypes.c_double)]


class hydro_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("queued", "active", "admitted", "finished", "ticks",
                                              "kernel_launches", "bytes_in_use", "peak_bytes", "budget_bytes")]


class hydro_stage_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


_lib = None
_lock = threading.Lock()
_VP = ctypes.c_void_p
_SZ = ctypes.c_size_t


def load(path: str | None = None):
    """Loads (building first if needed) libhydro_gb300.so; raises if that fails."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or _build.LIB_PATH
        if not os.path.exists(path) or not _build.up_to_date():
            _build.build()
        L = ctypes.CDLL(path)
        D = ctypes.POINTER(hydro_box_desc)
        i = ctypes.c_int
        L.hydro_workspace_size.argtypes = [D, i, ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)]
        L.hydro_box_layout.argtypes = [D, i, i, ctypes.POINTER(hydro_layout)]
        L.hydro_alloc.argtypes = [D, i, _VP, _SZ, _VP, _SZ, ctypes.POINTER(_VP)]
        L.hydro_free.argtypes = [_VP]
        L.hydro_fill_ghosts.argtypes = [_VP, _VP]
        L.hydro_compute_dt.argtypes = [_VP, _VP, _VP]
        L.hydro_step.argtypes = [_VP, _VP, i, _VP]
        L.hydro_sync.argtypes = [_VP, _VP]
        L.hydro_get_time.argtypes = [_VP, _VP, _VP]
        L.hydro_upload.argtypes = [_VP, _VP, _SZ, _VP]
        L.hydro_download.argtypes = [_VP, _VP, _SZ, _VP]
        L.hydro_debug_fields.argtypes = [D, i, i, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_int32)]
        L.hydro_kernel_launches.argtypes = [_VP, ctypes.POINTER(ctypes.c_int64)]
        L.hydro_profile_begin.argtypes = [_VP]
        L.hydro_profile_end.argtypes = [_VP, ctypes.POINTER(hydro_stage_time), i, ctypes.POINTER(i)]
        L.hydro_compute_dt_noalloc.argtypes = [D, i, _VP, _VP, _VP]
        L.hydro_measure_peaks.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(i), _VP]
        L.hydro_autotune.argtypes = [_VP, i, ctypes.POINTER(hydro_tuning), i, ctypes.POINTER(i), _VP]
        L.hydro_use_graphs.argtypes = [_VP, i]
        L.hydro_fuse_lines.argtypes = [_VP, i]
        L.hydro_fuse_tiles.argtypes = [_VP, i]
        L.hydro_persistent.argtypes = [_VP, i]
        L.hydro_set_spin_limit.argtypes = [_VP, ctypes.c_int64, i]
        L.hydro_set_tile_shape.argtypes = [_VP, i, i]
        L.hydro_set_neighbors.argtypes = [_VP, _VP]
        L.hydro_set_shared_dt.argtypes = [_VP, i]
        L.hydro_set_method.argtypes = [_VP, i, i]
        L.hydro_server_create.argtypes = [ctypes.POINTER(hydro_server_config), ctypes.POINTER(_VP)]
        L.hydro_server_destroy.argtypes = [_VP]
        L.hydro_submit.argtypes = [_VP, ctypes.POINTER(hydro_request), ctypes.POINTER(ctypes.c_int64)]
        L.hydro_poll.argtypes = [_VP, ctypes.c_int64, _VP, _SZ, ctypes.POINTER(hydro_result)]
        L.hydro_server_get_stats.argtypes = [_VP, ctypes.POINTER(hydro_server_stats)]
        L.hydro_last_error.restype = ctypes.c_char_p
        L.hydro_last_error.argtypes = []
        _lib = L
        return L


def hydro_last_error() -> str:
    return load().hydro_last_error().decode()


def _check(rc: int) -> int:
    if rc < 0:
        raise HydroError(rc, hydro_last_error())
    return rc


def _stream(stream) -> int | None:
    """torch.cuda.Stream, raw handle int, or None (torch's current stream)."""
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def desc_array(descs):
    arr = (hydro_box_desc * len(descs))()
    for k, d in enumerate(descs):
        arr[k] = d
    return arr


def make_desc(shape, dx, gamma, cfl, bc, precision=HYDRO_FP64) -> hydro_box_desc:
    d = hydro_box_desc()
    d.nx, d.ny, d.nz = (int(v) for v in shape)
    d.ng = HYDRO_NG
    d.dx, d.dy, d.dz = (float(v) for v in dx)
    d.gamma = float(gamma)
    d.cfl = float(cfl)
    for a in range(6):
        d.bc[a] = HYDRO_BC[bc[a]] if isinstance(bc[a], str) else int(bc[a])
    d.precision = int(precision)
    return d


def desc_of(problem, precision=HYDRO_FP64) -> hydro_box_desc:
    return make_desc(problem.shape, problem.dx, problem.gamma, problem.cfl, problem.bc, precision)


# ---------------------------------------------------------------- C names
def hydro_workspace_size(descs):
    arr = desc_array(descs)
    sb, wb = _SZ(), _SZ()
    _check(load().hydro_workspace_size(arr, len(descs), ctypes.byref(sb), ctypes.byref(wb)))
    return sb.value, wb.value


def hydro_box_layout(descs, box: int) -> hydro_layout:
    out = hydro_layout()
    _check(load().hydro_box_layout(desc_array(descs), len(descs), int(box), ctypes.byref(out)))
    return out


def hydro_debug_fields(descs, box: int):
    """(byte offset in scratch, number of fields, element bytes) of box's intermediates."""
    off, nf, eb = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().hydro_debug_fields(desc_array(descs), len(descs), int(box), ctypes.byref(off),
                                     ctypes.byref(nf), ctypes.byref(eb)))
    return off.value, nf.value, eb.value


def hydro_alloc(descs, state, state_bytes, scratch, scratch_bytes) -> int:
    h = _VP()
    _check(load().hydro_alloc(desc_array(descs), len(descs), _ptr(state), int(state_bytes), _ptr(scratch),
                              int(scratch_bytes), ctypes.byref(h)))
    return h.value


def hydro_free(h: int) -> None:
    _check(load().hydro_free(h))


def hydro_fill_ghosts(h: int, stream=None) -> None:
    _check(load().hydro_fill_ghosts(h, _stream(stream)))


def hydro_compute_dt(h: int, dt_dev, stream=None) -> None:
    _check(load().hydro_compute_dt(h, _ptr(dt_dev), _stream(stream)))


def hydro_step(h: int, dt_dev=None, nsteps: int = 1, stream=None) -> None:
    _check(load().hydro_step(h, _ptr(dt_dev), int(nsteps), _stream(stream)))


def hydro_sync(h: int, stream=None) -> int:
    return _check(load().hydro_sync(h, _stream(stream)))


def hydro_get_time(h: int, nboxes: int, stream=None) -> np.ndarray:
    out = np.zeros(nboxes)
    _check(load().hydro_get_time(h, out.ctypes.data, _stream(stream)))
    return out


def hydro_upload(h: int, host: np.ndarray, stream=None) -> None:
    host = np.ascontiguousarray(host, dtype=np.float64)
    _check(load().hydro_upload(h, host.ctypes.data, host.nbytes, _stream(stream)))


def hydro_download(h: int, host: np.ndarray, stream=None) -> None:
    assert host.dtype == np.float64 and host.flags["C_CONTIGUOUS"]
    _check(load().hydro_download(h, host.ctypes.data, host.nbytes, _stream(stream)))


def hydro_kernel_launches(h: int) -> int:
    c = ctypes.c_int64()
    _check(load().hydro_kernel_launches(h, ctypes.byref(c)))
    return c.value


def hydro_profile_begin(h: int) -> None:
    _check(load().hydro_profile_begin(h))


def hydro_profile_end(h: int) -> dict:
    """{stage name: (kernel launches, total device ms)} in launch order."""
    buf = (hydro_stage_time * 32)()
    n = ctypes.c_int()
    _check(load().hydro_profile_end(h, buf, 32, ctypes.byref(n)))
    return {buf[k].name.decode(): (buf[k].launches, buf[k].total_ms) for k in range(n.value)}


def hydro_autotune(h: int, reps: int = 3, stream=None) -> list:
    """[(table, precision, threads, order, ms, tile rows, tile segment)] chosen per stage table."""
    buf = (hydro_tuning * 64)()
    n = ctypes.c_int()
    _check(load().hydro_autotune(h, int(reps), buf, 64, ctypes.byref(n), _stream(stream)))
    return [(buf[k].name.decode(), buf[k].precision, buf[k].threads, buf[k].order, buf[k].ms, buf[k].tile_rows,
             buf[k].tile_seg) for k in range(n.value)]


def hydro_set_neighbors(h: int, neighbors) -> None:
    """neighbors: int array [nboxes][6] of neighbour box indices (-1: boundary condition)."""
    nb = np.ascontiguousarray(neighbors, dtype=np.int32)
    _check(load().hydro_set_neighbors(h, nb.ctypes.data))


def hydro_set_shared_dt(h: int, enable: bool) -> None:
    _check(load().hydro_set_shared_dt(h, int(bool(enable))))


def hydro_set_method(h: int, limiter: int = 0, riemann: int = 0) -> None:
    """limiter: HYDRO_LIMITER_CW84 / HYDRO_LIMITER_CS08; riemann: HYDRO_RIEMANN_HLLC / HYDRO_RIEMANN_TWO_SHOCK."""
    _check(load().hydro_set_method(h, int(limiter), int(riemann)))


def hydro_fuse_tiles(h: int, enable: bool) -> None:
    _check(load().hydro_fuse_tiles(h, int(bool(enable))))


def hydro_set_tile_shape(h: int, rows: int, seg: int) -> None:
    """Tile rows (2 or 6) and z-planes per segment (0: the whole box) of the fused tile stage."""
    _check(load().hydro_set_tile_shape(h, int(rows), int(seg)))


def hydro_persistent(h: int, enable: bool) -> None:
    _check(load().hydro_persistent(h, int(bool(enable))))


def hydro_set_spin_limit(h: int, polls: int, stall_box: int = -1) -> None:
    _check(load().hydro_set_spin_limit(h, int(polls), int(stall_box)))


def hydro_use_graphs(h: int, enable: bool) -> None:
    _check(load().hydro_use_graphs(h, int(bool(enable))))


def hydro_fuse_lines(h: int, enable: bool) -> None:
    _check(load().hydro_fuse_lines(h, int(bool(enable))))


def hydro_compute_dt_noalloc(descs, state_dev, dt_dev, stream=None) -> None:
    """Per-box CFL time steps for states laid out as hydro_box_layout says,
    without a handle or caller scratch (the library's static scratch is used)."""
    _check(load().hydro_compute_dt_noalloc(desc_array(descs), len(descs), _ptr(state_dev), _ptr(dt_dev),
                                           _stream(stream)))


def hydro_measure_peaks(stream=None) -> dict:
    """Measured FP64 and FP32 multiply-add rates (flop/s) and the SM count."""
    f64, f32, sms = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    _check(load().hydro_measure_peaks(ctypes.byref(f64), ctypes.byref(f32), ctypes.byref(sms), _stream(stream)))
    return {"fp64_flops": f64.value, "fp32_flops": f32.value, "sms": sms.value}


def hydro_server_create(pool_dev, pool_bytes: int, max_active: int, dry_run: bool = False) -> int:
    cfg = hydro_server_config(_ptr(pool_dev), int(pool_bytes), int(max_active), int(bool(dry_run)))
    s = _VP()
    _check(load().hydro_server_create(ctypes.byref(cfg), ctypes.byref(s)))
    return s.value


def hydro_server_destroy(s: int) -> None:
    _check(load().hydro_server_destroy(s))


def hydro_submit(s: int, desc: hydro_box_desc, ic: np.ndarray, nsteps: int) -> int:
    ic = np.ascontiguousarray(ic, dtype=np.float64)
    req = hydro_request(desc, ic.ctypes.data, int(nsteps))
    t = ctypes.c_int64()
    _check(load().hydro_submit(s, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def hydro_poll(s: int, ticket: int, out: np.ndarray | None = None):
    """(status code, hydro_result); HYDRO_PENDING while the request runs.  A
    failed request returns its (negative) error code and does not raise."""
    info = hydro_result()
    ptr = out.ctypes.data if out is not None else None
    nbytes = out.nbytes if out is not None else 0
    rc = load().hydro_poll(s, int(ticket), ptr, nbytes, ctypes.byref(info))
    if rc < 0 and info.status == 0:
        raise HydroError(rc, hydro_last_error())
    return rc, info


def hydro_server_get_stats(s: int) -> dict:
    st = hydro_server_stats()
    _check(load().hydro_server_get_stats(s, ctypes.byref(st)))
    return {n: getattr(st, n) for n, _ in hydro_server_stats._fields_}


class Server:
    """A hydro server over a torch-allocated device pool (the memory budget)."""

    def __init__(self, pool_bytes: int, max_active: int = 256, device="cuda", dry_run: bool = False):
        import torch
        self.pool = None if dry_run else torch.empty((pool_bytes + 7) // 8, dtype=torch.float64, device=device)
        self.s = hydro_server_create(self.pool, pool_bytes, max_active, dry_run)

    def submit(self, problem, nsteps=None, precision=HYDRO_FP64) -> int:
        n = problem.nsteps if nsteps is None else nsteps
        return hydro_submit(self.s, desc_of(problem, precision), problem.U, n)

    def wait(self, ticket, shape, timeout=600.0):
        """Blocks until the request is done; returns (result array or None, hydro_result)."""
        import time
        nx, ny, nz = shape
        out = np.zeros((5, nz, ny, nx))
        t0 = time.monotonic()
        while True:
            rc, info = hydro_poll(self.s, ticket, out)
            if rc != HYDRO_PENDING:
                return (out if rc == HYDRO_OK else None), info
            if time.monotonic() - t0 > timeout:
                raise TimeoutError(f"ticket {ticket} not done after {timeout} s")
            time.sleep(0.0005)

    def stats(self) -> dict:
        return hydro_server_get_stats(self.s)

    def close(self):
        if self.s:
            hydro_server_destroy(self.s)
            self.s = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ convenience
class Boxes:
    """Owns torch-allocated state and scratch for a set of boxes and a handle."""

    def __init__(self, problems_or_descs, device="cuda", precision=HYDRO_FP64, limiter=0, riemann=0):
        import torch
        items = list(problems_or_descs)
        self.descs = [p if isinstance(p, hydro_box_desc) else desc_of(p, precision) for p in items]
        self.nboxes = len(self.descs)
        sb, wb = hydro_workspace_size(self.descs)
        self.state_bytes, self.scratch_bytes = sb, wb
        self.state = torch.empty((sb + 7) // 8, dtype=torch.float64, device=device)
        self.scratch = torch.empty((wb + 7) // 8, dtype=torch.float64, device=device)
        self.layouts = [hydro_box_layout(self.descs, b) for b in range(self.nboxes)]
        self.h = hydro_alloc(self.descs, self.state, sb, self.scratch, wb)
        if limiter or riemann:
            hydro_set_method(self.h, limiter, riemann)
        self.dt = torch.zeros(self.nboxes, dtype=torch.float64, device=device)
        for k, p in enumerate(items):
            if not isinstance(p, hydro_box_desc):
                self.set_interior(k, p.U)

    def close(self):
        if self.h:
            hydro_free(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shape(self, b):
        d = self.descs[b]
        return d.nx, d.ny, d.nz

    def state_view(self, b):
        """[5][nz+2g][ny+2g][nx+2g] strided view of box b's state (ghosts included)."""
        import torch
        lay = self.layouts[b]
        nx, ny, nz = self.shape(b)
        g = HYDRO_NG
        return torch.as_strided(self.state, (5, nz + 2 * g, ny + 2 * g, nx + 2 * g),
                                (lay.var_stride, lay.plane, lay.pitch, 1), lay.offset)

    def field_view(self, b, first, count=1):
        """Diagnostic view of `count` scratch fields of box b starting at field `first`
        (float64 for FP64 boxes, float32 for mixed-precision boxes)."""
        import torch
        off, nf, eb = hydro_debug_fields(self.descs, b)
        lay = self.layouts[b]
        nx, ny, nz = self.shape(b)
        g = HYDRO_NG
        base = self.scratch.view(torch.float32) if eb == 4 else self.scratch
        assert off % eb == 0
        return torch.as_strided(base, (count, nz + 2 * g, ny + 2 * g, nx + 2 * g),
                                (lay.var_stride, lay.plane, lay.pitch, 1), off // eb + first * lay.var_stride)

    def set_interior(self, b, U):
        import torch
        g = HYDRO_NG
        v = self.state_view(b)
        v[:, g:-g, g:-g, g:-g] = torch.as_tensor(np.ascontiguousarray(U), device=self.state.device)

    def interior(self, b) -> np.ndarray:
        g = HYDRO_NG
        return self.state_view(b)[:, g:-g, g:-g, g:-g].cpu().numpy()

    def ghosted(self, b) -> np.ndarray:
        return self.state_view(b).cpu().numpy()

    def fill_ghosts(self, stream=None):
        hydro_fill_ghosts(self.h, stream)

    def compute_dt(self, stream=None):
        hydro_compute_dt(self.h, self.dt, stream)
        return self.dt

    def step(self, nsteps=1, dt=None, stream=None):
        hydro_step(self.h, dt, nsteps, stream)

    def sync(self, stream=None):
        return hydro_sync(self.h, stream)

    def time(self, stream=None):
        return hydro_get_time(self.h, self.nboxes, stream)
