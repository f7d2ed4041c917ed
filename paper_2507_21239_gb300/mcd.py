"""Python binding of libmcd.so (include/mcd.h), argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: all of it runs in the CUDA kernels behind the C ABI.
torch provides the device workspace and the CUDA stream.  Loading fails
loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MCD_OK, MCD_EINVAL, MCD_ENOMEM, MCD_ECUDA, MCD_ENAN, MCD_ETIMEOUT, MCD_EEMPTY, MCD_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
MCD_FP64, MCD_MIXED = 0, 1
MCD_HOST, MCD_DEVICE = 0, 1
(MCD_OPT_MAX_EVENTS, MCD_OPT_CAP_STOPS, MCD_OPT_REBUILD_EVERY, MCD_OPT_USE_GRAPH, MCD_OPT_DUMP_R,
 MCD_OPT_LOG_CELL, MCD_OPT_LPT, MCD_OPT_THREADS, MCD_OPT_EXCLUSIVE, MCD_OPT_DV_MATRIX, MCD_OPT_TRACER,
 MCD_OPT_DT_MAX, MCD_OPT_COURANT, MCD_OPT_SWARMS_PER_THREAD, MCD_OPT_PERSISTENT, MCD_OPT_AUTOTUNE,
 MCD_OPT_EXACT_TOTAL, MCD_OPT_CONTROL_WARP) = range(1, 19)
MCD_MAX_TRIALS = 12
PREC = {"fp64": MCD_FP64, "mixed": MCD_MIXED}


class McdError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {mcd_strerror(code)} ({code})")
        self.code = code


class mcd_disk_params(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "sigma0", "p", "T0", "q", "alpha", "v_frag", "erosion_ratio",
        "dust_to_gas", "r_in", "r_out", "m_star", "rho_s", "a_mono",
        "mu", "sigma_h2", "dm_group", "frag_xi", "erosion_chi",
        "K_const", "V_const", "m_init", "M_total", "frag_ramp")] + [
        (n, C.c_int32) for n in ("kernel_mode", "settle_form", "dv_flags", "tr_flags")]
    OPTIONAL = {"frag_ramp": 0.0}  # keys a caller's dict may leave out

    @classmethod
    def from_dict(cls, d: dict) -> "mcd_disk_params":
        p = cls()
        for name, _ in cls._fields_:
            setattr(p, name, d[name] if name in d or name not in cls.OPTIONAL else cls.OPTIONAL[name])
        return p


class mcd_grid(C.Structure):
    _fields_ = [("n_r", C.c_int32), ("n_z", C.c_int32), ("per_cell", C.c_int32), ("reserved", C.c_int32)]


class mcd_stats(C.Structure):
    _fields_ = [("t", C.c_double), ("step", C.c_int64), ("events", C.c_int64), ("n_alive", C.c_int64),
                ("accreted_mass", C.c_double), ("status", C.c_int32), ("reserved", C.c_int32)]


class mcd_collide_class(C.Structure):
    _fields_ = [("n_lo", C.c_int32), ("n_hi", C.c_int32), ("cells", C.c_int64), ("threads", C.c_int32),
                ("swarms_per_thread", C.c_int32), ("store", C.c_int32), ("persistent", C.c_int32),
                ("control_warp", C.c_int32), ("tuned", C.c_int32), ("n_trials", C.c_int32),
                ("trial_swarms", C.c_int32 * MCD_MAX_TRIALS), ("trial_store", C.c_int32 * MCD_MAX_TRIALS),
                ("trial_control_warp", C.c_int32 * MCD_MAX_TRIALS),
                ("trial_us_per_event", C.c_float * MCD_MAX_TRIALS)]


class mcd_peaks(C.Structure):
    _fields_ = [("smem_gbs", C.c_double), ("fp32_tflops", C.c_double), ("fp64_tflops", C.c_double),
                ("sm_count", C.c_int32), ("sm_clock_mhz", C.c_int32), ("l2_bytes", C.c_int32),
                ("smem_per_sm_bytes", C.c_int32), ("ms_smem", C.c_float), ("ms_fp32", C.c_float),
                ("ms_fp64", C.c_float)]


_lib = None
_vp = C.c_void_p
_P = C.POINTER


def lib():
    """Load libmcd.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libmcd.so not found at {_build.LIB}; build it with __graft_entry__.build()")
        L = C.CDLL(_build.LIB)
        L.mcd_workspace_size.argtypes = [_P(mcd_disk_params), _P(mcd_grid), C.c_int32, C.c_int32, _P(C.c_size_t)]
        L.mcd_init_disk.argtypes = [_P(_vp), _P(mcd_disk_params), _P(mcd_grid), C.c_int32, C.c_uint64, C.c_int32,
                                    _vp, C.c_size_t, _vp]
        L.mcd_collide.argtypes = [_vp, C.c_double]
        L.mcd_transport.argtypes = [_vp, C.c_double]
        L.mcd_regrid.argtypes = [_vp]
        L.mcd_step.argtypes = [_vp, C.c_double]
        L.mcd_get_particles.argtypes = [_vp, C.c_int32, _vp, _vp, _vp, _vp, _vp, _P(C.c_int64), C.c_int32]
        L.mcd_set_particles.argtypes = [_vp, C.c_int32, _vp, _vp, _vp, _vp, _vp, C.c_int64, C.c_int32]
        L.mcd_get_cells.argtypes = [_vp, C.c_int32, _vp, _vp, _vp, C.c_int32]
        L.mcd_get_rates.argtypes = [_vp, C.c_int32, _vp, C.c_int32]
        L.mcd_get_total_rates.argtypes = [_vp, C.c_int32, _vp, C.c_int32]
        L.mcd_probe_peaks.argtypes = [_P(mcd_peaks), _vp]
        L.mcd_get_collide_classes.argtypes = [_vp, _P(mcd_collide_class), C.c_int32, _P(C.c_int32)]
        L.mcd_get_cell_events.argtypes = [_vp, C.c_int32, _vp, C.c_int32]
        L.mcd_get_event_log.argtypes = [_vp, _vp, _vp, _vp, C.c_int64, _P(C.c_int64)]
        L.mcd_get_stats.argtypes = [_vp, C.c_int32, _P(mcd_stats)]
        L.mcd_set_clock.argtypes = [_vp, C.c_double, C.c_int64]
        L.mcd_set_counters.argtypes = [_vp, C.c_int32, C.c_int64, C.c_double]
        L.mcd_get_tracer.argtypes = [_vp, C.c_int32, _vp, C.c_int32]
        L.mcd_set_tracer.argtypes = [_vp, C.c_int32, _vp, C.c_int32]
        L.mcd_moments.argtypes = [_vp, C.c_int32, C.c_int32, _vp, _vp]
        L.mcd_sigma_map.argtypes = [_vp, C.c_int32, C.c_int32, _vp, C.c_int32, _vp, _vp]
        L.mcd_set_gas_table.argtypes = [_vp, C.c_int32, C.c_int32, _vp, _vp, _vp]
        L.mcd_set_option.argtypes = [_vp, C.c_int32, C.c_double]
        L.mcd_trace.argtypes = [_vp, C.c_int32]
        L.mcd_trace_read.argtypes = [_vp, _P(C.c_float)]
        L.mcd_get_launch_count.argtypes = [_vp, _P(C.c_int64)]
        L.mcd_regrid_noalloc.argtypes = [_P(mcd_disk_params), _P(mcd_grid)] + [_vp] * 16 + [_vp]
        L.mcd_sync.argtypes = [_vp]
        L.mcd_free.argtypes = [_vp]
        L.mcd_strerror.argtypes = [C.c_int]
        L.mcd_strerror.restype = C.c_char_p
        L.mcd_pair_probe.argtypes = [_P(mcd_disk_params), C.c_int32, C.c_double, C.c_double, C.c_int64, _vp, _vp,
                                     _vp, _vp, _vp]
        L.mcd_rate_probe.argtypes = [_P(mcd_disk_params), C.c_int32, C.c_double, C.c_double, C.c_double, C.c_int32,
                                     _vp, _vp, _vp, _vp, _vp]
        _lib = L
    return _lib


def mcd_strerror(code: int) -> str:
    return lib().mcd_strerror(code).decode()


def _check(rc: int, what: str) -> int:
    if rc != MCD_OK:
        raise McdError(rc, what)
    return rc


def _arrays(params, grids):
    if isinstance(params, dict):
        params = [params]
    if isinstance(grids, (tuple, list)) and grids and isinstance(grids[0], int):
        grids = [grids]
    n = len(params)
    P = (mcd_disk_params * n)(*[mcd_disk_params.from_dict(p) for p in params])
    G = (mcd_grid * n)(*[mcd_grid(int(g[0]), int(g[1]), int(g[2]), 0) for g in grids])
    return P, G, n


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return int(t.data_ptr())


def mcd_workspace_size(params, grids, prec: int) -> int:
    P, G, n = _arrays(params, grids)
    b = C.c_size_t(0)
    _check(lib().mcd_workspace_size(P, G, n, prec, C.byref(b)), "mcd_workspace_size")
    return int(b.value)


def mcd_init_disk(params, grids, seed: int, prec: int, workspace, stream=None) -> int:
    """Returns the context handle; workspace is a caller-owned CUDA uint8 tensor."""
    P, G, n = _arrays(params, grids)
    h = _vp()
    _check(lib().mcd_init_disk(C.byref(h), P, G, n, seed, prec, _ptr(workspace), workspace.numel(),
                               _stream_ptr(stream)), "mcd_init_disk")
    return h.value


def mcd_collide(ctx: int, t_end: float):
    _check(lib().mcd_collide(ctx, t_end), "mcd_collide")


def mcd_transport(ctx: int, dt: float):
    _check(lib().mcd_transport(ctx, dt), "mcd_transport")


def mcd_regrid(ctx: int):
    _check(lib().mcd_regrid(ctx), "mcd_regrid")


def mcd_step(ctx: int, dt: float):
    _check(lib().mcd_step(ctx, dt), "mcd_step")


def mcd_get_particles(ctx: int, disk: int, m=None, M=None, r=None, z=None, id=None, where: int = MCD_HOST) -> int:
    n = C.c_int64(0)
    _check(lib().mcd_get_particles(ctx, disk, _ptr(m), _ptr(M), _ptr(r), _ptr(z), _ptr(id), C.byref(n), where),
           "mcd_get_particles")
    return int(n.value)


def mcd_set_particles(ctx: int, disk: int, m, M, r, z, id, where: int = MCD_HOST):
    count = len(m) if isinstance(m, np.ndarray) else m.numel()
    _check(lib().mcd_set_particles(ctx, disk, _ptr(m), _ptr(M), _ptr(r), _ptr(z), _ptr(id), count, where),
           "mcd_set_particles")


def mcd_get_cells(ctx: int, disk: int, cell_off, bounds, V):
    _check(lib().mcd_get_cells(ctx, disk, _ptr(cell_off), _ptr(bounds), _ptr(V), MCD_HOST), "mcd_get_cells")


def mcd_get_rates(ctx: int, disk: int, R, where: int = MCD_HOST):
    _check(lib().mcd_get_rates(ctx, disk, _ptr(R), where), "mcd_get_rates")


def mcd_get_total_rates(ctx: int, disk: int, Rtot, where: int = MCD_HOST):
    _check(lib().mcd_get_total_rates(ctx, disk, _ptr(Rtot), where), "mcd_get_total_rates")


def mcd_probe_peaks(stream=None) -> dict:
    """This GPU's shared-memory bandwidth and FP32/FP64 FMA throughput."""
    out = mcd_peaks()
    _check(lib().mcd_probe_peaks(C.byref(out), _stream_ptr(stream)), "mcd_probe_peaks")
    return {name: getattr(out, name) for name, _ in mcd_peaks._fields_}


def mcd_get_collide_classes(ctx: int) -> list[dict]:
    """The collide's cell classes and the variant each runs (host records)."""
    n = C.c_int32(0)
    _check(lib().mcd_get_collide_classes(ctx, None, 0, C.byref(n)), "mcd_get_collide_classes")
    buf = (mcd_collide_class * max(n.value, 1))()
    _check(lib().mcd_get_collide_classes(ctx, buf, n.value, C.byref(n)), "mcd_get_collide_classes")
    out = []
    for k in buf[:n.value]:
        t = k.n_trials
        out.append({"n_lo": k.n_lo, "n_hi": k.n_hi, "cells": k.cells, "threads": k.threads,
                    "swarms_per_thread": k.swarms_per_thread, "store": k.store, "persistent": k.persistent,
                    "control_warp": k.control_warp, "tuned": k.tuned,
                    "trials": [{"swarms_per_thread": k.trial_swarms[q], "store": k.trial_store[q],
                                "control_warp": k.trial_control_warp[q],
                                "us_per_event": k.trial_us_per_event[q]} for q in range(t)]})
    return out


def mcd_get_cell_events(ctx: int, disk: int, events, where: int = MCD_HOST):
    _check(lib().mcd_get_cell_events(ctx, disk, _ptr(events), where), "mcd_get_cell_events")


def mcd_get_event_log(ctx: int, cap: int):
    ijo = np.zeros((max(cap, 1), 3), np.int32)
    t = np.zeros(max(cap, 1))
    m = np.zeros(max(cap, 1))
    n = C.c_int64(0)
    _check(lib().mcd_get_event_log(ctx, ijo.ctypes.data, t.ctypes.data, m.ctypes.data, cap, C.byref(n)),
           "mcd_get_event_log")
    k = min(int(n.value), cap)
    return ijo[:k], t[:k], m[:k], int(n.value)


def mcd_get_stats(ctx: int, disk: int) -> mcd_stats:
    s = mcd_stats()
    _check(lib().mcd_get_stats(ctx, disk, C.byref(s)), "mcd_get_stats")
    return s


MCD_MAX_BINS = 1024


def mcd_moments(ctx: int, disk: int, edges) -> np.ndarray:
    """Per radial bin [edges[b], edges[b+1]) of the disk: (sum M, sum M m,
    sum M m^2, sum M m^3, count), an (nbins, 5) array (see include/mcd.h)."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    out = np.zeros((e.size - 1, 5))
    _check(lib().mcd_moments(ctx, disk, e.size - 1, e.ctypes.data, out.ctypes.data), "mcd_moments")
    return out


def mcd_sigma_map(ctx: int, disk: int, r_edges, m_edges) -> np.ndarray:
    """Swarm mass per (radial bin, mass bin) of the disk, an (nr, nm) array
    (see include/mcd.h)."""
    re = np.ascontiguousarray(r_edges, dtype=np.float64)
    me = np.ascontiguousarray(m_edges, dtype=np.float64)
    out = np.zeros((re.size - 1, me.size - 1))
    _check(lib().mcd_sigma_map(ctx, disk, re.size - 1, re.ctypes.data, me.size - 1, me.ctypes.data,
                               out.ctypes.data), "mcd_sigma_map")
    return out


MCD_MAX_GAS_KNOTS = 1024


def mcd_set_gas_table(ctx: int, disk: int, table):
    """The disk's gas tabulated in radius: table rows (r, Sigma_g, T), or None
    for the power laws (see include/mcd.h)."""
    if table is None:
        _check(lib().mcd_set_gas_table(ctx, disk, 0, None, None, None), "mcd_set_gas_table")
        return
    t = np.asarray(table, dtype=np.float64).reshape(-1, 3)
    r, S, T = (np.ascontiguousarray(t[:, k]) for k in range(3))
    _check(lib().mcd_set_gas_table(ctx, disk, t.shape[0], r.ctypes.data, S.ctypes.data, T.ctypes.data),
           "mcd_set_gas_table")


def mcd_get_tracer(ctx: int, disk: int, q, where: int = MCD_HOST):
    _check(lib().mcd_get_tracer(ctx, disk, _ptr(q), where), "mcd_get_tracer")


def mcd_set_tracer(ctx: int, disk: int, q, where: int = MCD_HOST):
    _check(lib().mcd_set_tracer(ctx, disk, _ptr(q), where), "mcd_set_tracer")


def mcd_set_clock(ctx: int, t: float, step: int):
    _check(lib().mcd_set_clock(ctx, t, step), "mcd_set_clock")


def mcd_set_counters(ctx: int, disk: int, events: int, accreted_mass: float):
    _check(lib().mcd_set_counters(ctx, disk, events, accreted_mass), "mcd_set_counters")


def mcd_set_option(ctx: int, key: int, value: float):
    _check(lib().mcd_set_option(ctx, key, float(value)), "mcd_set_option")


def mcd_trace(ctx: int, on: bool):
    _check(lib().mcd_trace(ctx, 1 if on else 0), "mcd_trace")


def mcd_trace_read(ctx: int) -> list[float]:
    """Phase durations of the last traced step [regrid, order, collide, transport] in ms."""
    ms = (C.c_float * 4)()
    _check(lib().mcd_trace_read(ctx, ms), "mcd_trace_read")
    return [float(x) for x in ms]


def mcd_get_launch_count(ctx: int) -> int:
    n = C.c_int64(0)
    _check(lib().mcd_get_launch_count(ctx, C.byref(n)), "mcd_get_launch_count")
    return int(n.value)


def mcd_sync(ctx: int) -> int:
    """Returns the latched device status (an MCD_* code); raises on CUDA errors."""
    rc = lib().mcd_sync(ctx)
    if rc == MCD_ECUDA:
        raise McdError(rc, "mcd_sync")
    return rc


def mcd_free(ctx: int):
    _check(lib().mcd_free(ctx), "mcd_free")


def mcd_regrid_noalloc(params: dict, grid, inputs, outputs, stream=None):
    """Context-free regrid of one disk that allocates nothing (device tensors).

    inputs: (m, M, r, z, id); outputs: (m, M, r, z, id, cell_start, cell_n,
    bounds, V, n_alive, status).  See include/mcd.h for the callers it serves
    and its limits."""
    P = mcd_disk_params.from_dict(params)
    G = mcd_grid(int(grid[0]), int(grid[1]), int(grid[2]), 0)
    args = [_ptr(t) for t in inputs] + [_ptr(t) for t in outputs]
    _check(lib().mcd_regrid_noalloc(C.byref(P), C.byref(G), *args, _stream_ptr(stream)), "mcd_regrid_noalloc")


def mcd_pair_probe(params: dict, prec: int, rc: float, zc: float, mi, mj, dv, K, stream=None):
    P = mcd_disk_params.from_dict(params)
    _check(lib().mcd_pair_probe(C.byref(P), prec, rc, zc, mi.numel(), _ptr(mi), _ptr(mj), _ptr(dv), _ptr(K),
                                _stream_ptr(stream)), "mcd_pair_probe")


def mcd_rate_probe(params: dict, prec: int, rc: float, zc: float, V: float, m, M, rate, R, stream=None):
    P = mcd_disk_params.from_dict(params)
    _check(lib().mcd_rate_probe(C.byref(P), prec, rc, zc, V, m.numel(), _ptr(m), _ptr(M), _ptr(rate), _ptr(R),
                                _stream_ptr(stream)), "mcd_rate_probe")


class Disk:
    """Convenience owner of one context and its workspace (one or more disks)."""

    def __init__(self, params, grids, seed: int = 0, prec: str | int = "mixed", stream=None, device="cuda"):
        import torch
        self.prec = PREC[prec] if isinstance(prec, str) else prec
        self.params, self.grids, self.n_disks = params, grids, len(_arrays(params, grids)[0])
        nbytes = mcd_workspace_size(params, grids, self.prec)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.stream = stream
        self.ctx = mcd_init_disk(params, grids, seed, self.prec, self.workspace, stream)
        for d, p in enumerate([params] if isinstance(params, dict) else params):
            if p.get("gas_table") is not None:  # after the initial draw, which keeps the power laws
                self.set_gas_table(p["gas_table"], d)

    def step(self, dt: float):
        mcd_step(self.ctx, dt)

    def particles(self, disk: int = 0) -> dict:
        g = self.grids[disk] if isinstance(self.grids[0], (tuple, list)) else self.grids
        n = int(g[0]) * int(g[1]) * int(g[2])
        out = {k: np.zeros(n) for k in ("m", "M", "r", "z")}
        out["id"] = np.zeros(n, np.uint32)
        mcd_get_particles(self.ctx, disk, out["m"], out["M"], out["r"], out["z"], out["id"], MCD_HOST)
        return out

    def particles_device(self, disk: int = 0) -> dict:
        """The disk's particles in cell order as CUDA tensors (m, M, r, z float64;
        id int32 holding the uint32 ids), copied on the device; the current torch
        stream is ordered after the copy."""
        import torch
        g = self.grids[disk] if isinstance(self.grids[0], (tuple, list)) else self.grids
        n = int(g[0]) * int(g[1]) * int(g[2])
        dev = self.workspace.device
        out = {k: torch.empty(n, dtype=torch.float64, device=dev) for k in ("m", "M", "r", "z")}
        out["id"] = torch.empty(n, dtype=torch.int32, device=dev)
        if self.stream is not None:
            self.stream.wait_stream(torch.cuda.current_stream())  # the fresh tensors before the copy
        mcd_get_particles(self.ctx, disk, out["m"], out["M"], out["r"], out["z"], out["id"], MCD_DEVICE)
        if self.stream is not None:
            torch.cuda.current_stream().wait_stream(self.stream)
        return out

    def stats(self, disk: int = 0) -> mcd_stats:
        return mcd_get_stats(self.ctx, disk)

    def tracer(self, disk: int = 0) -> np.ndarray:
        g = self.grids[disk] if isinstance(self.grids[0], (tuple, list)) else self.grids
        q = np.zeros(int(g[0]) * int(g[1]) * int(g[2]))
        mcd_get_tracer(self.ctx, disk, q)
        return q

    def set_tracer(self, q, disk: int = 0):
        mcd_set_tracer(self.ctx, disk, np.ascontiguousarray(q, dtype=np.float64))

    def set_gas_table(self, table, disk: int = 0):
        mcd_set_gas_table(self.ctx, disk, table)

    def moments(self, edges, disk: int = 0) -> np.ndarray:
        return mcd_moments(self.ctx, disk, edges)

    def sigma_map(self, r_edges, m_edges, disk: int = 0) -> np.ndarray:
        return mcd_sigma_map(self.ctx, disk, r_edges, m_edges)

    def close(self):
        if self.ctx:
            mcd_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
