"""Test infrastructure only: the plain FP64 CPU oracle (``mcd_oracle.c``).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It never imports the CUDA library or
its Python binding, and the CUDA library never imports it.

Every call marshals numpy arrays into the C oracle; no arithmetic of the
method lives here.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcd_oracle.c")
_LIB = os.path.join(_HERE, "libmcd_oracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENAN, ETIMEOUT = 0, -1, -4, -5
DV_BM, DV_TURB, DV_RAD, DV_PHI, DV_SET = 1, 2, 4, 8, 16
TR_RADIAL, TR_VERTICAL, TR_ST_MIDPLANE = 1, 2, 4


def compile_lib(src: str, out: str) -> str:
    """gcc -O2, FP contraction off, OpenMP on: src -> shared library out."""
    tmp = out + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            compile_lib(_SRC, _LIB)
    return _LIB


class Params(C.Structure):
    """Mirror of ``orc_params`` in mcd_oracle.c (oracle-side layout)."""

    _fields_ = [(n, C.c_double) for n in (
        "sigma0", "p", "T0", "q", "alpha", "v_frag", "erosion_ratio",
        "dust_to_gas", "r_in", "r_out", "m_star", "rho_s", "a_mono",
        "mu", "sigma_h2", "dm_group", "frag_xi", "erosion_chi",
        "K_const", "V_const", "m_init", "M_total", "frag_ramp")] + [
        (n, C.c_int32) for n in ("kernel_mode", "settle_form", "dv_flags", "tr_flags")] + [
        ("gas_tab", C.c_void_p), ("gas_n", C.c_int32)]

    OPTIONAL = {"frag_ramp": 0.0}  # keys a caller's dict may leave out

    @classmethod
    def from_dict(cls, d: dict) -> "Params":
        """d may hold "gas_table": rows (r, Sigma_g, T) of a tabulated gas disk."""
        p = cls()
        for name, _ in cls._fields_:
            if name in ("gas_tab", "gas_n"):
                continue
            setattr(p, name, d[name] if name in d or name not in cls.OPTIONAL else cls.OPTIONAL[name])
        tab = d.get("gas_table")
        if tab is not None:
            t = np.ascontiguousarray(tab, dtype=np.float64).reshape(-1, 3)
            p._tab = t  # kept alive with the structure
            p.gas_tab = t.ctypes.data
            p.gas_n = t.shape[0]
        else:
            p.gas_tab, p.gas_n = None, 0
        return p


class Event(C.Structure):
    _fields_ = [("i", C.c_int32), ("j", C.c_int32), ("outcome", C.c_int32), ("t", C.c_double),
                ("m_new", C.c_double)]


_P = C.POINTER
_d = _P(C.c_double)
_i64 = _P(C.c_int64)
_u32 = _P(C.c_uint32)
_u64 = _P(C.c_uint64)
_i32 = _P(C.c_int32)


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = load(_LIB)
    return _lib


def load(path: str):
    """The oracle library at path with its argument types declared (the
    tests also load copies built from altered source, to check that the pins
    catch planted mistakes)."""
    L = C.CDLL(path)
    L.orc_philox4x64_10.argtypes = [_u64, _u64, _u64]
    L.orc_gas_probe.argtypes = [_P(Params), C.c_int64, _d, _d, _d]
    L.orc_particle_probe.argtypes = [_P(Params), C.c_double, C.c_double, C.c_int64, _d, _d, _d, _i32]
    L.orc_pair_probe.argtypes = [_P(Params), C.c_double, C.c_double, C.c_int64, _d, _d, _d, _d, _d, _d]
    L.orc_rate_matrix.argtypes = [_P(Params), C.c_double, C.c_double, C.c_double, C.c_int64, _d, _d, _d, _d]
    L.orc_fragment_probe.argtypes = [_P(Params), C.c_double, C.c_double, C.c_double]
    L.orc_fragment_probe.restype = C.c_double
    L.orc_outcome_probe.argtypes = [_P(Params), C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                    _P(C.c_int32)]
    L.orc_outcome_probe.restype = C.c_double
    L.orc_disk_dust_mass.argtypes = [_P(Params)]
    L.orc_disk_dust_mass.restype = C.c_double
    L.orc_collide_cell.argtypes = [_P(Params), C.c_double, C.c_double, C.c_double, C.c_int64, _d, _d,
                                   C.c_double, C.c_double, C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64,
                                   C.c_int64, C.c_int64, _i64, _d, _P(Event), C.c_int64]
    L.orc_init_disk.argtypes = [_P(Params), C.c_int64, C.c_uint64, C.c_uint64, _d, _d, _d, _d, _u32]
    L.orc_regrid.argtypes = [_P(Params), C.c_int32, C.c_int32, C.c_int64, _d, _d, _d, _d, _u32, _i64, _i64,
                             _d, _d, _i64]
    L.orc_transport.argtypes = [_P(Params), C.c_int64, _d, _d, _d, _d, _u32, C.c_double, C.c_uint64,
                                C.c_uint64, C.c_uint64, _d]
    L.orc_collide_all.argtypes = [_P(Params), C.c_int32, C.c_int32, _i64, _d, _d, _d, _d, C.c_double,
                                  C.c_double, C.c_uint64, C.c_uint64, C.c_uint64, C.c_int64, C.c_int64,
                                  _i64, C.c_int32]
    L.orc_run.argtypes = [_P(Params), C.c_int32, C.c_int32, C.c_int64, _d, _d, _d, _d, _u32, C.c_double,
                          C.c_double, C.c_int64, C.c_int64, C.c_uint64, C.c_uint64, C.c_int64, C.c_int64,
                          _d, _i64, C.c_int32]
    L.orc_moments.argtypes = [C.c_int64, _d, _d, _d, C.c_int32, _d, _d]
    L.orc_tracer_update.argtypes = [_P(Params), C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                    C.c_int32]
    L.orc_tracer_update.restype = C.c_double
    L.orc_collide_cell_q.argtypes = [_P(Params), C.c_double, C.c_double, C.c_double, C.c_int64, _d, _d, _d,
                                     C.c_double, C.c_double, C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64,
                                     C.c_int64, C.c_int64, _i64, _d, _P(Event), C.c_int64]
    L.orc_run_q.argtypes = [_P(Params), C.c_int32, C.c_int32, C.c_int64, _d, _d, _d, _d, _u32, _d, C.c_double,
                            C.c_double, C.c_int64, C.c_int64, C.c_uint64, C.c_uint64, C.c_int64, C.c_int64,
                            _d, _i64, C.c_int32]
    L.orc_sigma_map.argtypes = [C.c_int64, _d, _d, _d, C.c_int32, _d, C.c_int32, _d, _d]
    L.orc_adaptive_dt.argtypes = [_P(Params), C.c_int64, _i64, _d, C.c_int64, _d, _d, _d, C.c_double,
                                  C.c_double]
    L.orc_adaptive_dt.restype = C.c_double
    L.orc_run_adaptive.argtypes = [_P(Params), C.c_int32, C.c_int32, C.c_int64, _d, _d, _d, _d, _u32, _d,
                                   C.c_double, C.c_double, C.c_double, C.c_int64, C.c_int64, C.c_uint64,
                                   C.c_uint64, C.c_int64, C.c_int64, _d, _i64, C.c_int32, _d]
    return L


def _ptr(a, ct):
    return a.ctypes.data_as(_P(ct)) if a is not None else None


YR = 3.15576e7  # Julian year [s] (the oracle's ORC_YR)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


NO_CAP = 1 << 62


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, np.uint64)
    lib().orc_philox4x64_10(_ptr(c, C.c_uint64), _ptr(k, C.c_uint64), _ptr(out, C.c_uint64))
    return out


GAS_FIELDS = ("Sigma", "T", "cs", "Omega", "H", "rho", "vth", "lambda", "nu", "etavk", "D", "vg2", "St_eta", "asw")


def gas(params: dict, r, z):
    r, z = _f64(np.atleast_1d(r)), _f64(np.atleast_1d(z))
    out = np.zeros((r.size, 14))
    P = Params.from_dict(params)
    lib().orc_gas_probe(C.byref(P), r.size, _ptr(r, C.c_double), _ptr(z, C.c_double), _ptr(out, C.c_double))
    return {k: out[:, i] for i, k in enumerate(GAS_FIELDS)}


def particle(params: dict, r: float, z: float, m):
    m = _f64(np.atleast_1d(m))
    a, St = np.zeros(m.size), np.zeros(m.size)
    stk = np.zeros(m.size, np.int32)
    P = Params.from_dict(params)
    lib().orc_particle_probe(C.byref(P), r, z, m.size, _ptr(m, C.c_double), _ptr(a, C.c_double),
                             _ptr(St, C.c_double), _ptr(stk, C.c_int32))
    return a, St, stk


def pairs(params: dict, rc: float, zc: float, mi, mj):
    mi, mj = _f64(np.atleast_1d(mi)), _f64(np.atleast_1d(mj))
    n = mi.size
    dv, K, dst = np.zeros(n), np.zeros(n), np.zeros(n)
    terms = np.zeros((n, 5))
    P = Params.from_dict(params)
    lib().orc_pair_probe(C.byref(P), rc, zc, n, _ptr(mi, C.c_double), _ptr(mj, C.c_double), _ptr(dv, C.c_double),
                         _ptr(K, C.c_double), _ptr(terms, C.c_double), _ptr(dst, C.c_double))
    return {"dv": dv, "K": K, "terms": terms, "dst": dst}


def rate_matrix(params: dict, rc: float, zc: float, V: float, m, M):
    m, M = _f64(m), _f64(M)
    n = m.size
    rate, R = np.zeros((n, n)), np.zeros(n)
    P = Params.from_dict(params)
    lib().orc_rate_matrix(C.byref(P), rc, zc, V, n, _ptr(m, C.c_double), _ptr(M, C.c_double),
                          _ptr(rate, C.c_double), _ptr(R, C.c_double))
    return rate, R


def fragment(params: dict, m0: float, mmax: float, u: float) -> float:
    P = Params.from_dict(params)
    return lib().orc_fragment_probe(C.byref(P), m0, mmax, u)


def disk_dust_mass(params: dict) -> float:
    P = Params.from_dict(params)
    return lib().orc_disk_dust_mass(C.byref(P))


def collide_cell(params: dict, rc, zc, V, m, M, t0, t_end, seed, disk, step, cell,
                 max_events=NO_CAP, rebuild_every=0, log_cap=0):
    """Run one cell's event loop; returns (status, m_new, events, R, log)."""
    m, M = _f64(m).copy(), _f64(M)
    n = m.size
    ev = np.zeros(1, np.int64)
    R = np.zeros(n)
    log = (Event * max(log_cap, 1))()
    P = Params.from_dict(params)
    st = lib().orc_collide_cell(C.byref(P), rc, zc, V, n, _ptr(m, C.c_double), _ptr(M, C.c_double), t0, t_end,
                                seed, disk, step, cell, max_events, rebuild_every, _ptr(ev, C.c_int64),
                                _ptr(R, C.c_double), log if log_cap > 0 else None, log_cap)
    k = int(min(ev[0], log_cap))
    lg = np.array([(log[e].i, log[e].j, log[e].outcome, log[e].t, log[e].m_new) for e in range(k)],
                  dtype=[("i", "i4"), ("j", "i4"), ("outcome", "i4"), ("t", "f8"), ("m_new", "f8")])
    return st, m, int(ev[0]), R, lg


class DiskState:
    """SoA particle state of one disk (oracle side)."""

    def __init__(self, m, M, r, z, id_, q=None):
        self.m, self.M, self.r, self.z = _f64(m).copy(), _f64(M).copy(), _f64(r).copy(), _f64(z).copy()
        self.id = np.ascontiguousarray(id_, dtype=np.uint32).copy()
        self.q = None if q is None else _f64(q).copy()  # optional tracer column
        self.accreted = 0.0
        self.events = 0

    def copy(self):
        s = DiskState(self.m, self.M, self.r, self.z, self.id, self.q)
        s.accreted, s.events = self.accreted, self.events
        return s


def init_disk(params: dict, N: int, seed: int, disk: int = 0) -> DiskState:
    m, M, r, z = (np.zeros(N) for _ in range(4))
    idv = np.zeros(N, np.uint32)
    P = Params.from_dict(params)
    lib().orc_init_disk(C.byref(P), N, seed, disk, _ptr(m, C.c_double), _ptr(M, C.c_double), _ptr(r, C.c_double),
                        _ptr(z, C.c_double), _ptr(idv, C.c_uint32))
    return DiskState(m, M, r, z, idv)


def regrid(params: dict, n_r: int, n_z: int, s: DiskState):
    """Regrid in place; returns (status, perm, cell_off, cell_b[ncell,6], cell_V, n_alive)."""
    N = s.m.size
    nc = n_r * n_z
    perm = np.zeros(N, np.int64)
    off = np.zeros(nc + 1, np.int64)
    cb = np.zeros((nc, 6))
    cv = np.zeros(nc)
    na = np.zeros(1, np.int64)
    P = Params.from_dict(params)
    st = lib().orc_regrid(C.byref(P), n_r, n_z, N, _ptr(s.m, C.c_double), _ptr(s.M, C.c_double),
                          _ptr(s.r, C.c_double), _ptr(s.z, C.c_double), _ptr(s.id, C.c_uint32),
                          _ptr(perm, C.c_int64), _ptr(off, C.c_int64), _ptr(cb, C.c_double), _ptr(cv, C.c_double),
                          _ptr(na, C.c_int64))
    if s.q is not None and st == 0:
        s.q = s.q[perm].copy()  # the tracer follows its particle
    return st, perm, off, cb, cv, int(na[0])


def transport(params: dict, s: DiskState, dt: float, seed: int, disk: int, step: int):
    acc = np.zeros(1)
    P = Params.from_dict(params)
    lib().orc_transport(C.byref(P), s.m.size, _ptr(s.r, C.c_double), _ptr(s.z, C.c_double), _ptr(s.m, C.c_double),
                        _ptr(s.M, C.c_double), _ptr(s.id, C.c_uint32), dt, seed, disk, step, _ptr(acc, C.c_double))
    s.accreted += float(acc[0])


def collide_all(params: dict, n_r, n_z, off, cb, cv, s: DiskState, t0, t_end, seed, disk, step,
                max_events=NO_CAP, rebuild_every=0, nthreads=0):
    ce = np.zeros(n_r * n_z, np.int64)
    P = Params.from_dict(params)
    st = lib().orc_collide_all(C.byref(P), n_r, n_z, _ptr(off, C.c_int64), _ptr(cb, C.c_double),
                               _ptr(cv, C.c_double), _ptr(s.m, C.c_double), _ptr(s.M, C.c_double), t0, t_end, seed,
                               disk, step, max_events, rebuild_every, _ptr(ce, C.c_int64), nthreads)
    s.events += int(ce.sum())
    return st, ce


def run(params: dict, n_r: int, n_z: int, s: DiskState, t0: float, dt: float, step0: int, n_steps: int,
        seed: int, disk: int = 0, max_events=NO_CAP, rebuild_every=0, nthreads=0, dt_max=None, courant=0.5,
        dts=None):
    """n_steps of regrid -> collide -> transport, in place; returns status.
    dt <= 0: the adaptive step, at most dt_max (default one year), each
    step's dt written to dts (an n_steps array) when given."""
    acc = np.zeros(1)
    ev = np.zeros(1, np.int64)
    P = Params.from_dict(params)
    if not dt > 0:
        out = np.zeros(n_steps) if dts is None else dts
        st = lib().orc_run_adaptive(C.byref(P), n_r, n_z, s.m.size, _ptr(s.m, C.c_double), _ptr(s.M, C.c_double),
                                    _ptr(s.r, C.c_double), _ptr(s.z, C.c_double), _ptr(s.id, C.c_uint32),
                                    _ptr(s.q, C.c_double), t0, YR if dt_max is None else dt_max, courant, step0,
                                    n_steps, seed, disk, max_events, rebuild_every, _ptr(acc, C.c_double),
                                    _ptr(ev, C.c_int64), nthreads, _ptr(out, C.c_double))
    elif s.q is None:
        st = lib().orc_run(C.byref(P), n_r, n_z, s.m.size, _ptr(s.m, C.c_double), _ptr(s.M, C.c_double),
                           _ptr(s.r, C.c_double), _ptr(s.z, C.c_double), _ptr(s.id, C.c_uint32), t0, dt, step0,
                           n_steps, seed, disk, max_events, rebuild_every, _ptr(acc, C.c_double),
                           _ptr(ev, C.c_int64), nthreads)
    else:
        st = lib().orc_run_q(C.byref(P), n_r, n_z, s.m.size, _ptr(s.m, C.c_double), _ptr(s.M, C.c_double),
                             _ptr(s.r, C.c_double), _ptr(s.z, C.c_double), _ptr(s.id, C.c_uint32),
                             _ptr(s.q, C.c_double), t0, dt, step0, n_steps, seed, disk, max_events, rebuild_every,
                             _ptr(acc, C.c_double), _ptr(ev, C.c_int64), nthreads)
    s.accreted += float(acc[0])
    s.events += int(ev[0])
    return st


def adaptive_dt(params: dict, cell_off, cell_b, s: DiskState, dt_max: float, courant: float = 0.5) -> float:
    """The adaptive step for the cells (cell_off, cell_b) of a regrid of s."""
    off = np.ascontiguousarray(cell_off, dtype=np.int64)
    cb = _f64(np.ascontiguousarray(cell_b).reshape(-1))
    P = Params.from_dict(params)
    return lib().orc_adaptive_dt(C.byref(P), off.size - 1, _ptr(off, C.c_int64), _ptr(cb, C.c_double), s.m.size,
                                 _ptr(s.m, C.c_double), _ptr(s.r, C.c_double), _ptr(s.z, C.c_double), dt_max,
                                 courant)


def moments(m, M, r, edges):
    """Per radial bin [edges[b], edges[b+1]): (sum M, sum M m, sum M m^2,
    sum M m^3, count) over the particles, an (nbins, 5) array."""
    m, M, r, edges = _f64(m), _f64(M), _f64(r), _f64(edges)
    nb = edges.size - 1
    out = np.zeros((nb, 5))
    lib().orc_moments(m.size, _ptr(m, C.c_double), _ptr(M, C.c_double), _ptr(r, C.c_double), nb,
                      _ptr(edges, C.c_double), _ptr(out, C.c_double))
    return out


def sigma_map(m, M, r, r_edges, m_edges):
    """Swarm mass per (radial bin, mass bin), an (nr, nm) array."""
    m, M, r = _f64(m), _f64(M), _f64(r)
    re, me = _f64(r_edges), _f64(m_edges)
    out = np.zeros((re.size - 1, me.size - 1))
    lib().orc_sigma_map(m.size, _ptr(m, C.c_double), _ptr(M, C.c_double), _ptr(r, C.c_double), re.size - 1,
                        _ptr(re, C.c_double), me.size - 1, _ptr(me, C.c_double), _ptr(out, C.c_double))
    return out


def outcome(params: dict, mi: float, mj: float, dv: float, m0: float, u: float):
    """(new mass of i, kind) for one event: 0 stick, 1 fragment, 2 erode."""
    k = C.c_int32(0)
    P = Params.from_dict(params)
    mn = lib().orc_outcome_probe(C.byref(P), mi, mj, dv, m0, u, C.byref(k))
    return mn, int(k.value)


def tracer_update(params: dict, mi, mj, qi, qj, mnew, kind) -> float:
    """The tracer of representative i after one event of the given kind."""
    P = Params.from_dict(params)
    return lib().orc_tracer_update(C.byref(P), mi, mj, qi, qj, mnew, kind)


def collide_cell_q(params: dict, rc, zc, V, m, M, q, t0, t_end, seed, disk, step, cell,
                   max_events=NO_CAP, rebuild_every=0, log_cap=0):
    """collide_cell carrying the tracer column; returns (status, m_new, q_new, events, R, log)."""
    m, M, q = _f64(m).copy(), _f64(M), _f64(q).copy()
    n = m.size
    ev = np.zeros(1, np.int64)
    R = np.zeros(n)
    log = (Event * max(log_cap, 1))()
    P = Params.from_dict(params)
    st = lib().orc_collide_cell_q(C.byref(P), rc, zc, V, n, _ptr(m, C.c_double), _ptr(M, C.c_double),
                                  _ptr(q, C.c_double), t0, t_end, seed, disk, step, cell, max_events, rebuild_every,
                                  _ptr(ev, C.c_int64), _ptr(R, C.c_double), log if log_cap > 0 else None, log_cap)
    k = int(min(ev[0], log_cap))
    lg = np.array([(log[e].i, log[e].j, log[e].outcome, log[e].t, log[e].m_new) for e in range(k)],
                  dtype=[("i", "i4"), ("j", "i4"), ("outcome", "i4"), ("t", "f8"), ("m_new", "f8")])
    return st, m, q, int(ev[0]), R, lg
