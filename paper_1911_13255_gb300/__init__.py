"""GB300-native multi-resolution SPH fluid-structure interaction (arXiv 1911.13255).

Thin ctypes binding over the C-ABI library ``libsphfsi.so`` (include/sphfsi.h).
Every step of the method runs in the library's CUDA kernels; this module only
marshals arguments.  There is no CPU fallback: if the library cannot be
built or loaded, importing :func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

__all__ = ["lib", "Simulation", "SphError", "library_path"]

_lock = threading.Lock()
_lib = None


class SphError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {lib().sphfsi_strerror(code).decode()} ({code})")


class Params(C.Structure):
    _fields_ = [("dim", C.c_int32), ("periodic_x", C.c_int32), ("gravity", C.c_double * 3),
                ("x_lo", C.c_double), ("Lx", C.c_double), ("free_surface", C.c_int32),
                ("n_reinit", C.c_int32), ("domain_lo", C.c_double * 3), ("domain_hi", C.c_double * 3),
                ("cell_reach", C.c_int32)]


class Inflow(C.Structure):
    _fields_ = [("on", C.c_int32), ("profile", C.c_int32), ("width", C.c_double), ("y0", C.c_double),
                ("H", C.c_double), ("U", C.c_double), ("t_ramp", C.c_double), ("period", C.c_double),
                ("womersley", C.c_double), ("z0", C.c_double), ("Hz", C.c_double)]


class Info(C.Structure):
    _fields_ = [("n_fluid", C.c_int64), ("n_solid", C.c_int64), ("n_wall", C.c_int64), ("n_cells", C.c_int64),
                ("step", C.c_int64), ("t", C.c_double), ("last_dt", C.c_double), ("last_K", C.c_int32),
                ("status", C.c_int32), ("pairs_ff", C.c_int64), ("pairs_fw", C.c_int64),
                ("pairs_fs", C.c_int64), ("pairs_sf", C.c_int64), ("pairs_ss", C.c_int64),
                ("pairs_total", C.c_int64), ("vmax_f", C.c_double), ("vmax_s", C.c_double),
                ("amax_s", C.c_double), ("mom_fs_fluid", C.c_double * 3), ("mom_fs_solid", C.c_double * 3),
                ("solid_path", C.c_int32), ("kernels_per_step", C.c_int32),
                ("learned_accepted", C.c_int64), ("learned_rejected", C.c_int64), ("learned_residual", C.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["mom_fs_fluid"] = np.array(self.mom_fs_fluid[:])
        d["mom_fs_solid"] = np.array(self.mom_fs_solid[:])
        return d


class Tuning(C.Structure):
    _fields_ = [("lanes", C.c_int32), ("block", C.c_int32), ("solid_variant", C.c_int32), ("step_ms", C.c_float),
                ("compact", C.c_int32), ("tile", C.c_int32), ("records", C.c_int32), ("rows", C.c_int32),
                ("list", C.c_int32), ("list_lanes", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp = C.c_void_p

# name -> (restype, argtypes)
_SIGS = {
    "sphfsi_create": (C.c_int, [C.POINTER(_vp), C.POINTER(Params), _vp]),
    "sphfsi_create_batch": (C.c_int, [C.POINTER(_vp), C.c_int32, C.POINTER(Params), _vp]),
    "sphfsi_select": (C.c_int, [_vp, C.c_int32]),
    "sphfsi_pairs_total": (C.c_int, [_vp, C.POINTER(C.c_int64)]),
    "sphfsi_get_solid_positions_all": (C.c_int, [_vp, _vp]),
    "sphfsi_get_solid_positions_async": (C.c_int, [_vp, _vp]),
    "sphfsi_set_tuning": (C.c_int, [_vp, C.POINTER(Tuning)]),
    "sphfsi_get_tuning": (C.c_int, [_vp, C.POINTER(Tuning)]),
    "sphfsi_autotune": (C.c_int, [_vp, C.c_double, C.c_int32, C.POINTER(Tuning)]),
    "sphfsi_add_fluid": (C.c_int, [_vp, C.c_int64, _vp, _vp, _vp, C.c_double, C.c_double, C.c_double, C.c_double]),
    "sphfsi_set_walls": (C.c_int, [_vp, C.c_int64, _vp, _vp, C.c_double]),
    "sphfsi_add_solid": (C.c_int, [_vp, C.c_int64, _vp, _vp, _vp, _vp, C.c_double, C.c_double, C.c_double,
                                   C.c_double]),
    "sphfsi_set_inflow": (C.c_int, [_vp, C.POINTER(Inflow)]),
    "sphfsi_finalize": (C.c_int, [_vp]),
    "sphfsi_set_substeps": (C.c_int, [_vp, C.c_int32]),
    "sphfsi_set_time_stepping": (C.c_int, [_vp, C.c_int32]),
    "sphfsi_set_advection_cadence": (C.c_int, [_vp, C.c_int32]),
    "sphfsi_set_wait_limit": (C.c_int, [_vp, C.c_int64]),
    "sphfsi_step": (C.c_int, [_vp, C.c_double]),
    "sphfsi_run": (C.c_int, [_vp, C.c_int64, C.c_double]),
    "sphfsi_sync": (C.c_int, [_vp]),
    "sphfsi_get_fluid": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "sphfsi_get_solid": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "sphfsi_set_fluid_state": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "sphfsi_set_solid_state": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "sphfsi_set_time": (C.c_int, [_vp, C.c_double, C.c_int64]),
    "sphfsi_get_info": (C.c_int, [_vp, C.POINTER(Info)]),
    "sphfsi_suggest_dt": (C.c_int, [_vp, _vp, _vp, _vp]),
    "sphfsi_state_size": (C.c_int, [_vp, _vp]),
    "sphfsi_get_state": (C.c_int, [_vp, _vp, C.c_int64]),
    "sphfsi_set_state": (C.c_int, [_vp, _vp, C.c_int64]),
    "sphfsi_debug_neighbors": (C.c_int, [_vp, C.c_int, _vp, _vp, C.POINTER(C.c_int64)]),
    "sphfsi_set_profiling": (C.c_int, [_vp, C.c_int]),
    "sphfsi_set_solid_path": (C.c_int, [_vp, C.c_int]),
    "sphfsi_stage_times": (C.c_int, [_vp, _vp, C.c_int]),
    "sphfsi_step_time": (C.c_int, [_vp, _vp]),
    "sphfsi_neighbor_counts_noalloc": (C.c_int, [C.POINTER(Params), C.c_int64, _vp, C.c_double, _vp, _vp]),
    "sphfsi_gemm_bf16": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int64, C.c_int64, C.c_int64, _vp]),
    "sphfsi_tc_status": (C.c_int, [C.POINTER(C.c_int32), C.c_int32]),
    "sphfsi_solid_graph": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "sphfsi_set_learned": (C.c_int, [_vp, _vp, _vp, C.c_double]),
    "sphfsi_get_learned_features": (C.c_int, [_vp, _vp]),
    "sphfsi_mpnn_n_params": (C.c_int64, [C.c_int32]),
    "sphfsi_mpnn_create": (C.c_int, [C.POINTER(_vp), C.c_int32, C.c_int64, C.c_int64, _vp, _vp, _vp, _vp, C.c_int32,
                                     _vp]),
    "sphfsi_mpnn_set_params": (C.c_int, [_vp, _vp]),
    "sphfsi_mpnn_get_params": (C.c_int, [_vp, _vp]),
    "sphfsi_mpnn_forward": (C.c_int, [_vp, _vp, _vp]),
    "sphfsi_mpnn_backward": (C.c_int, [_vp, _vp, _vp]),
    "sphfsi_mpnn_train_step": (C.c_int, [_vp, _vp, _vp, _vp, C.c_float, _vp]),
    "sphfsi_mpnn_sync": (C.c_int, [_vp]),
    "sphfsi_mpnn_destroy": (None, [_vp]),
    "sphfsi_destroy": (None, [_vp]),
    "sphfsi_strerror": (C.c_char_p, [C.c_int]),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """Load (building first if stale) the CUDA library; raises if impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc, what):
    if rc != 0:
        raise SphError(rc, what)


def _ptr(a):
    """Address of a contiguous numpy array or a torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr()
    assert a.flags.c_contiguous
    return a.ctypes.data


def _f64(a, shape=None):
    if hasattr(a, "data_ptr"):   # torch tensor (host, pinned or device): passed through
        import torch
        assert a.dtype == torch.float64 and a.is_contiguous()
        return a if shape is None else a.reshape(shape)
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a if shape is None else a.reshape(shape)


def _params(dim, gravity=(0, 0, 0), periodic_x=0, x_lo=0.0, Lx=0.0, free_surface=0, n_reinit=0,
            domain_lo=(0, 0, 0), domain_hi=(1, 1, 1), cell_reach=1):
    p = Params()
    p.dim, p.periodic_x, p.x_lo, p.Lx = dim, int(periodic_x), float(x_lo), float(Lx)
    p.free_surface, p.n_reinit = int(free_surface), int(n_reinit)
    p.cell_reach = int(cell_reach)
    for k in range(3):
        p.gravity[k] = float(gravity[k]) if k < len(gravity) else 0.0
        p.domain_lo[k] = float(domain_lo[k]) if k < len(domain_lo) else 0.0
        p.domain_hi[k] = float(domain_hi[k]) if k < len(domain_hi) else 1.0
    return p


def _case_params(case):
    return _params(case.dim, case.gravity, case.periodic_x, case.x_lo, case.Lx, case.free_surface,
                   case.n_reinit, case.domain_lo, case.domain_hi, getattr(case, "cell_reach", 1))


def _stream_handle(stream):
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Simulation:
    """One FSI problem, or a batch of independent ones, on the current CUDA
    device (see include/sphfsi.h).  Per-instance calls act on the instance
    chosen by select()."""

    def __init__(self, dim, gravity=(0, 0, 0), periodic_x=0, x_lo=0.0, Lx=0.0, free_surface=0,
                 n_reinit=0, domain_lo=(0, 0, 0), domain_hi=(1, 1, 1), stream=None, params=None):
        L = lib()
        if params is None:
            params = [_params(dim, gravity, periodic_x, x_lo, Lx, free_surface, n_reinit, domain_lo, domain_hi)]
        arr = (Params * len(params))(*params)
        self._stream = stream
        h = _vp()
        _check(L.sphfsi_create_batch(C.byref(h), len(params), arr, _stream_handle(stream)), "sphfsi_create_batch")
        self.h = h
        self.dim = dim
        self.n_instances = len(params)
        self._sel = 0
        self._counts = [[0, 0, 0] for _ in params]   # nf, ns, nw per instance

    @property
    def nf(self):
        return self._counts[self._sel][0]

    @property
    def ns(self):
        return self._counts[self._sel][1]

    @property
    def nw(self):
        return self._counts[self._sel][2]

    def select(self, b):
        """Address instance b with the per-instance calls."""
        _check(lib().sphfsi_select(self.h, int(b)), "sphfsi_select")
        self._sel = int(b)
        return self

    # --- set-up -----------------------------------------------------------
    def add_fluid(self, r, v, p_init, dp, rho0, c0, eta):
        r, v = _f64(r), _f64(v)
        p = None if p_init is None else _f64(p_init)
        self._counts[self._sel][0] = len(r)
        _check(lib().sphfsi_add_fluid(self.h, self.nf, _ptr(r), _ptr(v), _ptr(p), dp, rho0, c0, eta),
               "sphfsi_add_fluid")

    def set_walls(self, r, nrm, dp):
        r, nrm = _f64(r), _f64(nrm)
        self._counts[self._sel][2] = len(r)
        _check(lib().sphfsi_set_walls(self.h, self.nw, _ptr(r), _ptr(nrm), dp), "sphfsi_set_walls")

    def add_solid(self, r0, v0, n0, constrained, dp, rho0, E, nu):
        r0, v0, n0 = _f64(r0), _f64(v0), _f64(n0)
        cons = np.ascontiguousarray(np.asarray(constrained, np.uint8))
        self._counts[self._sel][1] = len(r0)
        _check(lib().sphfsi_add_solid(self.h, self.ns, _ptr(r0), _ptr(v0), _ptr(n0), _ptr(cons), dp, rho0, E,
                                      nu), "sphfsi_add_solid")

    def set_inflow(self, on, profile, width, y0, H, U, t_ramp, period=0.0, womersley=0.0, z0=0.0, Hz=0.0):
        f = Inflow(int(on), int(profile), float(width), float(y0), float(H), float(U), float(t_ramp),
                   float(period), float(womersley), float(z0), float(Hz))
        _check(lib().sphfsi_set_inflow(self.h, C.byref(f)), "sphfsi_set_inflow")

    def finalize(self):
        _check(lib().sphfsi_finalize(self.h), "sphfsi_finalize")
        return self

    def _add_case(self, case):
        self.add_fluid(case.f_r, case.f_v, case.f_p, case.f_dp, case.f_rho0, case.f_c0, case.f_eta)
        if case.nw:
            self.set_walls(case.w_r, case.w_n, case.w_dp)
        if case.ns:
            self.add_solid(case.s_r0, case.s_v0, case.s_n0, case.s_cons, case.s_dp, case.s_rho0, case.s_E,
                           case.s_nu)
        if case.inflow_on:
            self.set_inflow(1, case.inflow_profile, case.inflow_width, case.inflow_y0, case.inflow_H,
                            case.inflow_U, case.inflow_tramp, getattr(case, "inflow_period", 0.0),
                            getattr(case, "inflow_wo", 0.0), getattr(case, "inflow_z0", 0.0),
                            getattr(case, "inflow_Hz", 0.0))

    @classmethod
    def from_case(cls, case, stream=None):
        """Build from any object with the attributes of a test/bench case."""
        s = cls(case.dim, stream=stream, params=[_case_params(case)])
        s._add_case(case)
        return s.finalize()

    @classmethod
    def from_cases(cls, cases, stream=None):
        """One batched context holding every case as an independent instance."""
        cases = list(cases)
        s = cls(cases[0].dim, stream=stream, params=[_case_params(c) for c in cases])
        for b, case in enumerate(cases):
            s.select(b)
            s._add_case(case)
        s.finalize()
        return s.select(0)

    def autotune(self, dt=0.0, steps=10):
        """Pick the fastest launch shape on this workload (state left unchanged)."""
        t = Tuning()
        _check(lib().sphfsi_autotune(self.h, float(dt), int(steps), C.byref(t)), "sphfsi_autotune")
        return t.as_dict()

    def set_tuning(self, lanes, block=128, solid_variant=0, compact=None, tile=0, records=None, rows=None,
                   list=None, list_lanes=0):
        """Launch shape (include/sphfsi.h, sphfsi_tuning); compact, records,
        rows and list default to the current setting (rows and list are 0
        with tiles)."""
        cur = self.tuning()
        if compact is None:
            compact = cur["compact"]
        if records is None:
            records = cur["records"]
        if rows is None:
            rows = 0 if tile else cur["rows"]
        if list is None:
            list = 0 if tile else cur["list"]
        t = Tuning(int(lanes), int(block), int(solid_variant), 0.0, int(compact), int(tile), int(records), int(rows),
                   int(list), int(list_lanes))
        _check(lib().sphfsi_set_tuning(self.h, C.byref(t)), "sphfsi_set_tuning")

    def tuning(self):
        t = Tuning()
        _check(lib().sphfsi_get_tuning(self.h, C.byref(t)), "sphfsi_get_tuning")
        return t.as_dict()

    def solid_graph(self):
        """(ptr, idx, w, g) of the selected instance's body, original order."""
        n = self.ns
        nnz = self.info()["pairs_ss"]
        ptr = np.zeros(n + 1, np.int64)
        idx = np.zeros(max(nnz, 1), np.int64)
        w = np.zeros(max(nnz, 1))
        g = np.zeros((max(nnz, 1), self.dim))
        _check(lib().sphfsi_solid_graph(self.h, _ptr(ptr), _ptr(idx), _ptr(w), _ptr(g)), "sphfsi_solid_graph")
        return ptr, idx[:nnz], w[:nnz], g[:nnz]

    def set_learned(self, theta, scales, tol):
        """Learned sub-stepper with parameters theta and scales
        (s_u, s_v, s_f, s_t, s_du, s_dv, s_H); tol < 0 switches it off."""
        th = np.ascontiguousarray(theta, np.float32)
        sc = np.ascontiguousarray(scales, np.float64)
        _check(lib().sphfsi_set_learned(self.h, _ptr(th), _ptr(sc), float(tol)), "sphfsi_set_learned")

    def learned_features(self):
        """Input rows (n_solid x 64, original order) the last learned step fed the network."""
        x = np.zeros((self.ns, 64), np.float32)
        _check(lib().sphfsi_get_learned_features(self.h, _ptr(x)), "sphfsi_get_learned_features")
        return x

    def pairs_total(self):
        """Pair interactions of all instances since creation."""
        t = C.c_int64()
        _check(lib().sphfsi_pairs_total(self.h, C.byref(t)), "sphfsi_pairs_total")
        return t.value

    # --- stepping ---------------------------------------------------------
    def set_substeps(self, K):
        _check(lib().sphfsi_set_substeps(self.h, int(K)), "sphfsi_set_substeps")

    TIME_STEPPING = {"multiple": 0, "single": 1, "single_solid": 2}

    def set_time_stepping(self, mode):
        """"multiple" (kappa sub-steps), "single" (Section 2.2 criterion,
        K = 1) or "single_solid" (min(dt_ac, dt_S), K = 1)."""
        m = self.TIME_STEPPING[mode] if isinstance(mode, str) else int(mode)
        _check(lib().sphfsi_set_time_stepping(self.h, m), "sphfsi_set_time_stepping")

    def set_advection_cadence(self, n):
        """Hold the pair configuration over n coarse steps (Algorithm 1); 1 rebuilds it every step;
        0 or "auto": over the advection steps of the advection criterion (Eq. dtf-advection)."""
        n = 0 if n == "auto" else int(n)
        _check(lib().sphfsi_set_advection_cadence(self.h, n), "sphfsi_set_advection_cadence")

    def set_wait_limit(self, iterations):
        """Polling iterations before a bounded device wait gives up (0: the default)."""
        _check(lib().sphfsi_set_wait_limit(self.h, int(iterations)), "sphfsi_set_wait_limit")

    def step(self, dt=0.0):
        _check(lib().sphfsi_step(self.h, float(dt)), "sphfsi_step")

    def run(self, nsteps, dt=0.0):
        _check(lib().sphfsi_run(self.h, int(nsteps), float(dt)), "sphfsi_run")

    def sync(self):
        _check(lib().sphfsi_sync(self.h), "sphfsi_sync")

    # --- state ------------------------------------------------------------
    def get_fluid(self):
        d, n = self.dim, self.nf
        r = np.zeros((n, d))
        v = np.zeros((n, d), np.float32)
        rho = np.zeros(n)
        rd = np.zeros(n, np.float32)
        a = np.zeros((n, d), np.float32)
        _check(lib().sphfsi_get_fluid(self.h, _ptr(r), _ptr(v), _ptr(rho), _ptr(rd), _ptr(a)),
               "sphfsi_get_fluid")
        return dict(r=r, v=v, rho=rho, drho=rd, dvdt=a)

    def get_solid(self):
        d, n = self.dim, self.ns
        r = np.zeros((n, d))
        v = np.zeros((n, d), np.float32)
        F = np.zeros((n, d, d))
        vb = np.zeros((n, d))
        ab = np.zeros((n, d))
        fF = np.zeros((n, d), np.float32)
        nrm = np.zeros((n, d), np.float32)
        _check(lib().sphfsi_get_solid(self.h, _ptr(r), _ptr(v), _ptr(F), _ptr(vb), _ptr(ab), _ptr(fF),
                                      _ptr(nrm)), "sphfsi_get_solid")
        return dict(r=r, v=v, F=F, vbar=vb, abar=ab, fF=fF, nrm=nrm)

    def get_solid_positions(self, out):
        """Solid positions into a caller buffer (numpy host array or CUDA tensor), n x dim FP64."""
        _check(lib().sphfsi_get_solid(self.h, _ptr(out), None, None, None, None, None, None),
               "sphfsi_get_solid")
        return out

    def get_solid_positions_all(self, out):
        """Solid positions of all instances (concatenated, original order) into a caller buffer."""
        _check(lib().sphfsi_get_solid_positions_all(self.h, _ptr(out)), "sphfsi_get_solid_positions_all")
        return out

    def get_solid_positions_async(self, out):
        """The same rows enqueued on the context's stream without waiting; `out`
        (a pinned host tensor for a copy that overlaps later steps) is complete
        once the stream has reached the copy (sync, or an event recorded after)."""
        _check(lib().sphfsi_get_solid_positions_async(self.h, _ptr(out)), "sphfsi_get_solid_positions_async")
        return out

    def set_fluid_state(self, r=None, v=None, rho=None, drho=None):
        args = [None if x is None else _f64(x) for x in (r, v, rho, drho)]
        _check(lib().sphfsi_set_fluid_state(self.h, *[_ptr(x) for x in args]), "sphfsi_set_fluid_state")

    def set_solid_state(self, r=None, v=None, F=None, vbar=None, abar=None, nrm=None):
        args = [None if x is None else _f64(x) for x in (r, v, F, vbar, abar, nrm)]
        _check(lib().sphfsi_set_solid_state(self.h, *[_ptr(x) for x in args]), "sphfsi_set_solid_state")

    def set_time(self, t, step):
        _check(lib().sphfsi_set_time(self.h, float(t), int(step)), "sphfsi_set_time")

    def suggest_dt(self):
        """(dt_ac, dt_ad, dt_S) of the selected instance (include/sphfsi.h)."""
        out = [C.c_double(), C.c_double(), C.c_double()]
        _check(lib().sphfsi_suggest_dt(self.h, *[C.byref(o) for o in out]), "sphfsi_suggest_dt")
        return tuple(o.value for o in out)

    def get_state(self):
        """The whole device state as bytes (a checkpoint)."""
        n = C.c_int64()
        _check(lib().sphfsi_state_size(self.h, C.byref(n)), "sphfsi_state_size")
        buf = np.empty(n.value, np.uint8)
        _check(lib().sphfsi_get_state(self.h, _ptr(buf), n.value), "sphfsi_get_state")
        return buf.tobytes()

    def set_state(self, blob):
        """Restore a checkpoint taken from a context built the same way."""
        buf = np.frombuffer(bytes(blob), np.uint8)
        _check(lib().sphfsi_set_state(self.h, _ptr(buf), buf.size), "sphfsi_set_state")

    def info(self):
        i = Info()
        _check(lib().sphfsi_get_info(self.h, C.byref(i)), "sphfsi_get_info")
        return i.as_dict()

    STAGES = ("bin_sort", "reinit", "momentum", "solid_fluid_force",
              "continuity", "solid_substeps", "finish", "neighbour_rows")

    def set_solid_path(self, path):
        """0 automatic (cluster-resident when the body fits), 2 cooperative grid."""
        _check(lib().sphfsi_set_solid_path(self.h, int(path)), "sphfsi_set_solid_path")

    def set_profiling(self, on=True):
        _check(lib().sphfsi_set_profiling(self.h, int(bool(on))), "sphfsi_set_profiling")

    def stage_times(self):
        """Device ms of the last step's stages (needs set_profiling(True))."""
        ms = np.zeros(len(self.STAGES), np.float32)
        rc = lib().sphfsi_stage_times(self.h, _ptr(ms), len(self.STAGES))
        if rc < 0:
            _check(rc, "sphfsi_stage_times")
        return dict(zip(self.STAGES, ms.tolist()))

    def step_time(self):
        """Device ms of the whole last step (needs set_profiling(True))."""
        ms = np.zeros(1, np.float32)
        _check(lib().sphfsi_step_time(self.h, _ptr(ms)), "sphfsi_step_time")
        return float(ms[0])

    def debug_neighbors(self, which):
        """(ptr, idx) neighbour CSR in original order with the FP64 support test."""
        nrows = self.ns if which == 3 else self.nf
        nnz = C.c_int64()
        ptr = np.zeros(nrows + 1, np.int64)
        _check(lib().sphfsi_debug_neighbors(self.h, which, _ptr(ptr), None, C.byref(nnz)),
               "sphfsi_debug_neighbors")
        idx = np.zeros(max(nnz.value, 1), np.int64)
        _check(lib().sphfsi_debug_neighbors(self.h, which, _ptr(ptr), _ptr(idx), C.byref(nnz)),
               "sphfsi_debug_neighbors")
        return ptr, idx[:nnz.value]

    def close(self):
        if getattr(self, "h", None):
            lib().sphfsi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gemm_bf16(A, B, bias=None, out=None, stream=None):
    """C = A . B^T (+ bias) on the tensor cores: A (M x K), B (N x K) bfloat16
    CUDA tensors, C FP32 (M x N); M % 128 == 0, N % 16 == 0, K % 64 == 0."""
    import torch
    assert A.dtype == torch.bfloat16 and B.dtype == torch.bfloat16 and A.is_cuda and B.is_cuda
    M, K = A.shape
    N = B.shape[0]
    if out is None:
        out = torch.empty((M, N), dtype=torch.float32, device=A.device)
    _check(lib().sphfsi_gemm_bf16(_ptr(A.contiguous()), _ptr(B.contiguous()), _ptr(bias), _ptr(out), M, N, K,
                                  _stream_handle(stream)), "sphfsi_gemm_bf16")
    return out


def tc_status(reset=False):
    s = C.c_int32()
    _check(lib().sphfsi_tc_status(C.byref(s), int(bool(reset))), "sphfsi_tc_status")
    return s.value


class Mpnn:
    """The learned sub-stepper's network over one body's graph, replicated
    `replicas` times (see include/sphfsi.h).  Arrays may be numpy (host) or
    CUDA tensors; FP32 for x, out, targets, parameters."""

    FIN, NOUT, C = 64, 16, 128

    def __init__(self, dim, graph, replicas=1, stream=None):
        ptr, idx, w, g = graph
        self.dim, self.n, self.replicas = dim, len(ptr) - 1, int(replicas)
        self._g = [np.ascontiguousarray(ptr, np.int64), np.ascontiguousarray(idx, np.int64),
                   np.ascontiguousarray(w, np.float64), np.ascontiguousarray(g, np.float64)]
        self._stream = stream
        h = _vp()
        _check(lib().sphfsi_mpnn_create(C.byref(h), dim, self.n, len(self._g[1]), *[_ptr(a) for a in self._g],
                                        self.replicas, _stream_handle(stream)), "sphfsi_mpnn_create")
        self.h = h
        self.n_params = int(lib().sphfsi_mpnn_n_params(dim))

    def set_params(self, theta):
        t = np.ascontiguousarray(theta, np.float32) if not hasattr(theta, "data_ptr") else theta
        _check(lib().sphfsi_mpnn_set_params(self.h, _ptr(t)), "sphfsi_mpnn_set_params")

    def get_params(self):
        t = np.zeros(self.n_params, np.float32)
        _check(lib().sphfsi_mpnn_get_params(self.h, _ptr(t)), "sphfsi_mpnn_get_params")
        return t

    def forward(self, x):
        x = np.ascontiguousarray(x, np.float32) if not hasattr(x, "data_ptr") else x
        out = np.zeros((self.n * self.replicas, self.NOUT), np.float32)
        _check(lib().sphfsi_mpnn_forward(self.h, _ptr(x), _ptr(out)), "sphfsi_mpnn_forward")
        self.sync()
        return out

    def backward(self, dout):
        d = np.ascontiguousarray(dout, np.float32)
        grad = np.zeros(self.n_params, np.float32)
        _check(lib().sphfsi_mpnn_backward(self.h, _ptr(d), _ptr(grad)), "sphfsi_mpnn_backward")
        self.sync()
        return grad

    def train_step(self, x, target, mask=None, lr=1e-3):
        conv = lambda a, dt: a if (a is None or hasattr(a, "data_ptr")) else np.ascontiguousarray(a, dt)
        x, target, mask = conv(x, np.float32), conv(target, np.float32), conv(mask, np.uint8)
        loss = np.zeros(1, np.float32)
        _check(lib().sphfsi_mpnn_train_step(self.h, _ptr(x), _ptr(target), _ptr(mask), float(lr), _ptr(loss)),
               "sphfsi_mpnn_train_step")
        self.sync()
        return float(loss[0])

    def sync(self):
        _check(lib().sphfsi_mpnn_sync(self.h), "sphfsi_mpnn_sync")

    def close(self):
        if getattr(self, "h", None):
            lib().sphfsi_mpnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
