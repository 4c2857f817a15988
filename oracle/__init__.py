"""FP64 CPU oracle for the multi-resolution SPH FSI method (arXiv 1911.13255).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow reference the GPU
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the benchmark's ``cpu_baseline`` / ``--impl reference`` legs may import it; the
product package never does, and the two share no code.

The arithmetic lives in ``sph_oracle.c`` (plain C, FP64, no FMA contraction,
single threaded); this module compiles it with gcc and drives it through
ctypes on numpy arrays in original particle order.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libsph_oracle.so")
_LIB_OMP = os.path.join(_HERE, "_build", "libsph_oracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None


def _build_one(path, extra, force):
    if force or not os.path.exists(path) or os.path.getmtime(path) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "sph_oracle.h"))):
        tmp = path + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared"] + extra +
                              ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, FP64, -ffp-contract=off): the plain
    single-threaded library and the OpenMP build of the same source that the
    benchmark times on all host cores."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    _build_one(_LIB_OMP, ["-fopenmp"], force)
    return _build_one(_LIB, [], force)


class Params(C.Structure):
    _fields_ = [("dim", C.c_int32), ("periodic_x", C.c_int32), ("g", C.c_double * 3),
                ("x_lo", C.c_double), ("Lx", C.c_double), ("free_surface", C.c_int32),
                ("n_reinit", C.c_int32), ("inflow_on", C.c_int32), ("inflow_profile", C.c_int32),
                ("inflow_width", C.c_double), ("inflow_y0", C.c_double), ("inflow_H", C.c_double),
                ("inflow_U", C.c_double), ("inflow_tramp", C.c_double), ("inflow_period", C.c_double),
                ("inflow_wo", C.c_double), ("inflow_z0", C.c_double), ("inflow_Hz", C.c_double)]


_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)


class Fluid(C.Structure):
    _fields_ = [("n", C.c_int64), ("dp", C.c_double), ("rho0", C.c_double), ("c0", C.c_double),
                ("eta", C.c_double), ("r", _dp), ("v", _dp), ("rho", _dp), ("drho", _dp),
                ("dvdt", _dp)]


class Wall(C.Structure):
    _fields_ = [("n", C.c_int64), ("dp", C.c_double), ("r", _dp), ("nrm", _dp)]


class Solid(C.Structure):
    _fields_ = [("n", C.c_int64), ("dp", C.c_double), ("rho0", C.c_double), ("E", C.c_double),
                ("nu", C.c_double), ("cons", C.POINTER(C.c_uint8)),
                ("r0", _dp), ("n0", _dp), ("r", _dp), ("v", _dp), ("F", _dp), ("Fdot", _dp),
                ("B0", _dp), ("nrm", _dp), ("vbar", _dp), ("abar", _dp), ("fF", _dp),
                ("nb_ptr", _i64p), ("nb_idx", _i64p)]


class Diag(C.Structure):
    _fields_ = [("n_ff", C.c_int64), ("n_fw", C.c_int64), ("n_fs", C.c_int64), ("n_sf", C.c_int64),
                ("n_ss", C.c_int64), ("vmax_f", C.c_double), ("vmax_s", C.c_double),
                ("amax_s", C.c_double), ("mom_fs_fluid", C.c_double * 3),
                ("mom_fs_solid", C.c_double * 3), ("abs_fs", C.c_double)]

    def as_dict(self):
        return dict(n_ff=self.n_ff, n_fw=self.n_fw, n_fs=self.n_fs, n_sf=self.n_sf, n_ss=self.n_ss,
                    vmax_f=self.vmax_f, vmax_s=self.vmax_s, amax_s=self.amax_s,
                    mom_fs_fluid=np.array(self.mom_fs_fluid[:]),
                    mom_fs_solid=np.array(self.mom_fs_solid[:]), abs_fs=self.abs_fs)


def lib(threaded=False):
    """The oracle library; threaded=True: its OpenMP build (same bits)."""
    global _lib, _lib_omp
    with _lock:
        if threaded:
            if _lib_omp is None:
                build()
                _lib_omp = _declare(C.CDLL(_LIB_OMP))
            return _lib_omp
        if _lib is None:
            _lib = _declare(C.CDLL(build()))
    return _lib


def threads():
    """Threads the OpenMP build of the oracle runs its loops on."""
    return lib(threaded=True).or_threads()


def _declare(L):
    """Argument and result types of the oracle's entry points."""
    L.or_kernel_W.restype = C.c_double
    L.or_kernel_W.argtypes = [C.c_int, C.c_double, C.c_double]
    L.or_kernel_dW.restype = C.c_double
    L.or_kernel_dW.argtypes = [C.c_int, C.c_double, C.c_double]
    L.or_lattice_sigma0.restype = C.c_double
    L.or_lattice_sigma0.argtypes = [C.c_int, C.c_double, C.c_double]
    L.or_eos_p.restype = C.c_double
    L.or_eos_p.argtypes = [C.c_double] * 3
    L.or_eos_rho.restype = C.c_double
    L.or_eos_rho.argtypes = [C.c_double] * 3
    L.or_riemann.restype = C.c_double
    L.or_riemann.argtypes = [C.c_int, _dp, _dp, _dp] + [C.c_double] * 5 + [_dp]
    L.or_neo_hookean_P.restype = None
    L.or_neo_hookean_P.argtypes = [C.c_int, _dp, C.c_double, C.c_double, _dp]
    L.or_solid_sound_speed.restype = C.c_double
    L.or_solid_sound_speed.argtypes = [C.c_double] * 3
    L.or_pairs_count.restype = C.c_int64
    L.or_pairs_count.argtypes = [C.POINTER(Params), C.c_int, _dp, C.c_int64, _dp, C.c_int64,
                                 C.c_double, C.c_int, C.c_int]
    L.or_pairs_fill.restype = C.c_int
    L.or_pairs_fill.argtypes = [C.POINTER(Params), C.c_int, _dp, C.c_int64, _dp, C.c_int64,
                                C.c_double, C.c_int, C.c_int, _i64p, _i64p]
    L.or_solid_count.restype = C.c_int64
    L.or_solid_count.argtypes = [C.POINTER(Params), C.POINTER(Solid)]
    L.or_solid_setup.restype = C.c_int
    L.or_solid_setup.argtypes = [C.POINTER(Params), C.POINTER(Solid)]
    L.or_solid_F_from_positions.restype = C.c_int
    L.or_solid_F_from_positions.argtypes = [C.POINTER(Params), C.POINTER(Solid), _dp]
    L.or_solid_accel.restype = C.c_int
    L.or_solid_accel.argtypes = [C.POINTER(Params), C.POINTER(Solid), _dp, _dp]
    L.or_inflow_u.restype = C.c_double
    L.or_inflow_u.argtypes = [C.POINTER(Params), C.c_double, C.c_double]
    L.or_inflow_u3.restype = C.c_double
    L.or_inflow_u3.argtypes = [C.POINTER(Params), C.c_double, C.c_double, C.c_double]
    L.or_step.restype = C.c_int
    L.or_step.argtypes = [C.POINTER(Params), C.POINTER(Fluid), C.POINTER(Wall),
                          C.POINTER(Solid), C.c_double, C.c_int, C.c_double, C.c_int64,
                          C.POINTER(Diag)]
    L.or_step_ex.restype = C.c_int
    L.or_step_ex.argtypes = L.or_step.argtypes + [C.POINTER(Cache)]
    L.or_cache_free.restype = None
    L.or_cache_free.argtypes = [C.POINTER(Cache)]
    L.or_suggest_dt.restype = None
    L.or_suggest_dt.argtypes = [C.POINTER(Params), C.POINTER(Fluid), C.POINTER(Solid),
                                C.c_double, C.c_double, C.c_double, _dp, _dp, _dp]
    L.or_substeps.restype = C.c_int
    L.or_substeps.argtypes = [C.c_double, C.c_double]
    L.or_single_dt.restype = C.c_double
    L.or_single_dt.argtypes = [C.POINTER(Params), C.POINTER(Fluid), C.POINTER(Solid), C.c_int,
                               C.c_double, C.c_double, C.c_double]
    L.or_eos_rho_array.restype = None
    L.or_eos_rho_array.argtypes = [C.c_int64, _dp, _dp, C.c_double, C.c_double]
    L.or_threads.restype = C.c_int
    L.or_threads.argtypes = []
    return L


def _p(a):
    """Pointer to a C-contiguous float64 array (kept alive by the caller)."""
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(np.array(a, dtype=dtype, copy=True))


def make_params(case) -> Params:
    P = Params()
    P.dim = case.dim
    P.periodic_x = case.periodic_x
    for k in range(3):
        P.g[k] = float(case.gravity[k])
    P.x_lo, P.Lx = case.x_lo, case.Lx
    P.free_surface, P.n_reinit = case.free_surface, case.n_reinit
    P.inflow_on, P.inflow_profile = case.inflow_on, case.inflow_profile
    P.inflow_width, P.inflow_y0, P.inflow_H = case.inflow_width, case.inflow_y0, case.inflow_H
    P.inflow_U, P.inflow_tramp = case.inflow_U, case.inflow_tramp
    P.inflow_period, P.inflow_wo = getattr(case, "inflow_period", 0.0), getattr(case, "inflow_wo", 0.0)
    P.inflow_z0, P.inflow_Hz = getattr(case, "inflow_z0", 0.0), getattr(case, "inflow_Hz", 0.0)
    return P


# ---------------------------------------------------------------------------
# scalar helpers (for the pins)
# ---------------------------------------------------------------------------

def kernel_W(dim, r, h):
    return lib().or_kernel_W(dim, r, h)


def kernel_dW(dim, r, h):
    return lib().or_kernel_dW(dim, r, h)


def lattice_sigma0(dim, dp, h):
    return lib().or_lattice_sigma0(dim, dp, h)


def eos_p(rho, rho0, c0):
    return lib().or_eos_p(rho, rho0, c0)


def eos_rho(p, rho0, c0):
    return lib().or_eos_rho(p, rho0, c0)


def riemann(e, vL, vR, pL, pR, rhoL, rhoR, c0):
    e, vL, vR = _c(e), _c(vL), _c(vR)
    vs = np.zeros(len(e))
    ps = lib().or_riemann(len(e), _p(e), _p(vL), _p(vR), pL, pR, rhoL, rhoR, c0, _p(vs))
    return ps, vs


def neo_hookean_P(F, mu, lam):
    F = _c(F)
    d = F.shape[0]
    P = np.zeros_like(F)
    lib().or_neo_hookean_P(d, _p(F), mu, lam, _p(P))
    return P


def pairs(case_or_params, A, B, rc, same, brute=False):
    """Neighbour CSR (ptr, idx) of points A against B within rc (r^2 < rc^2)."""
    P = case_or_params if isinstance(case_or_params, Params) else make_params(case_or_params)
    A, B = _c(A), _c(B)
    dim = A.shape[1]
    n = lib().or_pairs_count(C.byref(P), dim, _p(A), len(A), _p(B), len(B), rc, int(same), int(brute))
    ptr = np.zeros(len(A) + 1, np.int64)
    idx = np.zeros(max(n, 1), np.int64)
    lib().or_pairs_fill(C.byref(P), dim, _p(A), len(A), _p(B), len(B), rc, int(same), int(brute),
                        ptr.ctypes.data_as(_i64p), idx.ctypes.data_as(_i64p))
    return ptr, idx[:n]


# ---------------------------------------------------------------------------
# whole-simulation driver
# ---------------------------------------------------------------------------

class Cache(C.Structure):
    """Pair configuration frozen over an advection step (reading F2)."""
    _fields_ = [("valid", C.c_int32), ("nf", C.c_int64), ("ns", C.c_int64), ("lists", C.c_void_p),
                ("fr", C.POINTER(C.c_double)), ("sr", C.POINTER(C.c_double))]


class OracleSim:
    """The oracle's simulation state for one Case (all FP64, original order).
    threaded=True steps with the OpenMP build (the same bits, many cores)."""

    def __init__(self, case, threaded=False):
        L = self._L = lib(threaded)
        self.case = case
        d = case.dim
        self.dim = d
        self.P = make_params(case)
        # fluid
        self.f_r = _c(case.f_r).reshape(-1, d)
        self.f_v = _c(case.f_v).reshape(-1, d)
        self.f_rho = np.zeros(case.nf)
        p0 = _c(case.f_p)
        if case.nf:
            L.or_eos_rho_array(case.nf, _p(p0), _p(self.f_rho), case.f_rho0, case.f_c0)
        self.f_drho = np.zeros(case.nf)
        self.f_dvdt = np.zeros((case.nf, d))
        self.F = Fluid(case.nf, case.f_dp, case.f_rho0, case.f_c0, case.f_eta, _p(self.f_r),
                       _p(self.f_v), _p(self.f_rho), _p(self.f_drho), _p(self.f_dvdt))
        # walls
        self.w_r = _c(case.w_r).reshape(-1, d)
        self.w_n = _c(case.w_n).reshape(-1, d)
        self.W = Wall(case.nw, case.w_dp, _p(self.w_r), _p(self.w_n))
        # solid
        ns = case.ns
        self.s_cons = np.ascontiguousarray(np.asarray(case.s_cons, np.uint8)).reshape(-1)
        self.s_r0 = _c(case.s_r0).reshape(-1, d)
        self.s_n0 = _c(case.s_n0).reshape(-1, d)
        self.s_r = self.s_r0.copy()
        self.s_v = _c(case.s_v0).reshape(-1, d)
        self.s_F = np.zeros((ns, d, d))
        self.s_Fdot = np.zeros((ns, d, d))
        self.s_B0 = np.zeros((ns, d, d))
        self.s_nrm = self.s_n0.copy()
        # time averages start from the initial velocity (reading R14)
        self.s_vbar = self.s_v.copy()
        self.s_abar = np.zeros((ns, d))
        self.s_fF = np.zeros((ns, d))
        self.s_nb_ptr = np.zeros(ns + 1, np.int64)
        self.s_nb_idx = np.zeros(1, np.int64)
        self._mk_solid()
        if ns:
            nnz = L.or_solid_count(C.byref(self.P), C.byref(self.S))
            self.s_nb_idx = np.zeros(max(nnz, 1), np.int64)
            self._mk_solid()
            L.or_solid_setup(C.byref(self.P), C.byref(self.S))
            self.s_vbar[:] = self.s_v
        self.t = 0.0
        self.step_index = 0
        self.diag = Diag()
        self.last = None

    def _mk_solid(self):
        c = self.case
        self.S = Solid(c.ns, c.s_dp, c.s_rho0, c.s_E, c.s_nu,
                       self.s_cons.ctypes.data_as(C.POINTER(C.c_uint8)),
                       _p(self.s_r0), _p(self.s_n0), _p(self.s_r), _p(self.s_v),
                       _p(self.s_F), _p(self.s_Fdot), _p(self.s_B0), _p(self.s_nrm),
                       _p(self.s_vbar), _p(self.s_abar), _p(self.s_fF),
                       self.s_nb_ptr.ctypes.data_as(_i64p), self.s_nb_idx.ctypes.data_as(_i64p))

    # --- time-step criteria (Section 3.2)
    def suggest_dt(self, vmax_f=None, vmax_s=None, amax_s=None):
        if vmax_f is None:
            vmax_f = float(np.sqrt((self.f_v ** 2).sum(1)).max()) if self.case.nf else 0.0
        if vmax_s is None:
            vmax_s = float(np.sqrt((self.s_v ** 2).sum(1)).max()) if self.case.ns else 0.0
        if amax_s is None:
            amax_s = 0.0
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        self._L.or_suggest_dt(C.byref(self.P), C.byref(self.F), C.byref(self.S), vmax_f, vmax_s, amax_s,
                            C.byref(a), C.byref(b), C.byref(c))
        return a.value, b.value, c.value

    def substeps(self, dt_f, dt_s):
        return self._L.or_substeps(dt_f, dt_s)

    def single_dt(self, mode=1, vmax_f=None, vmax_s=None, amax_s=None):
        """Step of the single-time-step baselines (K = 1): mode 1 the
        criterion of Section 2.2, mode 2 min(dt_ac^F, dt^S) (Section 3.2)."""
        if vmax_f is None:
            vmax_f = float(np.sqrt((self.f_v ** 2).sum(1)).max()) if self.case.nf else 0.0
        if vmax_s is None:
            vmax_s = float(np.sqrt((self.s_v ** 2).sum(1)).max()) if self.case.ns else 0.0
        if amax_s is None:
            amax_s = 0.0
        return self._L.or_single_dt(C.byref(self.P), C.byref(self.F), C.byref(self.S), int(mode), vmax_f, vmax_s,
                                  amax_s)

    def set_advection_cadence(self, n):
        """Reading F2 (Algorithm 1): neighbour lists and kernel values built
        once every n steps (an advection step of n acoustic steps) and held
        over them; n = 1 rebuilds them every step (R15).  n = 0 or "auto"
        (reading F3): an advection step lasts while the acoustic steps taken
        in it sum to at most dt_ad, the advection criterion (Eq.
        dtf-advection) at the fluid speed maximum each step starts from, the
        smallest value over the advection step counting."""
        n = 0 if n == "auto" else int(n)
        if n < 0:
            raise ValueError("cadence must be >= 0")
        if getattr(self, "cache", None) is not None:
            self._L.or_cache_free(C.byref(self.cache))
        self.cadence = n
        self.cache = Cache()
        self.rebuilds = []          # step indices that built the configuration
        self._rebuild_next = True   # Algorithm 1 starts an advection step
        self._t_ad = self._t_acc = 0.0

    def __del__(self):
        if getattr(self, "cache", None) is not None and getattr(self, "_L", None) is not None:
            self._L.or_cache_free(C.byref(self.cache))
            self.cache = None

    def step(self, dt, K):
        cache = getattr(self, "cache", None)
        if cache is not None:
            if self.cadence == 0:
                # reading F3: dt_ad at the maximum this step starts from (the
                # last step's post-kick maximum, else the initial speeds)
                v0 = self.last["vmax_f"] if getattr(self, "last", None) else (
                    float(np.sqrt((self.f_v ** 2).sum(1)).max()) if self.case.nf else 0.0)
                _, ad, _ = self.suggest_dt(vmax_f=v0)
                rebuild = self._rebuild_next
                self._t_ad = ad if rebuild else min(self._t_ad, ad)
            else:
                rebuild = self.step_index % self.cadence == 0
            if rebuild:
                cache.valid = 0
                self.rebuilds.append(self.step_index)
            rc = self._L.or_step_ex(C.byref(self.P), C.byref(self.F), C.byref(self.W), C.byref(self.S), dt, int(K),
                                  self.t, self.step_index, C.byref(self.diag), C.byref(cache))
            if self.cadence == 0:
                self._t_acc = (0.0 if rebuild else self._t_acc) + dt
                self._rebuild_next = self._t_acc > self._t_ad
        else:
            rc = self._L.or_step(C.byref(self.P), C.byref(self.F), C.byref(self.W), C.byref(self.S), dt, int(K),
                               self.t, self.step_index, C.byref(self.diag))
        if rc != 0:
            raise RuntimeError(f"oracle step failed ({rc})")
        self.t += dt
        self.step_index += 1
        self.last = self.diag.as_dict()
        return self.last

    # --- pieces used by the pins
    def F_from_positions(self):
        out = np.zeros_like(self.s_F)
        self._L.or_solid_F_from_positions(C.byref(self.P), C.byref(self.S), _p(out))
        return out

    def solid_accel(self, F=None):
        F = self.s_F if F is None else _c(F).reshape(self.s_F.shape)
        out = np.zeros_like(self.s_r)
        self._L.or_solid_accel(C.byref(self.P), C.byref(self.S), _p(F), _p(out))
        return out

    def set_solid_positions(self, r):
        self.s_r[:] = r

    def load_state(self, st):
        """Overwrite the dynamic state from a dict of arrays (original order)."""
        for k in ("f_r", "f_v", "f_rho", "f_drho", "s_r", "s_v", "s_F", "s_vbar", "s_abar", "s_nrm"):
            if k in st and st[k] is not None:
                getattr(self, k)[...] = np.asarray(st[k], np.float64).reshape(getattr(self, k).shape)
        if "t" in st:
            self.t = float(st["t"])
        if "step_index" in st:
            self.step_index = int(st["step_index"])
