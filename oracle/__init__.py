"""FP64 CPU oracle for the particle-side hot path of arXiv 2108.01814.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The GPU product path never imports it, and this package imports
nothing of the GPU path.

The arithmetic lives in ``prs_oracle.c`` (plain C, FP64, ``-ffp-contract=off``);
this module compiles it with gcc on first use and wraps it with ctypes.
Each wrapper names the passage of the paper it follows.

Parity status per function (pins are in ``tests/test_oracle_*.py``):
  phi, template, interp, spread, ibm_step forcing/summation, pairs,
  dem_substep: pinned (identities, closed forms, brute force, library
  routines). The IBM step as a whole has no value printed in the paper to
  compare against: its physics is "parity unpinned"; each of its parts is
  pinned separately.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "prs_oracle.c"), os.path.join(_HERE, "prs_oracle.h")]
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_PP = 12
MAX_WALL = 6


def build(force: bool = False) -> str:
    """Compile the oracle library (gcc, FP64, no FMA contraction), with
    OpenMP where the compiler has it, else single-threaded."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SRC)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", _SRC[0], "-o", tmp, "-lm"]
        try:
            subprocess.check_call(cmd[:1] + ["-fopenmp"] + cmd[1:],
                                  stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Grid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("h", C.c_double), ("periodic", C.c_int * 3),
                ("off", (C.c_double * 3) * 3), ("kernel", C.c_int)]


class Dem(C.Structure):
    _fields_ = [("R", C.c_double), ("m", C.c_double), ("J", C.c_double),
                ("kn_pp", C.c_double), ("dn_pp", C.c_double), ("kt_pp", C.c_double),
                ("dt_pp", C.c_double), ("kn_pw", C.c_double), ("dn_pw", C.c_double),
                ("kt_pw", C.c_double), ("dt_pw", C.c_double), ("mu", C.c_double),
                ("g", C.c_double * 3), ("L", C.c_double * 3), ("periodic", C.c_int * 3),
                ("clip_normal", C.c_int), ("model", C.c_int), ("e_n", C.c_double),
                ("T_c", C.c_double), ("actm_beta", C.c_double), ("actm_S", C.c_double),
                ("u_min", C.c_double), ("mu_f", C.c_double), ("eps_d_pp", C.c_double),
                ("eps_d_pw", C.c_double), ("eps_s", C.c_double)]


class _Hist(C.Structure):
    _fields_ = [("cnt", C.c_void_p), ("pid", C.c_void_p), ("uin", C.c_void_p),
                ("dlt", C.c_void_p), ("wact", C.c_void_p), ("wuin", C.c_void_p),
                ("wdlt", C.c_void_p)]


_dp = C.POINTER(C.c_double)


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            lib.orc_set_threads.restype = C.c_int
            lib.orc_set_threads.argtypes = [C.c_int]
            lib.orc_phi.restype = C.c_double
            lib.orc_phi.argtypes = [C.c_double]
            lib.orc_phi4.restype = C.c_double
            lib.orc_phi4.argtypes = [C.c_double]
            lib.orc_marker_count.restype = C.c_int
            lib.orc_marker_count.argtypes = [C.c_double, C.c_double]
            lib.orc_marker_volume.restype = C.c_double
            lib.orc_marker_volume.argtypes = [C.c_double, C.c_double, C.c_int]
            lib.orc_template.restype = None
            lib.orc_template.argtypes = [C.c_int, C.c_void_p]
            lib.orc_interp.restype = None
            lib.orc_interp.argtypes = [C.POINTER(Grid), C.c_int, C.c_void_p, C.c_long,
                                       C.c_void_p, C.c_void_p]
            lib.orc_spread.restype = None
            lib.orc_spread.argtypes = [C.POINTER(Grid), C.c_int, C.c_void_p, C.c_long,
                                       C.c_void_p, C.c_void_p, C.c_double]
            lib.orc_ibm_step.restype = C.c_int
            lib.orc_ibm_step.argtypes = (
                [C.POINTER(Grid), C.c_int, C.c_double, C.c_double, C.c_int, C.c_void_p,
                 C.c_double] + [C.c_void_p] * 9 +
                [C.c_double, C.c_double, C.c_int, C.c_double] + [C.c_void_p] * 3 + [_dp])
            lib.orc_ibm_step_warm.restype = C.c_int
            lib.orc_ibm_step_warm.argtypes = (
                [C.POINTER(Grid), C.c_int, C.c_double, C.c_double, C.c_int, C.c_void_p,
                 C.c_double] + [C.c_void_p] * 9 +
                [C.c_double, C.c_double, C.c_int, C.c_double, C.c_void_p] +
                [C.c_void_p] * 3 + [_dp])
            lib.orc_dem_params.restype = None
            lib.orc_dem_params.argtypes = ([C.POINTER(Dem)] + [C.c_double] * 7 +
                                           [C.c_void_p, C.c_void_p, C.c_void_p])
            lib.orc_actm_unit.restype = None
            lib.orc_actm_unit.argtypes = [C.c_double, _dp, _dp]
            lib.orc_actm_calibrate.restype = None
            lib.orc_actm_calibrate.argtypes = [C.c_double, _dp, _dp]
            lib.orc_lub_lambda.restype = C.c_double
            lib.orc_lub_lambda.argtypes = [C.c_int, C.c_double]
            lib.orc_pairs.restype = C.c_long
            lib.orc_pairs.argtypes = [C.POINTER(Dem), C.c_int, C.c_void_p, C.c_double,
                                      C.c_void_p, C.c_long]
            lib.orc_dem_substep.restype = C.c_int
            lib.orc_dem_substep.argtypes = ([C.POINTER(Dem), C.c_int, C.c_double] +
                                            [C.c_void_p] * 5 +
                                            [C.POINTER(_Hist), C.POINTER(_Hist)] +
                                            [C.c_void_p] * 5)
            _lib = lib
    return _lib


def set_threads(n: int) -> int:
    """Host threads for the loops over particles, markers and grid slabs
    (1 by default); returns the count in use, 1 when the library was built
    without OpenMP. Results do not depend on it."""
    return int(_lib_handle().orc_set_threads(int(n)))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


# ---------------------------------------------------------------- delta kernel
def phi(r) -> np.ndarray:
    """Roma-Peskin-Berger 3-point regularised delta, one axis (Sec. 3.3)."""
    lib = _lib_handle()
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    return np.array([lib.orc_phi(float(v)) for v in r.ravel()]).reshape(r.shape)


def phi4(r) -> np.ndarray:
    """Peskin's 4-point regularised delta, one axis (a variant of Sec. 3.3's
    delta function)."""
    lib = _lib_handle()
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    return np.array([lib.orc_phi4(float(v)) for v in r.ravel()]).reshape(r.shape)


# ---------------------------------------------------------------- markers
def marker_count(R: float, h: float = 1.0) -> int:
    """Markers per sphere, thin-shell rule (Sec. 3.5 quotes 315 at D/h = 10)."""
    return int(_lib_handle().orc_marker_count(R, h))


def marker_volume(R: float, h: float, n_l: int) -> float:
    """Volume carried by one marker: shell volume / N_L."""
    return float(_lib_handle().orc_marker_volume(R, h, n_l))


def template(n_l: int) -> np.ndarray:
    """Unit surface points of the shared marker template, shape (3, n_l)."""
    t = np.zeros((3, n_l))
    _lib_handle().orc_template(n_l, _ptr(t))
    return t


# ---------------------------------------------------------------- grid
def make_grid(n, h=1.0, periodic=(1, 1, 1), off=None, kernel=3) -> Grid:
    """Grid of n cells; off[c][a] offsets of component c; kernel 3 (Roma et
    al., the default) or 4 (Peskin) for the regularised delta."""
    if kernel not in (3, 4):
        raise ValueError("kernel must be 3 or 4")
    g = Grid()
    g.kernel = int(kernel)
    for a in range(3):
        g.n[a] = int(n[a])
        g.periodic[a] = int(bool(periodic[a]))
    g.h = float(h)
    off = np.full((3, 3), 0.5) if off is None else np.asarray(off, dtype=np.float64)
    for c in range(3):
        for a in range(3):
            g.off[c][a] = float(off[c][a])
    return g


def _grid_shape(g: Grid):
    return (g.n[2], g.n[1], g.n[0])


def interp(g: Grid, c: int, field, X) -> np.ndarray:
    """U(X_l) = sum over the 27-point stencil of u * delta_d * h^3 (Sec. 3.3)."""
    field = _f64(field)
    assert field.size == g.n[0] * g.n[1] * g.n[2]
    X = _f64(X)
    n_m = X.shape[1]
    U = np.zeros(n_m)
    _lib_handle().orc_interp(C.byref(g), c, _ptr(field), n_m, _ptr(X), _ptr(U))
    return U


def spread(g: Grid, c: int, field, X, F, dV: float) -> np.ndarray:
    """field += sum_l F_l delta_d dV (Sec. 3.3). Returns the updated copy."""
    out = _f64(field).copy()
    X = _f64(X)
    F = _f64(F)
    _lib_handle().orc_spread(C.byref(g), c, _ptr(out), X.shape[1], _ptr(X), _ptr(F), dV)
    return out


def ibm_step(g: Grid, R: float, rho_f: float, t, dV: float, x, up, om,
             u, v, w, fx, fy, fz, dt: float, alpha: float = 1.0,
             n_mdf_max: int = 1, tol: float = 0.0, want_marker_force: bool = False,
             dF0=None):
    """One direct-forcing step (Sec. 2.1 and 3.3) on copies of the fields.

    Returns a dict with the updated u, v, w, fx, fy, fz, the per-particle
    hydrodynamic force F_h and torque T_h (3, n_p), the marker forces
    (3, n_p * n_l) if asked, the number of forcing iterations and the
    residual max |U_d - U| of the last interpolation.

    dF0 (3, n_p * n_l), if given, is added to the first forcing increment
    only (the learned warm start; the paper has no counterpart).
    """
    lib = _lib_handle()
    t = _f64(t)
    n_l = t.shape[1]
    x, up, om = _f64(x), _f64(up), _f64(om)
    n_p = x.shape[1]
    flds = [_f64(a).copy() for a in (u, v, w, fx, fy, fz)]
    F_h = np.zeros((3, n_p))
    T_h = np.zeros((3, n_p))
    F_l = np.zeros((3, n_p * n_l)) if want_marker_force else None
    res = C.c_double(0.0)
    if dF0 is None:
        it = lib.orc_ibm_step(C.byref(g), n_p, R, rho_f, n_l, _ptr(t), dV, _ptr(x), _ptr(up),
                              _ptr(om), *[_ptr(a) for a in flds], dt, alpha, n_mdf_max, tol,
                              _ptr(F_h), _ptr(T_h), _ptr(F_l), C.byref(res))
    else:
        dF0 = _f64(dF0, (3, n_p * n_l))
        it = lib.orc_ibm_step_warm(C.byref(g), n_p, R, rho_f, n_l, _ptr(t), dV, _ptr(x),
                                   _ptr(up), _ptr(om), *[_ptr(a) for a in flds], dt, alpha,
                                   n_mdf_max, tol, _ptr(dF0), _ptr(F_h), _ptr(T_h),
                                   _ptr(F_l), C.byref(res))
    if it < 0:
        raise MemoryError("oracle ibm_step: allocation failed")
    out = dict(zip(("u", "v", "w", "fx", "fy", "fz"), flds))
    out.update(F_h=F_h, T_h=T_h, F_l=F_l, iterations=it, residual=res.value)
    return out


# ---------------------------------------------------------------- DEM
def actm_unit(beta):
    """The unit Hertzian collision x'' + beta x' + x^(3/2) = 0, x(0) = 0,
    x'(0) = 1 (the adaptive collision time model in units of the impact):
    its duration S and restitution e."""
    S, e = C.c_double(), C.c_double()
    _lib_handle().orc_actm_unit(beta, C.byref(S), C.byref(e))
    return S.value, e.value


def actm_calibrate(e_n):
    """(beta*, S*): the unit collision's damping that rebounds with e_n, and
    its duration."""
    b, S = C.c_double(), C.c_double()
    _lib_handle().orc_actm_calibrate(e_n, C.byref(b), C.byref(S))
    return b.value, S.value


def lub_lambda(wall, eps):
    """Stokes amplification of the small-gap normal resistance at eps =
    delta_n / R (wall: sphere and wall; else two equal spheres)."""
    return _lib_handle().orc_lub_lambda(1 if wall else 0, float(eps))


def dem_params(R, rho_p, rho_f, e_n, e_t, mu, T_c, g, L, periodic, clip_normal=False,
               model="linear", u_min=None, mu_f=0.0, eps_d=(0.05, 0.05), eps_s=0.001) -> Dem:
    """Spring-dashpot constants from T_c and the restitution coefficients
    (ACTM family, Sec. 2.1), inertia of Eq. 7-8 in rigid-body form.
    clip_normal: the variant whose normal force (Eq. 9) is clipped to be
    repulsive; the plain law otherwise.
    model="actm": the Hertzian normal law whose stiffness and damping are
    calibrated per contact from its impact speed (never below u_min; default
    |g| T_c, or 1e-3 R / T_c without gravity).
    mu_f > 0: lubrication between spheres and against walls for gaps below
    eps_d = (sphere-sphere, sphere-wall) times R, held at eps_s R below."""
    d = Dem()
    g = _f64(g)
    L = _f64(L)
    per = np.ascontiguousarray(periodic, dtype=np.int32)
    _lib_handle().orc_dem_params(C.byref(d), R, rho_p, rho_f, e_n, e_t, mu, T_c,
                                 _ptr(g), _ptr(L), _ptr(per))
    d.clip_normal = 1 if clip_normal else 0
    if model == "actm":
        d.model = 1
        d.actm_beta, d.actm_S = actm_calibrate(e_n)
        gm = float(np.linalg.norm(g))
        d.u_min = float(u_min) if u_min is not None else (gm * T_c if gm > 0 else 1e-3 * R / T_c)
    elif model != "linear":
        raise ValueError("model must be 'linear' or 'actm'")
    d.mu_f = float(mu_f)
    d.eps_d_pp, d.eps_d_pw = (float(v) for v in eps_d)
    d.eps_s = float(eps_s)
    return d


def pairs(d: Dem, x, cutoff: float) -> np.ndarray:
    """All pairs (p < q) with centre distance < cutoff, minimum image on
    periodic axes (A.1, A.3), lexicographic order. Shape (n_pairs, 2)."""
    x = _f64(x)
    n_p = x.shape[1]
    lib = _lib_handle()
    cap = max(16, 8 * n_p)
    while True:
        buf = np.zeros((cap, 2), dtype=np.int32)
        n = lib.orc_pairs(C.byref(d), n_p, _ptr(x), cutoff, _ptr(buf), cap)
        if n <= cap:
            return buf[:n].copy()
        cap = int(n)


class History:
    """Contact history M_p (Sec. 3.4): 12 particle slots + 6 wall slots per
    particle, partner ids ascending."""

    def __init__(self, n_p: int):
        self.cnt = np.zeros(n_p, dtype=np.int32)
        self.pid = np.full((n_p, MAX_PP), -1, dtype=np.int32)
        self.uin = np.zeros((n_p, MAX_PP))
        self.dlt = np.zeros((n_p, MAX_PP, 3))
        self.wact = np.zeros((n_p, MAX_WALL), dtype=np.uint8)
        self.wuin = np.zeros((n_p, MAX_WALL))
        self.wdlt = np.zeros((n_p, MAX_WALL, 3))

    def copy(self) -> "History":
        h = History(len(self.cnt))
        for k in ("cnt", "pid", "uin", "dlt", "wact", "wuin", "wdlt"):
            setattr(h, k, getattr(self, k).copy())
        return h

    def _struct(self) -> _Hist:
        s = _Hist()
        for k in ("cnt", "pid", "uin", "dlt", "wact", "wuin", "wdlt"):
            setattr(s, k, getattr(self, k).ctypes.data)
        return s


def dem_substep(d: Dem, dt_p: float, x, up, om, F_h, T_h, hist: History):
    """One particle sub-step: contacts, history events, spring-dashpot
    forces (Eq. 9-10, A.1-A.11, Sec. 3.4) and the semi-implicit Euler update
    of Eq. 7-8. Returns (x, u, omega, F_c, T_c, new_history, overflow)."""
    lib = _lib_handle()
    x, up, om, F_h, T_h = (_f64(a) for a in (x, up, om, F_h, T_h))
    n_p = x.shape[1]
    neu = History(n_p)
    xo, uo, oo, Fc, Tc = (np.zeros((3, n_p)) for _ in range(5))
    old_s, neu_s = hist._struct(), neu._struct()
    st = lib.orc_dem_substep(C.byref(d), n_p, dt_p, _ptr(x), _ptr(up), _ptr(om), _ptr(F_h),
                             _ptr(T_h), C.byref(old_s), C.byref(neu_s), _ptr(xo), _ptr(uo),
                             _ptr(oo), _ptr(Fc), _ptr(Tc))
    for p in range(n_p):
        neu.pid[p, neu.cnt[p]:] = -1
    return xo, uo, oo, Fc, Tc, neu, bool(st)


def dem_run(d: Dem, dt_p: float, n_sub: int, x, up, om, F_h, T_h, hist: History):
    """n_sub sub-steps with F_h, T_h held fixed (Sec. 2.1: dt_p = dt_f / 50)."""
    overflow = False
    Fc = Tc = None
    for _ in range(n_sub):
        x, up, om, Fc, Tc, hist, ov = dem_substep(d, dt_p, x, up, om, F_h, T_h, hist)
        overflow |= ov
    return x, up, om, Fc, Tc, hist, overflow
