"""Thin ctypes binding of the C ABI in ``include/pr_sed.h``.

Argument marshalling only: every step of the hot path runs in the CUDA
kernels of ``libprsed.so``. PyTorch provides device memory (through the
allocator callback) and the stream. There is no CPU fallback: if the
library cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

PRS_FP64, PRS_FP32 = 0, 1
PRS_HOST, PRS_DEVICE = 0, 1
MAX_CONTACTS, MAX_WALLS = 12, 6

STATUS = {
    0: "PRS_OK", 1: "PRS_WARN_NOT_CONVERGED", -1: "PRS_ERR_ARG", -2: "PRS_ERR_OOM",
    -3: "PRS_ERR_CUDA", -4: "PRS_ERR_STATE", -5: "PRS_ERR_CONTACT_OVERFLOW",
    -6: "PRS_ERR_NONFINITE", -7: "PRS_ERR_CAPACITY", -8: "PRS_ERR_TIMEOUT",
}
globals().update({v: k for k, v in STATUS.items()})  # PRS_OK, PRS_ERR_OOM, ...

# every function the header declares, for the export check
EXPORTS = [
    "prs_create_grid", "prs_create_particles", "prs_write_state", "prs_read_state",
    "prs_ibm_step", "prs_dem_step", "prs_read_forces", "prs_read_marker_forces",
    "prs_read_template", "prs_read_history", "prs_write_history", "prs_find_pairs",
    "prs_get_stats", "prs_set_stream", "prs_sync", "prs_destroy", "prs_last_error_string",
    "prs_set_profiling", "prs_set_graphs", "prs_read_profile", "prs_find_pairs_noalloc",
    "prs_mlp_set_params", "prs_mlp_get_params", "prs_mlp_forward", "prs_mlp_grad",
    "prs_mlp_train_step", "prs_mlp_train_step_sampled", "prs_mlp_collect",
    "prs_bed_detect", "prs_track_saltation", "prs_reset_saltation", "prs_predict",
    "prs_probe_wait",
]
MLP_NPARAM = 4995  # PRS_MLP_NPARAM
NOALLOC_MAX_PARTICLES = 65536  # PRS_NOALLOC_MAX_PARTICLES
NOALLOC_MAX_CELLS = 262144      # PRS_NOALLOC_MAX_CELLS
PHASES = ("ibm_bin", "interp", "spread", "dem_cells", "dem_contacts", "dem_update", "mlp")
# prs_event, one closed impact event of a saltating sphere
EVENT_DTYPE = np.dtype([("particle", np.int32), ("rebound", np.int32),
                        ("t_impact", np.float64), ("t_departure", np.float64),
                        ("u_impact", np.float64, 3), ("omega_impact", np.float64, 3),
                        ("u_departure", np.float64, 3), ("omega_departure", np.float64, 3)])


class PrsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Allocator(C.Structure):
    _fields_ = [("alloc", C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)),
                ("free", C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)),
                ("user", C.c_void_p)]


class _IbmOpts(C.Structure):
    _fields_ = [("n_mdf_max", C.c_int), ("tol", C.c_double), ("grid_where", C.c_int),
                ("final_residual", C.c_int), ("learned", C.c_int), ("host_async", C.c_int),
                ("delta_kernel", C.c_int)]


class _AdamOpts(C.Structure):
    _fields_ = [("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double),
                ("eps", C.c_double)]


class _DemOpts(C.Structure):
    _fields_ = [("e_n", C.c_double), ("e_t", C.c_double), ("mu", C.c_double),
                ("T_c", C.c_double), ("g", C.c_double * 3), ("clip_normal", C.c_int),
                ("model", C.c_int), ("u_min", C.c_double), ("mu_f", C.c_double),
                ("eps_d_pp", C.c_double), ("eps_d_pw", C.c_double), ("eps_s", C.c_double)]


PRS_CONTACT_LINEAR, PRS_CONTACT_ACTM = 0, 1


class _Stats(C.Structure):
    _fields_ = [("mdf_passes", C.c_int), ("residual", C.c_double), ("n_markers", C.c_longlong),
                ("n_contacts", C.c_longlong), ("n_wall_contacts", C.c_longlong),
                ("error_word", C.c_int), ("n_launches", C.c_longlong),
                ("h2d_bytes", C.c_longlong), ("d2h_bytes", C.c_longlong),
                ("dem_graph", C.c_int)]


_lib = None
_lock = threading.Lock()
_vp = C.c_void_p


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libprsed.so (compiling it with nvcc first if it is missing or
    older than its sources). Raises if it cannot be built or loaded."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_needed:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libprsed.so not built ({_build.LIB}); run build() first")
        lib = C.CDLL(_build.LIB)
        sig = {
            "prs_create_grid": [C.c_int, C.c_int, C.c_int, C.c_double, _vp, _vp, C.c_int,
                                C.POINTER(_Allocator), _vp, C.POINTER(_vp)],
            "prs_create_particles": [_vp, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int],
            "prs_write_state": [_vp, _vp, _vp, _vp, C.c_int],
            "prs_read_state": [_vp, _vp, _vp, _vp, C.c_int],
            "prs_ibm_step": [_vp] * 7 + [C.c_double, C.c_double, C.POINTER(_IbmOpts)],
            "prs_predict": [_vp, C.c_int, _vp, _vp, _vp] + [C.c_double] * 4,
            "prs_dem_step": [_vp, C.c_double, C.c_int, C.POINTER(_DemOpts)],
            "prs_read_forces": [_vp] * 5 + [C.c_int],
            "prs_read_marker_forces": [_vp, _vp, C.c_int],
            "prs_read_template": [_vp, _vp, _vp, _vp],
            "prs_read_history": [_vp] * 8,
            "prs_write_history": [_vp] * 8,
            "prs_find_pairs": [_vp, C.c_double, _vp, C.c_longlong, C.POINTER(C.c_longlong)],
            "prs_get_stats": [_vp, C.POINTER(_Stats)],
            "prs_set_stream": [_vp, _vp],
            "prs_sync": [_vp],
            "prs_set_profiling": [_vp, C.c_int],
            "prs_set_graphs": [_vp, C.c_int],
            "prs_read_profile": [_vp, _vp, _vp],
            "prs_find_pairs_noalloc": [_vp, C.c_int, _vp, _vp, C.c_double, _vp, C.c_longlong,
                                       _vp, _vp],
            "prs_mlp_set_params": [_vp, _vp],
            "prs_mlp_get_params": [_vp, _vp],
            "prs_mlp_forward": [_vp, _vp, C.c_longlong, _vp],
            "prs_mlp_grad": [_vp, _vp, _vp, C.c_longlong, _vp, _vp],
            "prs_mlp_train_step": [_vp, _vp, _vp, C.c_longlong, C.POINTER(_AdamOpts), _vp],
            "prs_mlp_train_step_sampled": [_vp, _vp, _vp, C.c_longlong, C.c_longlong,
                                           C.c_longlong, C.c_longlong, C.POINTER(_AdamOpts),
                                           _vp],
            "prs_mlp_collect": [_vp] * 7 + [C.c_double, C.c_double, C.POINTER(_IbmOpts), _vp,
                                            _vp],
            "prs_bed_detect": [_vp, _vp, C.POINTER(C.c_longlong), C.c_int],
            "prs_track_saltation": [_vp, C.c_double, C.c_double, C.c_double, _vp, C.c_longlong,
                                    C.POINTER(C.c_longlong), C.c_int],
            "prs_reset_saltation": [_vp],
            "prs_probe_wait": [_vp, C.c_longlong],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = C.c_int
        lib.prs_destroy.argtypes = [_vp]
        lib.prs_destroy.restype = None
        lib.prs_last_error_string.argtypes = []
        lib.prs_last_error_string.restype = C.c_char_p
        _lib = lib
        return lib


def _check(st, allow_warn=False):
    if st == 0 or (allow_warn and st > 0):
        return st
    msg = _lib.prs_last_error_string().decode()
    raise PrsError(st, msg)


def _torch():
    import torch
    return torch


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _vec_ptr(a, n_p):
    """Pointer and `where` for a [3][n_p] FP64 array (numpy host or torch device)."""
    if _is_torch(a):
        torch = _torch()
        assert a.dtype == torch.float64 and a.is_cuda and a.is_contiguous()
        assert a.numel() == 3 * n_p
        return C.c_void_p(a.data_ptr()), PRS_DEVICE, a
    h = np.ascontiguousarray(a, dtype=np.float64)
    assert h.size == 3 * n_p
    return h.ctypes.data_as(_vp), PRS_HOST, h


class _TorchAllocator:
    """Device memory for the library, taken from PyTorch's caching allocator;
    with a budget (bytes), allocations that would exceed it are refused and
    the library call that asked returns PRS_ERR_OOM."""

    def __init__(self, device, budget=None):
        self.device = device
        self.blocks = {}
        self.budget = budget
        self.used = 0
        self._alloc_cb = _Allocator._fields_[0][1](self._alloc)
        self._free_cb = _Allocator._fields_[1][1](self._free)
        self.struct = _Allocator(self._alloc_cb, self._free_cb, None)

    def _alloc(self, nbytes, stream, user):
        torch = _torch()
        if self.budget is not None and self.used + int(nbytes) > self.budget:
            return None
        try:
            t = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        except RuntimeError:
            return None
        self.blocks[t.data_ptr()] = t
        self.used += int(nbytes)
        return t.data_ptr()

    def _free(self, ptr, stream, user):
        t = self.blocks.pop(ptr, None)
        if t is not None:
            self.used -= t.numel()


@dataclass
class Stats:
    mdf_passes: int
    residual: float
    n_markers: int
    n_contacts: int
    n_wall_contacts: int
    error_word: int
    n_launches: int
    h2d_bytes: int = 0
    d2h_bytes: int = 0
    dem_graph: int = 0


class Context:
    """One grid + one population of equal spheres (prs_ctx)."""

    def __init__(self, n, h=1.0, periodic=(1, 1, 1), offset=None, precision="fp64",
                 device=None, stream=None, use_torch_allocator=True, device_budget=None):
        torch = _torch()
        self.lib = load()
        self.n = tuple(int(v) for v in n)
        self.h = float(h)
        self.periodic = tuple(int(bool(v)) for v in periodic)
        self.precision = PRS_FP64 if precision in ("fp64", PRS_FP64) else PRS_FP32
        self.dtype = torch.float64 if self.precision == PRS_FP64 else torch.float32
        self.np_dtype = np.float64 if self.precision == PRS_FP64 else np.float32
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        torch.cuda.init()
        with torch.cuda.device(self.device):
            st = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.stream = st
        self._alloc = (_TorchAllocator(self.device, device_budget) if use_torch_allocator
                       else None)
        per = (C.c_int * 3)(*self.periodic)
        off = None
        if offset is not None:
            self._off = (C.c_double * 9)(*np.asarray(offset, dtype=np.float64).ravel())
            off = C.cast(self._off, _vp)
        h_out = _vp()
        _check(self.lib.prs_create_grid(
            self.n[0], self.n[1], self.n[2], self.h, C.cast(per, _vp), off, self.precision,
            C.byref(self._alloc.struct) if self._alloc else None,
            C.c_void_p(st.cuda_stream), C.byref(h_out)))
        self.ctx = h_out
        self.n_p = 0
        self.n_l = 0

    # ---------------------------------------------------------------- lifecycle
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.prs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---------------------------------------------------------------- particles
    def create_particles(self, n_p, R, rho_p, rho_f, n_markers=0):
        _check(self.lib.prs_create_particles(self.ctx, int(n_p), float(R), float(rho_p),
                                             float(rho_f), int(n_markers)))
        self.n_p = int(n_p)
        _, _, self.n_l = self.read_template(want_t=False)
        self.R = float(R)
        return self

    def write_state(self, x, u, om):
        px, w1, kx = _vec_ptr(x, self.n_p)
        pu, w2, ku = _vec_ptr(u, self.n_p)
        po, w3, ko = _vec_ptr(om, self.n_p)
        assert w1 == w2 == w3, "x, u, omega must all be host or all device"
        _check(self.lib.prs_write_state(self.ctx, px, pu, po, w1))

    def read_state(self, device=False, out=None):
        if device:
            torch = _torch()
            out = [torch.empty((3, self.n_p), dtype=torch.float64, device=self.device)
                   for _ in range(3)]
            _check(self.lib.prs_read_state(self.ctx, *[C.c_void_p(t.data_ptr()) for t in out],
                                           PRS_DEVICE))
            return out
        if out is None:
            out = [np.zeros((3, self.n_p)) for _ in range(3)]
        for a in out:
            assert a.dtype == np.float64 and a.shape == (3, self.n_p) and a.flags["C_CONTIGUOUS"]
        _check(self.lib.prs_read_state(self.ctx, *[a.ctypes.data_as(_vp) for a in out],
                                       PRS_HOST))
        return out

    # ---------------------------------------------------------------- steps
    def _field_ptrs(self, flds):
        if all(_is_torch(a) for a in flds):
            for a in flds:
                assert a.is_cuda and a.dtype == self.dtype and a.is_contiguous()
                assert a.numel() == self.n[0] * self.n[1] * self.n[2]
            return [C.c_void_p(a.data_ptr()) for a in flds], PRS_DEVICE
        for a in flds:
            assert isinstance(a, np.ndarray) and a.dtype == self.np_dtype
            assert a.flags["C_CONTIGUOUS"]
        return [a.ctypes.data_as(_vp) for a in flds], PRS_HOST

    def ibm_step(self, u, v, w, fx, fy, fz, dt, alpha=1.0, n_mdf_max=1, tol=0.0,
                 final_residual=False, learned=False, host_async=False, delta_kernel=3):
        flds = [u, v, w, fx, fy, fz]
        if all(_is_torch(a) for a in flds):
            for a in flds:
                assert a.is_cuda and a.dtype == self.dtype and a.is_contiguous()
                assert a.numel() == self.n[0] * self.n[1] * self.n[2]
            ptrs = [C.c_void_p(a.data_ptr()) for a in flds]
            where = PRS_DEVICE
        else:
            for a in flds:
                assert isinstance(a, np.ndarray) and a.dtype == self.np_dtype
                assert a.flags["C_CONTIGUOUS"]
            ptrs = [a.ctypes.data_as(_vp) for a in flds]
            where = PRS_HOST
        opts = _IbmOpts(int(n_mdf_max), float(tol), where, int(bool(final_residual)),
                        int(bool(learned)), int(bool(host_async)), int(delta_kernel))
        return _check(self.lib.prs_ibm_step(self.ctx, *ptrs, float(dt), float(alpha),
                                            C.byref(opts)), allow_warn=True)

    def predict(self, component, u_in, u_out, H, nu, dt, alpha=1.0, beta=0.0):
        """prs_predict: u_out = u_in + dt (alpha nu lap(u_in) - beta H), then
        H = nu lap(u_in); CUDA tensors of the context's dtype and grid shape."""
        for a in (u_in, u_out, H):
            assert _is_torch(a) and a.is_cuda and a.dtype == self.dtype and a.is_contiguous()
            assert a.numel() == self.n[0] * self.n[1] * self.n[2]
        _check(self.lib.prs_predict(self.ctx, int(component), C.c_void_p(u_in.data_ptr()),
                                    C.c_void_p(u_out.data_ptr()), C.c_void_p(H.data_ptr()),
                                    float(nu), float(dt), float(alpha), float(beta)))

    # ---------------------------------------------------------------- warm-start network
    @staticmethod
    def _f32_dev(a, cols, name):
        torch = _torch()
        if not (_is_torch(a) and a.is_cuda and a.dtype == torch.float32 and a.is_contiguous()
                and a.dim() == 2 and a.shape[1] == cols):
            raise ValueError(f"{name} must be a contiguous CUDA float32 tensor [n][{cols}]")
        return C.c_void_p(a.data_ptr())

    def mlp_set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32).ravel()
        assert p.size == MLP_NPARAM
        _check(self.lib.prs_mlp_set_params(self.ctx, p.ctypes.data_as(_vp)))

    def mlp_get_params(self):
        p = np.zeros(MLP_NPARAM, dtype=np.float32)
        _check(self.lib.prs_mlp_get_params(self.ctx, p.ctypes.data_as(_vp)))
        return p

    def mlp_forward(self, feats, out=None):
        torch = _torch()
        n = feats.shape[0]
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float32, device=feats.device)
        _check(self.lib.prs_mlp_forward(self.ctx, self._f32_dev(feats, 9, "feats"), int(n),
                                        self._f32_dev(out, 3, "out")))
        return out

    def mlp_grad(self, feats, targets):
        g = np.zeros(MLP_NPARAM, dtype=np.float32)
        loss = C.c_float()
        _check(self.lib.prs_mlp_grad(self.ctx, self._f32_dev(feats, 9, "feats"),
                                     self._f32_dev(targets, 3, "targets"), int(feats.shape[0]),
                                     g.ctypes.data_as(_vp), C.byref(loss)))
        return g, loss.value

    def mlp_train_step(self, feats, targets, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                       want_loss=True):
        o = _AdamOpts(float(lr), float(beta1), float(beta2), float(eps))
        loss = C.c_float()
        _check(self.lib.prs_mlp_train_step(self.ctx, self._f32_dev(feats, 9, "feats"),
                                           self._f32_dev(targets, 3, "targets"),
                                           int(feats.shape[0]), C.byref(o),
                                           C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def mlp_train_step_sampled(self, feats, targets, n, start, stride, lr=1e-3, beta1=0.9,
                               beta2=0.999, eps=1e-8, want_loss=True):
        """One Adam step on the n pairs (start + i stride) mod n_total of
        feats/targets (n_total = their rows)."""
        o = _AdamOpts(float(lr), float(beta1), float(beta2), float(eps))
        loss = C.c_float()
        _check(self.lib.prs_mlp_train_step_sampled(
            self.ctx, self._f32_dev(feats, 9, "feats"), self._f32_dev(targets, 3, "targets"),
            int(feats.shape[0]), int(n), int(start), int(stride), C.byref(o),
            C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def mlp_collect(self, u, v, w, fx, fy, fz, dt, alpha=1.0, n_mdf_max=8):
        """Plain forcing step that also returns the training pairs of every
        marker: (feats [n_m][9], targets [n_m][3]) CUDA float32 tensors."""
        torch = _torch()
        ptrs, where = self._field_ptrs([u, v, w, fx, fy, fz])
        n_m = self.n_p * self.n_l
        feats = torch.empty((n_m, 9), dtype=torch.float32, device=self.device)
        targets = torch.empty((n_m, 3), dtype=torch.float32, device=self.device)
        opts = _IbmOpts(int(n_mdf_max), 0.0, where, 0, 0)
        _check(self.lib.prs_mlp_collect(self.ctx, *ptrs, float(dt), float(alpha), C.byref(opts),
                                        C.c_void_p(feats.data_ptr()),
                                        C.c_void_p(targets.data_ptr())), allow_warn=True)
        return feats, targets

    def dem_step(self, dt_p, n_sub, e_n, e_t, mu, T_c, g=(0.0, 0.0, 0.0), clip_normal=False,
                 model="linear", u_min=0.0, mu_f=0.0, eps_d=(0.0, 0.0), eps_s=0.0):
        """prs_dem_step. model: "linear" or "actm" (the adaptive collision
        time model); mu_f > 0 adds lubrication (eps_d: ranges over R for
        sphere-sphere and sphere-wall gaps, eps_s: saturation; 0 = defaults)."""
        models = {"linear": PRS_CONTACT_LINEAR, "actm": PRS_CONTACT_ACTM}
        if model not in models:
            raise ValueError("model must be 'linear' or 'actm'")
        o = _DemOpts(float(e_n), float(e_t), float(mu), float(T_c), (C.c_double * 3)(*g),
                     int(bool(clip_normal)), models[model], float(u_min), float(mu_f),
                     float(eps_d[0]), float(eps_d[1]), float(eps_s))
        _check(self.lib.prs_dem_step(self.ctx, float(dt_p), int(n_sub), C.byref(o)))

    # ---------------------------------------------------------------- reads
    def read_forces(self, out=None):
        """F_h, T_h, F_c, T_c as [3][n_p] float64 host arrays; `out` may give
        the four arrays (pinned ones copy fastest)."""
        if out is None:
            out = [np.zeros((3, self.n_p)) for _ in range(4)]
        for a in out:
            assert a.dtype == np.float64 and a.shape == (3, self.n_p) and a.flags["C_CONTIGUOUS"]
        _check(self.lib.prs_read_forces(self.ctx, *[a.ctypes.data_as(_vp) for a in out],
                                        PRS_HOST))
        return dict(zip(("F_h", "T_h", "F_c", "T_c"), out))

    def read_marker_forces(self):
        out = np.zeros((3, self.n_p * self.n_l), dtype=self.np_dtype)
        _check(self.lib.prs_read_marker_forces(self.ctx, out.ctypes.data_as(_vp), PRS_HOST))
        return out

    def read_template(self, want_t=True):
        dV = C.c_double()
        n_l = C.c_int()
        _check(self.lib.prs_read_template(self.ctx, None, C.byref(dV), C.byref(n_l)))
        t = None
        if want_t:
            t = np.zeros((3, n_l.value))
            _check(self.lib.prs_read_template(self.ctx, t.ctypes.data_as(_vp), None, None))
        return t, dV.value, n_l.value

    def read_history(self):
        n = self.n_p
        cnt = np.zeros(n, dtype=np.int32)
        pid = np.zeros((n, MAX_CONTACTS), dtype=np.int32)
        uin = np.zeros((n, MAX_CONTACTS))
        dlt = np.zeros((n, MAX_CONTACTS, 3))
        wact = np.zeros((n, MAX_WALLS), dtype=np.uint8)
        wuin = np.zeros((n, MAX_WALLS))
        wdlt = np.zeros((n, MAX_WALLS, 3))
        arrs = [cnt, pid, uin, dlt, wact, wuin, wdlt]
        _check(self.lib.prs_read_history(self.ctx, *[a.ctypes.data_as(_vp) for a in arrs]))
        return dict(zip(("cnt", "pid", "uin", "dlt", "wact", "wuin", "wdlt"), arrs))

    def write_history(self, cnt, pid, uin, dlt, wact, wuin, wdlt):
        arrs = [np.ascontiguousarray(cnt, dtype=np.int32), np.ascontiguousarray(pid, dtype=np.int32),
                np.ascontiguousarray(uin, dtype=np.float64), np.ascontiguousarray(dlt, dtype=np.float64),
                np.ascontiguousarray(wact, dtype=np.uint8), np.ascontiguousarray(wuin, dtype=np.float64),
                np.ascontiguousarray(wdlt, dtype=np.float64)]
        _check(self.lib.prs_write_history(self.ctx, *[a.ctypes.data_as(_vp) for a in arrs]))

    def find_pairs(self, cutoff, max_pairs=None):
        if max_pairs is None:
            max_pairs = 16 * self.n_p + 16
        buf = np.zeros((max_pairs, 2), dtype=np.int32)
        n = C.c_longlong()
        _check(self.lib.prs_find_pairs(self.ctx, float(cutoff), buf.ctypes.data_as(_vp),
                                       int(max_pairs), C.byref(n)))
        if n.value > max_pairs:
            return self.find_pairs(cutoff, int(n.value))
        return buf[:n.value].copy()

    def bed_detect(self):
        """Bed (1) / flying (0) flags of the current state, uint8 [n_p]."""
        f = np.zeros(self.n_p, dtype=np.uint8)
        n = C.c_longlong()
        _check(self.lib.prs_bed_detect(self.ctx, f.ctypes.data_as(_vp), C.byref(n), PRS_HOST))
        assert int(f.sum()) == n.value
        return f

    def track_saltation(self, t, h_r, t_cir, max_events=None):
        """Events the current state closes, a structured array of
        EVENT_DTYPE in sphere order."""
        cap = self.n_p if max_events is None else int(max_events)
        ev = np.zeros(max(cap, 1), dtype=EVENT_DTYPE)
        n = C.c_longlong()
        _check(self.lib.prs_track_saltation(self.ctx, float(t), float(h_r), float(t_cir),
                                            ev.ctypes.data_as(_vp), cap, C.byref(n), PRS_HOST))
        return ev[:n.value].copy()

    def reset_saltation(self):
        _check(self.lib.prs_reset_saltation(self.ctx))

    def stats(self) -> Stats:
        s = _Stats()
        _check(self.lib.prs_get_stats(self.ctx, C.byref(s)))
        return Stats(s.mdf_passes, s.residual, s.n_markers, s.n_contacts, s.n_wall_contacts,
                     s.error_word, s.n_launches, s.h2d_bytes, s.d2h_bytes, s.dem_graph)

    def set_profiling(self, on=True):
        _check(self.lib.prs_set_profiling(self.ctx, int(bool(on))))

    def set_graphs(self, on):
        """prs_set_graphs: the DEM sub-steps as a replayed CUDA graph."""
        _check(self.lib.prs_set_graphs(self.ctx, int(bool(on))))

    def read_profile(self):
        """{phase: (milliseconds, launches)} since the last read."""
        ms = (C.c_double * len(PHASES))()
        cnt = (C.c_longlong * len(PHASES))()
        _check(self.lib.prs_read_profile(self.ctx, C.cast(ms, _vp), C.cast(cnt, _vp)))
        return {p: (ms[i], cnt[i]) for i, p in enumerate(PHASES)}

    def sync(self):
        _check(self.lib.prs_sync(self.ctx))

    def probe_wait(self, polls):
        """prs_probe_wait: a bounded device wait that runs out on purpose."""
        _check(self.lib.prs_probe_wait(self.ctx, C.c_longlong(int(polls))))


def create_grid(n, h=1.0, periodic=(1, 1, 1), offset=None, precision="fp64", **kw) -> Context:
    """prs_create_grid: a new context."""
    return Context(n, h, periodic, offset, precision, **kw)


def find_pairs_noalloc(x, L, periodic, cutoff, pairs, n_pairs, stream=None):
    """prs_find_pairs_noalloc: all pairs p < q of the centres ``x`` (a
    contiguous CUDA float64 tensor [3][n_p]) closer than ``cutoff``, written
    into the caller's CUDA int32 tensor ``pairs`` [max_pairs][2] (order
    unspecified) with the total count in the caller's one-element CUDA int64
    tensor ``n_pairs``. The library allocates nothing; the call is
    asynchronous on ``stream`` (default: torch's current stream)."""
    torch = _torch()
    lib = load()
    if not (_is_torch(x) and x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()
            and x.dim() == 2 and x.shape[0] == 3):
        raise ValueError("x must be a contiguous CUDA float64 tensor of shape [3][n_p]")
    if not (_is_torch(pairs) and pairs.is_cuda and pairs.dtype == torch.int32
            and pairs.is_contiguous() and pairs.dim() == 2 and pairs.shape[1] == 2):
        raise ValueError("pairs must be a contiguous CUDA int32 tensor of shape [max_pairs][2]")
    if not (_is_torch(n_pairs) and n_pairs.is_cuda and n_pairs.dtype == torch.int64
            and n_pairs.numel() == 1):
        raise ValueError("n_pairs must be a one-element CUDA int64 tensor")
    Lh = (C.c_double * 3)(*[float(v) for v in L])
    ph = (C.c_int * 3)(*[int(bool(v)) for v in periodic])
    if not (pairs.device == x.device and n_pairs.device == x.device):
        raise ValueError("x, pairs and n_pairs must be on the same device")
    # the library picks its fixed array on the current device: make it x's
    with torch.cuda.device(x.device):
        if stream is None:
            stream = torch.cuda.current_stream(x.device).cuda_stream
        _check(lib.prs_find_pairs_noalloc(x.data_ptr(), int(x.shape[1]), C.cast(Lh, _vp),
                                          C.cast(ph, _vp), float(cutoff), pairs.data_ptr(),
                                          int(pairs.shape[0]), n_pairs.data_ptr(),
                                          _vp(stream)))
