"""Thin ctypes binding over the C ABI of libisam.so (include/isam.h).

Argument marshalling only: every step of the forward model, the adjoint and
the solve runs in the library's CUDA kernels.  PyTorch provides device
memory and the current CUDA stream.  There is no CPU fallback: if the shared
library is missing or cannot be loaded, the import of this module fails.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libisam.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run `python __graft_entry__.py` (build())")

_lib = ctypes.CDLL(LIB_PATH)

ISAM_FP32, ISAM_FP64 = 0, 1
ISAM_FLAG_NO_STOLT_TABLE = 1
ISAM_FLAG_AXIAL_MODEL = 4
STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error",
          4: "non-finite value in the solve", 6: "unsupported size or option"}


class IsamParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nk", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("k_min", ctypes.c_double), ("k_max", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("na", ctypes.c_double),
                ("z0", ctypes.c_double), ("n_disp", ctypes.c_int32),
                ("disp", ctypes.c_double * 4), ("precision", ctypes.c_int32),
                ("nufft_J", ctypes.c_int32), ("nufft_os", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("lambda_rel", ctypes.c_double), ("lambda_abs", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("tol", ctypes.c_double),
                ("check_every", ctypes.c_int32), ("w_dev", ctypes.c_void_p),
                ("residual_addback", ctypes.c_int32), ("L", ctypes.c_double),
                ("eps", ctypes.c_double), ("prior", ctypes.c_int32),
                ("objective", ctypes.c_int32), ("prior_iters", ctypes.c_int32)]


PRIORS = {"l1": 0, "haar_depth": 1, "tv": 2}


class SolveState(ctypes.Structure):
    _fields_ = [("z1", ctypes.c_void_p), ("z2", ctypes.c_void_p), ("k", ctypes.c_int32),
                ("lambda_", ctypes.c_double), ("L", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("rr", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("L", ctypes.c_double), ("status", ctypes.c_int32),
                ("objective", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("lateral_tile", ctypes.c_int32), ("stolt_table", ctypes.c_int32),
                ("axial_radix", ctypes.c_int32), ("lateral_radix", ctypes.c_int32)]


_P = ctypes.c_void_p
_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_SIGS = {
    "isam_plan_create": (ctypes.c_int, [ctypes.POINTER(IsamParams), _P, ctypes.POINTER(_P)]),
    "isam_plan_destroy": (None, [_P]),
    "isam_set_stream": (ctypes.c_int, [_P, _P]),
    "isam_forward": (ctypes.c_int, [_P, _P, _P]),
    "isam_adjoint": (ctypes.c_int, [_P, _P, _P]),
    "isam_solve": (ctypes.c_int, [_P, _P, ctypes.POINTER(SolveOpts), _P,
                                  ctypes.POINTER(SolveState), ctypes.POINTER(SolveInfo)]),
    "isam_solve_host": (ctypes.c_int, [_P, _P, ctypes.POINTER(SolveOpts), _P,
                                       ctypes.POINTER(SolveInfo)]),
    "isam_lipschitz": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double, _P,
                                      ctypes.POINTER(ctypes.c_double)]),
    "isam_max_abs": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_double)]),
    "isam_last_launch_count": (ctypes.c_int64, [_P]),
    "isam_profile_enable": (ctypes.c_int, [_P, ctypes.c_int32]),
    "isam_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]),
    "isam_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "isam_set_allocator": (ctypes.c_int, [_P, _P, _P]),     # function pointers as void*
    "isam_dispersion_compensated_ifft": (ctypes.c_int, [_P, _P, _P]),
    "isam_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, ctypes.POINTER(_P),
                                         ctypes.POINTER(SolveOpts), ctypes.POINTER(_P), _P,
                                         ctypes.POINTER(_P)]),
    "isam_batch_run": (ctypes.c_int, [_P, ctypes.POINTER(SolveInfo)]),
    "isam_autotune": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_int32)]),
    "isam_autotune_ex": (ctypes.c_int, [_P, ctypes.POINTER(Tuning)]),
    "isam_get_tuning": (ctypes.c_int, [_P, ctypes.POINTER(Tuning)]),
    "isam_set_tuning": (ctypes.c_int, [_P, ctypes.POINTER(Tuning)]),
    "isam_batch_kernel_count": (ctypes.c_int64, [_P]),
    "isam_data_fidelity": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    "isam_batch_entry_ms": (ctypes.c_int, [_P, _P]),
    "isam_batch_destroy": (None, [_P]),
    "isam_set_filter": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "isam_set_model": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                      ctypes.c_double]),
    "isam_param_grad": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    "isam_unrolled_checkpoint_images": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int32]),
    "isam_fista_unrolled": (ctypes.c_int, [_P, _P, ctypes.POINTER(SolveOpts), ctypes.c_int32,
                                           _P, _P]),
    "isam_fista_unrolled_vjp": (ctypes.c_int, [_P, _P, ctypes.POINTER(SolveOpts),
                                               ctypes.c_int32, _P, _P, _P,
                                               ctypes.POINTER(ctypes.c_double)]),
}
N_PARAMS = 5
PARAM_NAMES = ("a1", "a2", "a3", "a4", "z0")
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class IsamError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS.get(status, status)} (status {status})")
        self.status = status


def _check(st: int, where: str) -> None:
    if st != 0:
        raise IsamError(st, where)


def lib() -> ctypes.CDLL:
    return _lib


def make_params(geom, precision: str = "fp32", J: int = 6, stolt_table: bool = True,
                axial_model: bool = False) -> IsamParams:
    p = IsamParams()
    p.nx, p.ny, p.nk, p.nz = int(geom.nx), int(geom.ny), int(geom.nk), int(geom.nz or geom.nk)
    p.k_min, p.k_max = float(geom.k_min), float(geom.k_max)
    p.dx, p.dy = float(geom.dx), float(geom.dy)
    p.na, p.z0 = float(geom.na), float(geom.z0)
    disp = list(geom.disp) + [0.0] * (4 - len(geom.disp))
    p.n_disp = 4
    for i in range(4):
        p.disp[i] = float(disp[i])
    p.precision = ISAM_FP64 if precision == "fp64" else ISAM_FP32
    p.nufft_J = int(J)
    p.nufft_os = 2
    p.flags = (0 if stolt_table else ISAM_FLAG_NO_STOLT_TABLE) | \
        (ISAM_FLAG_AXIAL_MODEL if axial_model else 0)
    return p


def _stream_handle(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


# Every callback pair ever installed stays referenced: blocks are returned to
# the allocator that made them, possibly after another one was installed.
_ALLOCATORS = []


def set_allocator(alloc=None, free=None) -> None:
    """isam_set_allocator with Python callables: alloc(nbytes) -> device pointer
    (int, 0 on failure), free(ptr).  No arguments restores cudaMalloc."""
    if alloc is None and free is None:
        _check(_lib.isam_set_allocator(None, None, None), "isam_set_allocator")
        return

    def _a(n, ctx):
        try:
            return alloc(int(n)) or None
        except Exception:
            return None

    def _f(ptr, ctx):
        try:
            free(int(ptr))
        except Exception:
            pass
    pair = (_ALLOC_T(_a), _FREE_T(_f))
    _ALLOCATORS.append(pair)
    _check(_lib.isam_set_allocator(ctypes.cast(pair[0], _P), ctypes.cast(pair[1], _P), None),
           "isam_set_allocator")


def use_torch_allocator() -> None:
    """Plan workspace and tables from PyTorch's caching allocator."""
    import torch
    set_allocator(lambda n: torch.cuda.caching_allocator_alloc(n),
                  lambda p: torch.cuda.caching_allocator_delete(p))


class Plan:
    """A plan for one geometry: isam_plan_create / isam_forward / isam_adjoint / isam_solve."""

    def __init__(self, geom, precision: str = "fp32", J: int = 6, stream=None,
                 stolt_table: bool = True, axial_model: bool = False):
        import torch
        self.geom = geom
        self.precision = precision
        self.real_dtype = torch.float64 if precision == "fp64" else torch.float32
        self.cplx_dtype = torch.complex128 if precision == "fp64" else torch.complex64
        self.image_shape = (geom.ny, geom.nx, geom.nz or geom.nk)
        self.spec_shape = (geom.ny, geom.nx, geom.nk)
        self._params = make_params(geom, precision, J, stolt_table, axial_model)
        h = _P()
        _check(_lib.isam_plan_create(ctypes.byref(self._params), _P(_stream_handle(stream)),
                                     ctypes.byref(h)), "isam_plan_create")
        self._h = h

    # -- helpers -----------------------------------------------------------------
    def _dev(self, t, dtype, shape, name):
        import torch
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
            raise ValueError(f"{name}: need contiguous {dtype} {shape}, got {t.dtype} "
                             f"{tuple(t.shape)}")
        return _P(t.data_ptr())

    def _sync_stream(self):
        _check(_lib.isam_set_stream(self._h, _P(_stream_handle(None))), "isam_set_stream")

    @property
    def handle(self):
        return self._h

    def last_launch_count(self) -> int:
        return int(_lib.isam_last_launch_count(self._h))

    KERNEL_CLASSES = ("ax_fwd", "ax_adj", "ax_fused", "lat_update", "lat_fft", "misc")

    def profile(self, on: bool) -> None:
        """Time every kernel launch of this plan with CUDA events (per class)."""
        self._sync_stream()
        _check(_lib.isam_profile_enable(self._h, int(bool(on))), "isam_profile_enable")

    def profile_read(self, reset: bool = True) -> dict:
        n = len(self.KERNEL_CLASSES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        _check(_lib.isam_profile_read(self._h, ms, cnt, int(bool(reset))), "isam_profile_read")
        return {k: (ms[i], cnt[i]) for i, k in enumerate(self.KERNEL_CLASSES)}

    # -- operators ---------------------------------------------------------------
    def forward(self, eta, out=None):
        """s = A eta (real spectra)."""
        import torch
        self._sync_stream()
        if out is None:
            out = torch.empty(self.spec_shape, dtype=self.real_dtype, device=eta.device)
        _check(_lib.isam_forward(self._h, self._dev(eta, self.cplx_dtype, self.image_shape, "eta"),
                                 self._dev(out, self.real_dtype, self.spec_shape, "out")),
               "isam_forward")
        return out

    def data_fidelity(self, eta, s_d, r_out=None):
        """isam_data_fidelity: (1/2 ||A eta - s_d||^2, residual spectra A eta - s_d)."""
        import torch
        self._sync_stream()
        if r_out is None:
            r_out = torch.empty(self.spec_shape, dtype=self.real_dtype, device=eta.device)
        v = ctypes.c_double()
        _check(_lib.isam_data_fidelity(
            self._h, self._dev(eta, self.cplx_dtype, self.image_shape, "eta"),
            self._dev(s_d, self.real_dtype, self.spec_shape, "s_d"),
            self._dev(r_out, self.real_dtype, self.spec_shape, "r_out"), ctypes.byref(v)),
            "isam_data_fidelity")
        return v.value, r_out

    def adjoint(self, s, out=None):
        """eta = A^H s."""
        import torch
        self._sync_stream()
        if out is None:
            out = torch.empty(self.image_shape, dtype=self.cplx_dtype, device=s.device)
        _check(_lib.isam_adjoint(self._h, self._dev(s, self.real_dtype, self.spec_shape, "s"),
                                 self._dev(out, self.cplx_dtype, self.image_shape, "out")),
               "isam_adjoint")
        return out

    def dispersion_compensated_ifft(self, s, out=None):
        """Eq. 9: the direct full-range reconstruction of every A-scan."""
        import torch
        self._sync_stream()
        if out is None:
            out = torch.empty(self.image_shape, dtype=self.cplx_dtype, device=s.device)
        _check(_lib.isam_dispersion_compensated_ifft(
            self._h, self._dev(s, self.real_dtype, self.spec_shape, "s"),
            self._dev(out, self.cplx_dtype, self.image_shape, "out")),
            "isam_dispersion_compensated_ifft")
        return out

    def _opts(self, lambda_rel, lambda_abs, max_iter, tol, check_every, w, addback, L, eps,
              prior="l1", objective=False, prior_iters=0):
        o = SolveOpts()
        o.prior = PRIORS[prior]
        o.prior_iters = int(prior_iters)
        o.objective = int(bool(objective))
        o.lambda_rel, o.lambda_abs = float(lambda_rel), float(lambda_abs)
        o.max_iter, o.tol, o.check_every = int(max_iter), float(tol), int(check_every)
        o.w_dev = None if w is None else self._dev(w, self.real_dtype, (self.image_shape[2],), "w")
        o.residual_addback = int(bool(addback))
        o.L, o.eps = float(L), float(eps)
        return o

    def solve(self, s, lambda_rel=0.01, lambda_abs=0.0, max_iter=100, tol=0.0, check_every=10,
              w=None, addback=False, L=0.0, eps=0.0, out=None, state: Optional[dict] = None,
              prior: str = "l1", objective: bool = False, prior_iters: int = 0):
        """MBIR solve (Alg. 1).  Returns (eta, info dict).  ``state`` (optional) is a dict
        with CUDA tensors 'z1', 'z2' (images) and ints/floats 'k', 'lambda', 'L'; it is
        updated in place for checkpoint / resume."""
        import torch
        self._sync_stream()
        if out is None:
            out = torch.empty(self.image_shape, dtype=self.cplx_dtype, device=s.device)
        o = self._opts(lambda_rel, lambda_abs, max_iter, tol, check_every, w, addback, L, eps,
                       prior, objective, prior_iters)
        info = SolveInfo()
        st_ptr = None
        if state is not None:
            st = SolveState()
            st.z1 = self._dev(state["z1"], self.cplx_dtype, self.image_shape, "state.z1")
            st.z2 = self._dev(state["z2"], self.cplx_dtype, self.image_shape, "state.z2")
            st.k = int(state.get("k", 0))
            st.lambda_ = float(state.get("lambda", 0.0))
            st.L = float(state.get("L", 0.0))
            st_ptr = ctypes.byref(st)
        _check(_lib.isam_solve(self._h, self._dev(s, self.real_dtype, self.spec_shape, "s"),
                               ctypes.byref(o), self._dev(out, self.cplx_dtype, self.image_shape,
                                                          "out"), st_ptr, ctypes.byref(info)),
               "isam_solve")
        if state is not None:
            state["k"], state["lambda"], state["L"] = st.k, st.lambda_, st.L
        return out, dict(iterations=info.iterations, rr=info.rr, lam=info.lambda_, L=info.L,
                         status=info.status, objective=info.objective)

    def solve_host(self, s_host, out_host, lambda_rel=0.01, lambda_abs=0.0, max_iter=100,
                   tol=0.0, check_every=10, L=0.0, eps=0.0, addback=False):
        """Solve with host buffers (CPU tensors, ideally pinned): copies in and out."""
        self._sync_stream()
        o = self._opts(lambda_rel, lambda_abs, max_iter, tol, check_every, None, addback, L, eps)
        info = SolveInfo()
        for t, dt, shp, nm in ((s_host, self.real_dtype, self.spec_shape, "s_host"),
                               (out_host, self.cplx_dtype, self.image_shape, "out_host")):
            if t.is_cuda or t.dtype != dt or tuple(t.shape) != shp or not t.is_contiguous():
                raise ValueError(f"{nm}: need contiguous host {dt} {shp}")
        _check(_lib.isam_solve_host(self._h, _P(s_host.data_ptr()), ctypes.byref(o),
                                    _P(out_host.data_ptr()), ctypes.byref(info)),
               "isam_solve_host")
        return dict(iterations=info.iterations, rr=info.rr, lam=info.lambda_, L=info.L,
                    status=info.status)

    def lipschitz(self, iters=0, rtol=0.0, v0=None) -> float:
        """L = ||A^H A|| by power iteration; iters = 0 uses the library default
        (the estimate isam_solve caches when no L is given)."""
        self._sync_stream()
        L = ctypes.c_double()
        p = None if v0 is None else self._dev(v0, self.cplx_dtype, self.image_shape, "v0")
        _check(_lib.isam_lipschitz(self._h, int(iters), float(rtol), p, ctypes.byref(L)),
               "isam_lipschitz")
        return L.value

    # -- calibration of theta = (a1, a2, a3, a4, z0) -----------------------------
    def set_model(self, disp, z0: float) -> None:
        """isam_set_model: new dispersion coefficients a_1.. (up to 4) and focal depth."""
        self._sync_stream()
        self._theta = None
        d = [float(v) for v in disp]
        arr = (ctypes.c_double * 4)(*(d + [0.0] * (4 - len(d))))
        _check(_lib.isam_set_model(self._h, len(d), arr, float(z0)), "isam_set_model")

    def set_filter(self, table) -> None:
        """isam_set_filter: complex table [ny//2 + 1, nx//2 + 1, nk] over |q| classes
        (B of Eq. 3), or None for B = 1."""
        import numpy as np
        self._sync_stream()
        if table is None:
            _check(_lib.isam_set_filter(self._h, None), "isam_set_filter")
            return
        g = self.geom
        shape = ((g.ny // 2 + 1) if g.ny > 1 else 1, g.nx // 2 + 1, g.nk)
        t = np.ascontiguousarray(np.broadcast_to(np.asarray(table, np.complex128), shape))
        buf = t.view(np.float64).ravel()
        _check(_lib.isam_set_filter(self._h, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "isam_set_filter")

    def param_grad(self, x, y):
        """isam_param_grad: <dA/dtheta x, y> for theta = (a1..a4, z0), as a float64 array."""
        import numpy as np
        self._sync_stream()
        g = (ctypes.c_double * N_PARAMS)()
        _check(_lib.isam_param_grad(self._h, self._dev(x, self.cplx_dtype, self.image_shape, "x"),
                                    self._dev(y, self.real_dtype, self.spec_shape, "y"), g),
               "isam_param_grad")
        return np.array(g[:], dtype=np.float64)

    def _unrolled_opts(self, lam, L, K, w):
        return self._opts(0.0, lam, K, 0.0, 1, w, False, L, 0.0)

    def fista_unrolled(self, s, lam: float, L: float, K: int, every: int = 5, w=None,
                       checkpoints: bool = True):
        """isam_fista_unrolled: (z^K, checkpoint images or None)."""
        import torch
        self._sync_stream()
        o = self._unrolled_opts(lam, L, K, w)
        z = torch.empty(self.image_shape, dtype=self.cplx_dtype, device=s.device)
        ck = None
        if checkpoints:
            n = int(_lib.isam_unrolled_checkpoint_images(int(K), int(every)))
            ck = torch.empty((n,) + self.image_shape, dtype=self.cplx_dtype, device=s.device)
        _check(_lib.isam_fista_unrolled(self._h, self._dev(s, self.real_dtype, self.spec_shape, "s"),
                                        ctypes.byref(o), int(every),
                                        None if ck is None else _P(ck.data_ptr()),
                                        self._dev(z, self.cplx_dtype, self.image_shape, "z")),
               "isam_fista_unrolled")
        return z, ck

    def fista_unrolled_vjp(self, s, lam: float, L: float, K: int, every: int, ckpt, z_bar,
                           want_s_bar: bool = False, w=None):
        """isam_fista_unrolled_vjp: (d<z_bar, z^K>/dtheta as float64 array, d/ds_d or None)."""
        import numpy as np
        import torch
        self._sync_stream()
        o = self._unrolled_opts(lam, L, K, w)
        n = int(_lib.isam_unrolled_checkpoint_images(int(K), int(every)))
        if ckpt is None or tuple(ckpt.shape) != (n,) + self.image_shape or \
                ckpt.dtype != self.cplx_dtype or not ckpt.is_cuda or not ckpt.is_contiguous():
            raise ValueError(f"ckpt: need contiguous CUDA {self.cplx_dtype} {(n,) + self.image_shape}")
        sb = torch.empty(self.spec_shape, dtype=self.real_dtype, device=s.device) \
            if want_s_bar else None
        g = (ctypes.c_double * N_PARAMS)()
        _check(_lib.isam_fista_unrolled_vjp(
            self._h, self._dev(s, self.real_dtype, self.spec_shape, "s"), ctypes.byref(o),
            int(every), _P(ckpt.data_ptr()),
            self._dev(z_bar, self.cplx_dtype, self.image_shape, "z_bar"),
            None if sb is None else _P(sb.data_ptr()), g), "isam_fista_unrolled_vjp")
        return np.array(g[:], dtype=np.float64), sb

    @staticmethod
    def _tuning_dict(t: "Tuning") -> dict:
        return {"lateral_tile": t.lateral_tile, "stolt_table": bool(t.stolt_table),
                "axial_radix": t.axial_radix, "lateral_radix": t.lateral_radix}

    def autotune(self) -> dict:
        """isam_autotune_ex: time the plan's own iteration over the feasible tiles,
        table modes and FFT radices, and keep the fastest."""
        self._sync_stream()
        t = Tuning()
        _check(_lib.isam_autotune_ex(self._h, ctypes.byref(t)), "isam_autotune_ex")
        return self._tuning_dict(t)

    def tuning(self) -> dict:
        """isam_get_tuning: the launch shapes and radices the plan uses."""
        t = Tuning()
        _check(_lib.isam_get_tuning(self._h, ctypes.byref(t)), "isam_get_tuning")
        return self._tuning_dict(t)

    def set_tuning(self, lateral_tile=0, stolt_table=None, axial_radix=16,
                   lateral_radix=16) -> None:
        """isam_set_tuning; stolt_table None keeps the table when the plan has one."""
        self._sync_stream()
        if stolt_table is None:
            stolt_table = self.tuning()["stolt_table"]
        t = Tuning(int(lateral_tile), int(bool(stolt_table)), int(axial_radix),
                   int(lateral_radix))
        _check(_lib.isam_set_tuning(self._h, ctypes.byref(t)), "isam_set_tuning")

    def max_abs(self, eta) -> float:
        self._sync_stream()
        v = ctypes.c_double()
        _check(_lib.isam_max_abs(self._h, self._dev(eta, self.cplx_dtype, self.image_shape, "eta"),
                                 ctypes.byref(v)), "isam_max_abs")
        return v.value

    def close(self):
        if getattr(self, "_h", None):
            _lib.isam_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """isam_batch_create / isam_batch_run: independent solves of several plans
    recorded once as one CUDA graph and replayed with one launch.

    ``entries`` is a list of (plan, s_d, out, solve keyword dict); the keywords
    are those of Plan.solve (lambda_rel, lambda_abs, max_iter, tol, check_every,
    w, addback, L, eps, prior, prior_iters).  With tol > 0 the stop rule runs
    on the device inside the graph and run() reports each entry's stopping
    iteration and r_r.  The tensors are kept referenced by the batch."""

    def __init__(self, entries, stream=None):
        self._h = None
        n = len(entries)
        self._keep = []
        plans = (_P * n)()
        sds = (_P * n)()
        outs = (_P * n)()
        opts = (SolveOpts * n)()
        for i, (plan, s, out, kw) in enumerate(entries):
            plan._sync_stream()
            plans[i] = plan._h
            sds[i] = plan._dev(s, plan.real_dtype, plan.spec_shape, "s_d")
            outs[i] = plan._dev(out, plan.cplx_dtype, plan.image_shape, "out")
            opts[i] = plan._opts(kw.get("lambda_rel", 0.01), kw.get("lambda_abs", 0.0),
                                 kw.get("max_iter", 100), kw.get("tol", 0.0),
                                 kw.get("check_every", 10), kw.get("w"),
                                 kw.get("addback", False), kw.get("L", 0.0), kw.get("eps", 0.0),
                                 kw.get("prior", "l1"), False, kw.get("prior_iters", 0))
            self._keep.append((plan, s, out, kw.get("w")))
        self.n = n
        h = _P()
        sh = None if stream is None else _P(int(stream.cuda_stream))
        _check(_lib.isam_batch_create(plans, n, sds, opts, outs, sh, ctypes.byref(h)),
               "isam_batch_create")
        self._h = h

    def run(self):
        import torch
        torch.cuda.current_stream().synchronize()
        infos = (SolveInfo * self.n)()
        st = _lib.isam_batch_run(self._h, infos)
        if st not in (0, 4):            # a non-finite entry is reported in its info
            _check(st, "isam_batch_run")
        return [dict(iterations=f.iterations, rr=f.rr, lam=f.lambda_, L=f.L, status=f.status)
                for f in infos]

    def kernel_count(self) -> int:
        return int(_lib.isam_batch_kernel_count(self._h))

    def entry_ms(self) -> list:
        """Per-entry latency of the last run: device ms from the graph's start
        to the end of each entry's solve."""
        ms = (ctypes.c_double * self.n)()
        _check(_lib.isam_batch_entry_ms(self._h, ms), "isam_batch_entry_ms")
        return list(ms)

    def close(self):
        if getattr(self, "_h", None):
            _lib.isam_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

