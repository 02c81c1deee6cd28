"""ctypes binding of libmpm2p (include/mpm2p.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts NumPy arrays (host)
and torch CUDA tensors (device) to pointers, forwards the calls with the same names,
and raises ``MPMError`` on a non-zero status.  If the library is missing it raises at
import of the handle: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

(MPM_OK, MPM_ERR_ARG, MPM_ERR_CUDA, MPM_ERR_OOM, MPM_ERR_NOT_CONVERGED, MPM_ERR_STATE,
 MPM_ERR_TOO_LARGE) = range(7)
MEM_HOST, MEM_DEVICE = 0, 1
BC_DIRICHLET, BC_NEUMANN = 0, 1
PREC_FP64, PREC_FP32_IR, PREC_FP32_IR_ALL, PREC_TF32_IR, PREC_TF32X3_IR, PREC_BF16_IR = 0, 1, 2, 3, 4, 5
P_MRCM, P_DOWNSCALED = 0, 1
EXEC_GRAPH, EXEC_PDL = 1, 4

FUNCTIONS = [
    "mpm_create", "mpm_destroy", "mpm_last_error", "mpm_set_precision", "mpm_set_permeability",
    "mpm_set_source", "mpm_set_fluids", "mpm_set_boundary", "mpm_set_decomposition",
    "mpm_set_saturation", "mpm_build_basis", "mpm_eval_epsilon", "mpm_choose",
    "mpm_perturbation_solve", "mpm_interface_solve", "mpm_downscale", "mpm_saturation_step",
    "mpm_init", "mpm_step", "mpm_get_pressure", "mpm_get_flux", "mpm_get_saturation",
    "mpm_get_conductivity", "mpm_get_stats", "mpm_sync", "mpm_profile_enable", "mpm_profile_read",
    "mpm_set_execution", "mpm_set_downscale_reuse", "mpm_cfl_dt_noalloc", "mpm_get_eps_history", "mpm_get_tuning", "mpm_set_tuning",
    "mpm_autotune", "mpm_set_mpm_order", "mpm_perturbation_correction",
]
TUNE_KEYS = ["local_threads", "local_stage", "ds_threads", "ds_stage", "transport_rows", "sweep_terms"]

STAGES = ["transport", "ds_factor", "basis", "iface_factor", "perturb", "iface_solve", "downscale", "iface_up",
          "iface_down", "reconstruct"]


class MPMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mpm2p error {code}: {msg}")
        self.code = code


class Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_longlong), ("rebuilds", ctypes.c_longlong),
                ("mpm_updates", ctypes.c_longlong), ("last_eps_max", ctypes.c_double),
                ("last_dt_min", ctypes.c_double), ("ir_iters_max", ctypes.c_int),
                ("interface_dofs", ctypes.c_int), ("subdomains", ctypes.c_int), ("n_hat", ctypes.c_int),
                ("kernel_launches", ctypes.c_longlong), ("ds_factorisations", ctypes.c_longlong)]


_LIB = None


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libmpm2p (building it first if its sources are newer)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or _build.LIB
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} is missing: run paper_2103_11050_gb300.build.build() first")
    L = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    IP, DP = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    sig = {
        "mpm_create": ([ctypes.POINTER(P), I, I, I, D, D, P], I),
        "mpm_destroy": ([P], I),
        "mpm_last_error": ([P], ctypes.c_char_p),
        "mpm_set_precision": ([P, I, D, I], I),
        "mpm_set_permeability": ([P, P, I], I),
        "mpm_set_source": ([P, P, I], I),
        "mpm_set_fluids": ([P, D], I),
        "mpm_set_boundary": ([P, IP, DP, D], I),
        "mpm_set_decomposition": ([P, I, IP, I, IP, I, I, D, P], I),
        "mpm_set_saturation": ([P, P, I], I),
        "mpm_build_basis": ([P], I),
        "mpm_eval_epsilon": ([P, DP], I),
        "mpm_choose": ([P, D, IP], I),
        "mpm_perturbation_solve": ([P], I),
        "mpm_interface_solve": ([P], I),
        "mpm_downscale": ([P], I),
        "mpm_saturation_step": ([P, D, I, DP], I),
        "mpm_init": ([P, D], I),
        "mpm_step": ([P, D, D, I], I),
        "mpm_get_pressure": ([P, P, I, I], I),
        "mpm_get_flux": ([P, P, P, I], I),
        "mpm_get_saturation": ([P, P, I], I),
        "mpm_get_conductivity": ([P, P, I], I),
        "mpm_get_stats": ([P, ctypes.POINTER(Stats)], I),
        "mpm_sync": ([P], I),
        "mpm_profile_enable": ([P, I], I),
        "mpm_set_execution": ([P, I], I),
        "mpm_set_downscale_reuse": ([P, D], I),
        "mpm_cfl_dt_noalloc": ([P, P, I, I, I, D, D, D, P, P], I),
        "mpm_profile_read": ([P, DP, ctypes.POINTER(ctypes.c_longlong)], I),
        "mpm_get_eps_history": ([P, DP, IP, I, IP], I),
        "mpm_get_tuning": ([P, IP, I], I),
        "mpm_set_tuning": ([P, IP, I], I),
        "mpm_autotune": ([P, I, DP], I),
        "mpm_set_mpm_order": ([P, I], I),
        "mpm_perturbation_correction": ([P], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _LIB = L
    return L


def _stream_handle(stream):
    """cudaStream_t of a torch.cuda.Stream, a raw handle (int) or None (legacy default stream)."""
    if stream is None:
        return 0
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


def cfl_dt_noalloc(ux, uy, dt, h, M, cfl, stream=None):
    """mpm_cfl_dt_noalloc on torch CUDA tensors ux [R][ny][nx+1], uy [R][ny+1][nx], dt [R].

    The kernels address the three buffers directly, so every property they rely on is
    checked here first: float64, contiguous, on the current CUDA device, and shapes that
    agree (uy is [R][ny+1][nx] for the R, ny, nx of ux; dt holds at least R values)."""
    import torch
    for name, t in (("ux", ux), ("uy", uy), ("dt", dt)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != torch.float64 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float64 tensor")
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} is on cuda:{t.device.index}, not on the current device")
    if ux.dim() != 3:
        raise ValueError("ux must be [R][ny][nx+1]")
    R, ny, nx1 = ux.shape
    if tuple(uy.shape) != (R, ny + 1, nx1 - 1):
        raise ValueError(f"uy must be [R][ny+1][nx] = {(R, ny + 1, nx1 - 1)}, got {tuple(uy.shape)}")
    if dt.numel() < R:
        raise ValueError(f"dt must hold at least R = {R} values")
    L = load()
    rc = L.mpm_cfl_dt_noalloc(ctypes.c_void_p(ux.data_ptr()), ctypes.c_void_p(uy.data_ptr()), int(R), int(nx1 - 1),
                              int(ny), float(h), float(M), float(cfl), ctypes.c_void_p(dt.data_ptr()),
                              ctypes.c_void_p(_stream_handle(stream)))
    if rc != MPM_OK:
        raise MPMError(rc, "mpm_cfl_dt_noalloc failed")


def _ptr(x, n=None):
    """(pointer, mem) of a C-contiguous float64 NumPy array or torch tensor holding exactly n
    values (when n is given): the library reads or writes that many through the pointer, so
    a smaller buffer would be overrun.  A CUDA tensor must be on the current device (the
    context's)."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("expected a C-contiguous float64 array")
        if n is not None and x.size != n:
            raise ValueError(f"expected {n} values, got an array of {x.size}")
        return ctypes.c_void_p(x.ctypes.data), MEM_HOST
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise ValueError("expected a contiguous float64 tensor")
        if n is not None and x.numel() != n:
            raise ValueError(f"expected {n} values, got a tensor of {x.numel()}")
        if x.is_cuda and x.device.index != torch.cuda.current_device():
            raise ValueError(f"tensor on cuda:{x.device.index}, not on the current device")
        return ctypes.c_void_p(x.data_ptr()), (MEM_DEVICE if x.is_cuda else MEM_HOST)
    raise TypeError(f"unsupported array type {type(x)}")


class Context:
    """One mpm_ctx: R realisations of an nx x ny grid on [0,Lx]x[0,Ly]."""

    def __init__(self, R, nx, ny, Lx=1.0, Ly=None, stream=None):
        self.L = load()
        self.R, self.nx, self.ny = int(R), int(nx), int(ny)
        Ly = Lx * ny / nx if Ly is None else Ly
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(0 if stream is None else int(stream))
        rc = self.L.mpm_create(ctypes.byref(h), self.R, self.nx, self.ny, float(Lx), float(Ly), st)
        if rc != MPM_OK:
            raise MPMError(rc, "mpm_create failed (sizes or non-square cells)")
        self.h = h

    def _ck(self, rc):
        if rc != MPM_OK:
            raise MPMError(rc, self.L.mpm_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.mpm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- setters
    def set_precision(self, mode, ir_tol=1e-14, ir_max=30):
        self._ck(self.L.mpm_set_precision(self.h, int(mode), float(ir_tol), int(ir_max)))

    def _ncell(self):
        return self.R * self.ny * self.nx

    def set_permeability(self, K):
        p, mem = _ptr(K, self._ncell())
        self._ck(self.L.mpm_set_permeability(self.h, p, mem))

    def set_source(self, q=None):
        if q is None:
            self._ck(self.L.mpm_set_source(self.h, None, MEM_HOST))
        else:
            p, mem = _ptr(q, self._ncell())
            self._ck(self.L.mpm_set_source(self.h, p, mem))

    def set_fluids(self, M):
        self._ck(self.L.mpm_set_fluids(self.h, float(M)))

    def set_boundary(self, types, vals, s_inflow=1.0):
        t = (ctypes.c_int * 4)(*[int(v) for v in types])
        v = (ctypes.c_double * 4)(*[float(x) for x in vals])
        self._ck(self.L.mpm_set_boundary(self.h, t, v, float(s_inflow)))

    def set_decomposition(self, col_w, row_h, seg_len=4, degree=1, alpha=1.0, alpha_face=None):
        """alpha_face: None, or (alpha_x [ny][nx+1], alpha_y [ny+1][nx]) per fine face."""
        cw = (ctypes.c_int * len(col_w))(*[int(v) for v in col_w])
        rh = (ctypes.c_int * len(row_h))(*[int(v) for v in row_h])
        af = None
        if alpha_face is not None:
            ax = np.asarray(alpha_face[0], dtype=np.float64)
            ay = np.asarray(alpha_face[1], dtype=np.float64)
            if ax.shape != (self.ny, self.nx + 1) or ay.shape != (self.ny + 1, self.nx):
                raise ValueError("alpha_face must be (alpha_x [ny][nx+1], alpha_y [ny+1][nx])")
            af = np.ascontiguousarray(np.concatenate([ax.ravel(), ay.ravel()]))
        self._ck(self.L.mpm_set_decomposition(self.h, len(col_w), cw, len(row_h), rh, int(seg_len), int(degree),
                                              float(alpha), None if af is None else ctypes.c_void_p(af.ctypes.data)))

    def set_saturation(self, s):
        p, mem = _ptr(s, self._ncell())
        self._ck(self.L.mpm_set_saturation(self.h, p, mem))

    # ---- hot path
    def build_basis(self):
        self._ck(self.L.mpm_build_basis(self.h))

    def eval_epsilon(self, host=True):
        if not host:
            self._ck(self.L.mpm_eval_epsilon(self.h, None))
            return None
        out = np.zeros(self.R)
        self._ck(self.L.mpm_eval_epsilon(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def choose(self, eta, host=True):
        if not host:
            self._ck(self.L.mpm_choose(self.h, float(eta), None))
            return None
        out = np.zeros(self.R, dtype=np.int32)
        self._ck(self.L.mpm_choose(self.h, float(eta), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        return out

    def perturbation_solve(self):
        self._ck(self.L.mpm_perturbation_solve(self.h))

    def set_mpm_order(self, order):
        self._ck(self.L.mpm_set_mpm_order(self.h, int(order)))

    def perturbation_correction(self):
        self._ck(self.L.mpm_perturbation_correction(self.h))

    def interface_solve(self):
        self._ck(self.L.mpm_interface_solve(self.h))

    def downscale(self):
        self._ck(self.L.mpm_downscale(self.h))

    def saturation_step(self, cfl=0.5, n_sub=1, host=True):
        if not host:
            self._ck(self.L.mpm_saturation_step(self.h, float(cfl), int(n_sub), None))
            return None
        out = np.zeros(self.R)
        self._ck(self.L.mpm_saturation_step(self.h, float(cfl), int(n_sub),
                                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def init(self, eta):
        self._ck(self.L.mpm_init(self.h, float(eta)))

    def step(self, eta, cfl=0.5, n_sub=1):
        self._ck(self.L.mpm_step(self.h, float(eta), float(cfl), int(n_sub)))

    def sync(self):
        self._ck(self.L.mpm_sync(self.h))

    # ---- getters (host NumPy by default, or into a given array / CUDA tensor)
    def _get(self, fn, shape, out, *extra):
        if out is None:
            out = np.zeros(shape)
        p, mem = _ptr(out, int(np.prod(shape)))
        self._ck(fn(self.h, p, *extra, mem))
        return out

    def get_pressure(self, which=P_DOWNSCALED, out=None):
        if out is None:
            out = np.zeros((self.R, self.ny, self.nx))
        p, mem = _ptr(out, self._ncell())
        self._ck(self.L.mpm_get_pressure(self.h, p, int(which), mem))
        return out

    def get_flux(self, ux=None, uy=None):
        ux = np.zeros((self.R, self.ny, self.nx + 1)) if ux is None else ux
        uy = np.zeros((self.R, self.ny + 1, self.nx)) if uy is None else uy
        pu, mem = _ptr(ux, self.R * self.ny * (self.nx + 1))
        pv, mem_v = _ptr(uy, self.R * (self.ny + 1) * self.nx)
        if mem_v != mem:
            raise ValueError("ux and uy must both be host memory or both device memory")
        self._ck(self.L.mpm_get_flux(self.h, pu, pv, mem))
        return ux, uy

    def get_saturation(self, out=None):
        return self._get(self.L.mpm_get_saturation, (self.R, self.ny, self.nx), out)

    def get_conductivity(self, out=None):
        return self._get(self.L.mpm_get_conductivity, (self.R, self.ny, self.nx), out)

    def set_execution(self, graph=True, pdl=True):
        flags = (EXEC_GRAPH if graph else 0) | (EXEC_PDL if pdl else 0)
        self._ck(self.L.mpm_set_execution(self.h, flags))

    def set_downscale_reuse(self, tol):
        """Keep float32 downscaling factors while the transmissibilities stay within a relative
        tol of those they were computed from (0: refactor every step, negative: the default)."""
        self._ck(self.L.mpm_set_downscale_reuse(self.h, float(tol)))

    def profile_enable(self, on=True):
        self._ck(self.L.mpm_profile_enable(self.h, 1 if on else 0))

    def profile_read(self):
        """{stage: (ms, count)} since enabling or the last read."""
        ms = (ctypes.c_double * len(STAGES))()
        cnt = (ctypes.c_longlong * len(STAGES))()
        self._ck(self.L.mpm_profile_read(self.h, ms, cnt))
        return {name: (ms[i], cnt[i]) for i, name in enumerate(STAGES)}

    def get_eps_history(self, cap=4096):
        """(eps [R][k], rebuilt [R][k]) of the last k <= cap steps, oldest first."""
        eps = np.zeros((self.R, cap))
        reb = np.zeros((self.R, cap), dtype=np.int32)
        n = ctypes.c_int(0)
        self._ck(self.L.mpm_get_eps_history(self.h, eps.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                            reb.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(cap),
                                            ctypes.byref(n)))
        return eps[:, :n.value].copy(), reb[:, :n.value].copy()

    def get_tuning(self):
        v = (ctypes.c_int * len(TUNE_KEYS))()
        self._ck(self.L.mpm_get_tuning(self.h, v, len(TUNE_KEYS)))
        return dict(zip(TUNE_KEYS, list(v)))

    def set_tuning(self, tune):
        v = (ctypes.c_int * len(TUNE_KEYS))(*[int(tune[k]) for k in TUNE_KEYS])
        self._ck(self.L.mpm_set_tuning(self.h, v, len(TUNE_KEYS)))

    def autotune(self, reps=5):
        """Time every launch-shape candidate on this context's data and keep the fastest; returns
        (tuning dict, best ms of transport / local solve / downscaling solve / interface sweeps)."""
        ms = (ctypes.c_double * 4)()
        self._ck(self.L.mpm_autotune(self.h, int(reps), ms))
        return self.get_tuning(), list(ms)

    def get_stats(self):
        st = Stats()
        self._ck(self.L.mpm_get_stats(self.h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in Stats._fields_}
