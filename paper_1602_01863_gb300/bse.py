"""ctypes binding of the C ABI in include/bse.h (argument marshalling only).

Every computation runs in the CUDA library `libbse_gb300.so`, built in-tree by
`build.py`.  When the library is missing this module raises: there is no
Python or CPU fallback.  Device buffers are passed as raw pointers (e.g. a
torch tensor's `data_ptr()`); host buffers are numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .synth import ModelParams

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbse_gb300.so")

BSE_OK = 0
BSE_ERR_ARG = -1
BSE_ERR_OOM = -2
BSE_ERR_CUDA = -3
BSE_ERR_TIMEOUT = -4
BSE_ERR_UNSUPPORTED = -5
BSE_WARN_BREAKDOWN = 1

PREC_F64, PREC_F32, PREC_BF16 = 0, 1, 2
SCHEME_M1, SCHEME_M3, SCHEME_M2, NB1, NF_CUDA_CORES = 0, 1, 2, 16, 32
REORTH_CGS2, USE_GRAPH, PROFILE, STOP_CONVERGED = 1, 2, 4, 8

KERNEL_CLASSES = ("restrict", "kc_apply", "prolong", "near_field", "lanczos")

EXPORTED = ("bse_version", "bse_ctx_create", "bse_ctx_destroy", "bse_last_error", "bse_build_coarse",
            "bse_coarse_get_kc", "bse_free_coarse", "bse_interp_setup", "bse_free_interp", "bse_interp_info",
            "bse_dipoles", "bse_apply_h", "bse_apply_h_noalloc", "bse_haydock_run", "bse_last_kernel_times",
            "bse_spectrum", "bse_mlp_param_count", "bse_mlp_create", "bse_mlp_free", "bse_mlp_get_params",
            "bse_mlp_forward", "bse_mlp_gradients", "bse_mlp_train_step", "bse_pairs_generate",
            "bse_interp_set_learned", "bse_set_stop_rule", "bse_ctx_set_wait_limit", "bse_interp_kc_plan")


class BseError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"bse error {code}: {msg}")
        self.code = code


class bse_model(C.Structure):
    _fields_ = [("nv", C.c_int), ("nc", C.c_int),
                ("eps_inf", C.c_double), ("kappa", C.c_double), ("e_k", C.c_double),
                ("e_gap", C.c_double), ("band_width", C.c_double),
                ("direct_shells", C.c_int), ("h_const", C.c_int), ("h0", C.c_double),
                ("exchange_on", C.c_int),
                ("offsets", C.POINTER(C.c_double)), ("gen_v", C.POINTER(C.c_double)),
                ("gen_c", C.POINTER(C.c_double)), ("mu", C.POINTER(C.c_double)),
                ("dip", C.POINTER(C.c_double))]


class bse_dense_inputs(C.Structure):
    _fields_ = [("dE", C.POINTER(C.c_double)), ("P", C.POINTER(C.c_double)),
                ("Dv", C.POINTER(C.c_double)), ("Dc", C.POINTER(C.c_double))]


_lib = None
_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


def load(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run paper_1602_01863_gb300/build.py)")
    lib = C.CDLL(path)
    lib.bse_version.restype = C.c_int
    lib.bse_ctx_create.argtypes = [C.POINTER(_P), C.c_int, _P]
    lib.bse_ctx_destroy.argtypes = [_P]
    lib.bse_ctx_destroy.restype = None
    lib.bse_last_error.argtypes = [_P]
    lib.bse_last_error.restype = C.c_char_p
    lib.bse_build_coarse.argtypes = [_P, C.POINTER(bse_model), C.c_int, C.c_int, _P, C.POINTER(_P)]
    lib.bse_coarse_get_kc.argtypes = [_P, _P, _D]
    lib.bse_free_coarse.argtypes = [_P]
    lib.bse_free_coarse.restype = None
    lib.bse_interp_setup.argtypes = [_P, _P, C.c_int, C.c_int, C.c_double, C.c_int, C.POINTER(bse_dense_inputs),
                                     C.POINTER(_P)]
    lib.bse_set_stop_rule.argtypes = [_P, C.c_double, C.c_int, C.c_double, C.c_double, C.c_int, _D]
    lib.bse_ctx_set_wait_limit.argtypes = [_P, C.c_longlong]
    lib.bse_free_interp.argtypes = [_P]
    lib.bse_free_interp.restype = None
    lib.bse_interp_info.argtypes = [_P, C.POINTER(C.c_longlong)]
    lib.bse_interp_kc_plan.argtypes = [_P, _I]
    lib.bse_dipoles.argtypes = [_P, _P, C.c_int, _D, _P, _D]
    lib.bse_apply_h.argtypes = [_P, _P, C.c_int, _P, _P]
    lib.bse_apply_h_noalloc.argtypes = [_P, _P, C.c_int, _P, _P]
    lib.bse_haydock_run.argtypes = [_P, C.POINTER(_P), C.c_int, _I, _D, C.c_int, C.c_int, _D, _D, _D, _I]
    lib.bse_last_kernel_times.argtypes = [_P, _D, C.POINTER(C.c_longlong)]
    lib.bse_spectrum.argtypes = [_P, C.c_int, C.c_int, _I, _D, _D, _D, C.c_double, C.c_double, C.c_int, _D, _D]
    _F = C.POINTER(C.c_float)
    lib.bse_mlp_param_count.argtypes = [C.c_int]
    lib.bse_mlp_create.argtypes = [_P, C.c_int, C.c_int, _F, C.POINTER(_P)]
    lib.bse_mlp_free.argtypes = [_P]
    lib.bse_mlp_free.restype = None
    lib.bse_mlp_get_params.argtypes = [_P, _P, _F]
    lib.bse_mlp_forward.argtypes = [_P, _P, C.c_int, _P, _P]
    lib.bse_mlp_gradients.argtypes = [_P, _P, C.c_int, _P, _P, _F, _D]
    lib.bse_mlp_train_step.argtypes = [_P, _P, C.c_int, _P, _P, C.c_float, _D]
    lib.bse_pairs_generate.argtypes = [_P, _P, C.c_int, _I, _I, _P, _P]
    lib.bse_interp_set_learned.argtypes = [_P, _P, _P, C.c_int]
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _iptr(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(_I)


def model_struct(m: ModelParams):
    """bse_model for a ModelParams; returns (struct, arrays kept alive)."""
    keep = [np.ascontiguousarray(m.offsets, dtype=np.float64),
            np.ascontiguousarray(m.gen_v, dtype=np.complex128).view(np.float64),
            np.ascontiguousarray(m.gen_c, dtype=np.complex128).view(np.float64),
            np.ascontiguousarray(m.mu, dtype=np.complex128).view(np.float64),
            np.ascontiguousarray(m.dip, dtype=np.complex128).view(np.float64)]
    s = bse_model(nv=m.nv, nc=m.nc, eps_inf=m.eps_inf, kappa=m.kappa, e_k=m.e_k, e_gap=m.e_gap,
                  band_width=m.band_width, direct_shells=m.direct_shells, h_const=int(m.h_const),
                  h0=m.h0, exchange_on=int(m.exchange_on),
                  offsets=_dptr(keep[0]), gen_v=_dptr(keep[1]), gen_c=_dptr(keep[2]),
                  mu=_dptr(keep[3]), dip=_dptr(keep[4]))
    return s, keep


class Coarse:
    def __init__(self, ctx: "Context", handle, n: int, t: int, kc_prec: int):
        self.ctx, self.handle, self.n, self.t, self.kc_prec = ctx, handle, n, t, kc_prec
        self.Nc = t * n ** 3

    def get_kc(self) -> np.ndarray:
        out = np.empty((self.Nc, self.Nc), dtype=np.complex128)
        self.ctx._check(self.ctx.lib.bse_coarse_get_kc(self.ctx.h, self.handle, out.view(np.float64).ctypes.data_as(_D)))
        return out

    def free(self):
        if self.handle:
            self.ctx.lib.bse_free_coarse(self.handle)
            self.handle = None


class Interp:
    def __init__(self, ctx: "Context", handle, coarse: Coarse):
        self.ctx, self.handle, self.coarse = ctx, handle, coarse
        info = (C.c_longlong * 8)()
        ctx._check(ctx.lib.bse_interp_info(handle, info))
        self.N, self.Nk, self.Nc, self.t, self.n, self.n_div, self.n_near, self.vec_prec = [int(x) for x in info]

    def kc_plan(self):
        """(pipeline stages, k-blocks per chunk, CTAs) of the tensor-core K_c apply, or None (K_c not BF16)."""
        plan = (C.c_int * 3)()
        rc = self.ctx.lib.bse_interp_kc_plan(self.handle, plan)
        if rc == BSE_ERR_UNSUPPORTED:
            return None
        self.ctx._check(rc)
        return tuple(int(x) for x in plan)

    def free(self):
        if self.handle:
            self.ctx.lib.bse_free_interp(self.handle)
            self.handle = None


class Mlp:
    def __init__(self, ctx: "Context", handle, d_in: int, nparams: int):
        self.ctx, self.handle, self.d_in, self.nparams = ctx, handle, d_in, nparams

    def params(self) -> np.ndarray:
        p = np.zeros(self.nparams, dtype=np.float32)
        self.ctx._check(self.ctx.lib.bse_mlp_get_params(self.ctx.h, self.handle, p.ctypes.data_as(C.POINTER(C.c_float))))
        return p

    def free(self):
        if self.handle:
            self.ctx.lib.bse_mlp_free(self.handle)
            self.handle = None


def mlp_unflatten(p: np.ndarray, d_in: int, width: int = 128):
    """FP32 parameter vector (C-ABI layout) -> [[W, b], ...] float64 (oracle layout)."""
    dims = [d_in, width, width, width, 2]
    out, o = [], 0
    for i in range(4):
        w = p[o:o + dims[i + 1] * dims[i]].reshape(dims[i + 1], dims[i]).astype(np.float64)
        o += dims[i + 1] * dims[i]
        b = p[o:o + dims[i + 1]].astype(np.float64)
        o += dims[i + 1]
        out.append([w, b])
    return out


def mlp_flatten(params) -> np.ndarray:
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in params]).astype(np.float32)


class Context:
    """bse_ctx on one device and one CUDA stream (a cudaStream_t as int, or 0)."""

    def __init__(self, device: int = 0, stream: int = 0):
        self.lib = load()
        h = _P()
        rc = self.lib.bse_ctx_create(C.byref(h), device, _P(stream) if stream else None)
        if rc != BSE_OK:
            raise BseError(rc, "bse_ctx_create failed (no CUDA device?)")
        self.h = h

    def _check(self, rc: int) -> int:
        if rc < 0:
            raise BseError(rc, self.lib.bse_last_error(self.h).decode())
        return rc

    def close(self):
        if self.h:
            self.lib.bse_ctx_destroy(self.h)
            self.h = None

    # -- bse_build_coarse
    def bse_build_coarse(self, model: ModelParams, n_coarse: int, kc_prec: int = PREC_F64,
                         user_kc_ptr: int = 0) -> Coarse:
        """user_kc_ptr: device address of a complex128 [N_c, N_c] K_c replacing the model's (0: none)."""
        s, keep = model_struct(model)
        h = _P()
        self._check(self.lib.bse_build_coarse(self.h, C.byref(s), n_coarse, kc_prec,
                                              _P(user_kc_ptr) if user_kc_ptr else None, C.byref(h)))
        del keep
        return Coarse(self, h, n_coarse, model.nv * model.nc, kc_prec)

    # -- bse_interp_setup
    def bse_interp_setup(self, coarse: Coarse, n_div: int, scheme: int = SCHEME_M1, width: float = 1.0,
                         vec_prec: int = PREC_F64, dense: dict | None = None) -> Interp:
        """dense: optional host arrays replacing the model's dense tables, keys
        'dE' (float64 [N]), 'P' (complex128 [3, N]), 'Dv' (complex128 [N_k, 8, nv, nv]),
        'Dc' (complex128 [N_k, 8, nc, nc])."""
        h = _P()
        keep, din = [], None
        if dense:
            din = bse_dense_inputs()
            for key, dt in (("dE", np.float64), ("P", np.complex128), ("Dv", np.complex128), ("Dc", np.complex128)):
                if dense.get(key) is not None:
                    arr = np.ascontiguousarray(dense[key], dtype=dt)
                    keep.append(arr)
                    setattr(din, key, arr.view(np.float64).ctypes.data_as(_D))
        self._check(self.lib.bse_interp_setup(self.h, coarse.handle, n_div, scheme, float(width), vec_prec,
                                              C.byref(din) if din is not None else None, C.byref(h)))
        del keep
        return Interp(self, h, coarse)

    # -- bse_ctx_set_wait_limit (testing aid for the failure path)
    def bse_ctx_set_wait_limit(self, cycles: int) -> None:
        self._check(self.lib.bse_ctx_set_wait_limit(self.h, int(cycles)))

    # -- bse_set_stop_rule
    def bse_set_stop_rule(self, tol: float, check_every: int, s_eps: float, eta: float, omega: np.ndarray) -> None:
        w = np.ascontiguousarray(omega, dtype=np.float64)
        self._check(self.lib.bse_set_stop_rule(self.h, float(tol), int(check_every), float(s_eps), float(eta),
                                               w.size, _dptr(w)))

    # -- bse_dipoles
    def bse_dipoles(self, interp: Interp, pol_dirs: np.ndarray, out_ptr: int) -> np.ndarray:
        dirs = np.ascontiguousarray(pol_dirs, dtype=np.float64).reshape(-1, 3)
        pn2 = np.empty(dirs.shape[0])
        self._check(self.lib.bse_dipoles(self.h, interp.handle, dirs.shape[0], _dptr(dirs), _P(out_ptr), _dptr(pn2)))
        return pn2

    # -- bse_apply_h
    def bse_apply_h(self, interp: Interp, nvec: int, x_ptr: int, y_ptr: int) -> None:
        self._check(self.lib.bse_apply_h(self.h, interp.handle, nvec, _P(x_ptr), _P(y_ptr)))

    # -- bse_apply_h_noalloc (scratch from the library's static device array)
    def bse_apply_h_noalloc(self, interp: Interp, nvec: int, x_ptr: int, y_ptr: int) -> None:
        self._check(self.lib.bse_apply_h_noalloc(self.h, interp.handle, nvec, _P(x_ptr), _P(y_ptr)))

    # -- bse_haydock_run
    def bse_haydock_run(self, systems: list[Interp], npol: list[int], pol_dirs: np.ndarray, nsteps: int,
                        flags: int = 0):
        nsys = len(systems)
        handles = (_P * nsys)(*[s.handle for s in systems])
        npol_a = np.ascontiguousarray(npol, dtype=np.int32)
        chains = int(npol_a.sum())
        dirs = np.ascontiguousarray(pol_dirs, dtype=np.float64).reshape(chains, 3)
        a = np.zeros((chains, nsteps))
        b = np.zeros((chains, nsteps + 1))
        pn2 = np.zeros(chains)
        steps = np.zeros(chains, dtype=np.int32)
        rc = self._check(self.lib.bse_haydock_run(self.h, handles, nsys, _iptr(npol_a), _dptr(dirs), nsteps, flags,
                                                  _dptr(a), _dptr(b), _dptr(pn2), _iptr(steps)))
        return a, b, pn2, steps, rc

    def bse_last_kernel_times(self):
        ms = np.zeros(5)
        cnt = (C.c_longlong * 5)()
        self._check(self.lib.bse_last_kernel_times(self.h, _dptr(ms), cnt))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_CLASSES)}

    # -- learned near-diagonal residual
    def bse_mlp_create(self, d_in: int, max_batch: int, init_params: np.ndarray) -> "Mlp":
        p = np.ascontiguousarray(init_params, dtype=np.float32)
        assert p.size == self.lib.bse_mlp_param_count(d_in)
        h = _P()
        self._check(self.lib.bse_mlp_create(self.h, d_in, max_batch, p.ctypes.data_as(C.POINTER(C.c_float)), C.byref(h)))
        return Mlp(self, h, d_in, int(p.size))

    def bse_mlp_forward(self, mlp: "Mlp", batch: int, X_ptr: int, out_ptr: int) -> None:
        self._check(self.lib.bse_mlp_forward(self.h, mlp.handle, batch, _P(X_ptr), _P(out_ptr)))

    def bse_mlp_gradients(self, mlp: "Mlp", batch: int, X_ptr: int, Y_ptr: int):
        g = np.zeros(mlp.nparams, dtype=np.float32)
        loss = C.c_double()
        self._check(self.lib.bse_mlp_gradients(self.h, mlp.handle, batch, _P(X_ptr), _P(Y_ptr),
                                               g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss)))
        return g, loss.value

    def bse_mlp_train_step(self, mlp: "Mlp", batch: int, X_ptr: int, Y_ptr: int, lr: float) -> float:
        loss = C.c_double()
        self._check(self.lib.bse_mlp_train_step(self.h, mlp.handle, batch, _P(X_ptr), _P(Y_ptr), float(lr), C.byref(loss)))
        return loss.value

    def bse_pairs_generate(self, interp: Interp, kd: np.ndarray, kd2: np.ndarray, X_ptr: int, Y_ptr: int) -> None:
        a = np.ascontiguousarray(kd, dtype=np.int32)
        b = np.ascontiguousarray(kd2, dtype=np.int32)
        self._check(self.lib.bse_pairs_generate(self.h, interp.handle, a.size, _iptr(a), _iptr(b), _P(X_ptr), _P(Y_ptr)))

    def bse_interp_set_learned(self, interp: Interp, mlp: "Mlp | None", radius: int) -> None:
        self._check(self.lib.bse_interp_set_learned(self.h, interp.handle, mlp.handle if mlp else None, radius))

    # -- bse_spectrum
    def bse_spectrum(self, a: np.ndarray, b: np.ndarray, pnorm2: np.ndarray, steps_done: np.ndarray,
                     prefactor: float, eta: float, omega: np.ndarray) -> np.ndarray:
        a = np.ascontiguousarray(a, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        nch, m = a.shape
        pn2 = np.ascontiguousarray(pnorm2, dtype=np.float64)
        st = np.ascontiguousarray(steps_done, dtype=np.int32)
        w = np.ascontiguousarray(omega, dtype=np.float64)
        eps = np.zeros((nch, w.size), dtype=np.complex128)
        self._check(self.lib.bse_spectrum(self.h, nch, m, _iptr(st), _dptr(a), _dptr(b), _dptr(pn2), prefactor, eta,
                                          w.size, _dptr(w), eps.view(np.float64).ctypes.data_as(_D)))
        return eps
