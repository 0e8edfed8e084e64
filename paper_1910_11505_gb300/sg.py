"""Thin ctypes binding of the C ABI in ``include/sg.h`` (argument marshalling only).

Every computation runs in ``libsg_gb300.so``; this module only converts torch tensors to device
pointers and CUDA streams to handles.  There is no CPU fallback: if the library is missing or no
CUDA device is present, the calls raise.
"""

from __future__ import annotations

import ctypes
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("SG_LIB_PATH") or os.path.join(HERE, "_build", "libsg_gb300.so")

SG_OK = 0
SG_ERR_ARG = -1
SG_ERR_CUDA = -2
SG_ERR_OOM = -3
SG_ERR_NAN = -4
SG_ERR_NOT_CONVERGED = -5

SG_PC_NONE, SG_PC_MEAN, SG_PC_FS_GS, SG_PC_FS_JACOBI, SG_PC_MG, SG_PC_FG = 0, 1, 2, 3, 4, 5
SG_FP64, SG_MIXED_FP32, SG_MIXED_BF16 = 0, 1, 2

PRECONDS = {"none": SG_PC_NONE, "mean": SG_PC_MEAN, "fs_gs": SG_PC_FS_GS,
            "fs_jacobi": SG_PC_FS_JACOBI, "mg": SG_PC_MG, "fg": SG_PC_FG}
FG_RULES = {"paper": 0, "groups": 1, "whole": 2}
PRECISIONS = {"fp64": SG_FP64, "fp32": SG_MIXED_FP32, "bf16": SG_MIXED_BF16}
OP_KERNELS = {"auto": 0, "pairs": 1, "tile": 2}
ILU_ORDERS = {"natural": 0, "color4": 1}

EXPORTED = ["sg_default_params", "sg_setup", "sg_dims", "sg_nnz", "sg_matvec", "sg_matvec_lowp",
            "sg_precond_apply", "sg_precond_apply_lowp", "sg_precond_apply_noalloc", "sg_rhs",
            "sg_gmres_solve",
            "sg_export", "sg_launch_count", "sg_tune_plan", "sg_op_info", "sg_probe_fma",
            "sg_fg_splits",
            "sg_timing_start", "sg_timing_stop", "sg_free", "sg_last_error",
            "sgnet_create", "sgnet_set_stats", "sgnet_set_basis", "sgnet_forward", "sgnet_predict", "sgnet_loss_grad",
            "sgnet_adam_step", "sgnet_train_step", "sgnet_num_params", "sgnet_get", "sgnet_set",
            "sgnet_free"]

K_CLASSES = ["apply_f64", "apply_lowp", "ilu_solve", "gs_scatter", "arnoldi", "other"]


class SGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"SG error {code}: {msg}")
        self.code = code


class sg_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("M", ctypes.c_int), ("p", ctypes.c_int), ("q", ctypes.c_int),
                ("sigma", ctypes.c_double), ("ell", ctypes.c_double), ("a_min", ctypes.c_double),
                ("mu", ctypes.c_double), ("f", ctypes.c_double), ("precond", ctypes.c_int),
                ("inner_iters", ctypes.c_int), ("outer_sweeps", ctypes.c_int),
                ("restart", ctypes.c_int), ("max_iters", ctypes.c_int), ("rtol", ctypes.c_double),
                ("atol", ctypes.c_double), ("precision", ctypes.c_int),
                ("inner_rtol", ctypes.c_double), ("graphs", ctypes.c_int),
                ("mg_smoother", ctypes.c_int), ("mg_coarse", ctypes.c_int),
                ("op_kernel", ctypes.c_int), ("op_kappa", ctypes.c_int), ("op_ctas", ctypes.c_int),
                ("ilu_order", ctypes.c_int), ("coupling_bf16", ctypes.c_int),
                ("fg_rule", ctypes.c_int), ("fg_bf16", ctypes.c_int)]


class sg_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int), ("status", ctypes.c_int),
                ("rel_resid", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run __graft_entry__.build() (or "
                           "python paper_1910_11505_gb300/build.py) first")
    lib = ctypes.CDLL(path)
    vp, ip, c_int, c_dbl = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_double
    lib.sg_default_params.argtypes = [ctypes.POINTER(sg_params)]
    lib.sg_default_params.restype = None
    lib.sg_setup.argtypes = [ctypes.POINTER(sg_params), c_int, vp, ctypes.POINTER(vp)]
    lib.sg_dims.argtypes = [vp, c_int, ip, ip, ip]
    lib.sg_nnz.argtypes = [vp, c_int, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    lib.sg_matvec.argtypes = [vp, c_int, vp, vp, vp]
    lib.sg_matvec_lowp.argtypes = [vp, c_int, vp, vp, vp]
    lib.sg_precond_apply.argtypes = [vp, c_int, vp, vp, vp]
    lib.sg_precond_apply_lowp.argtypes = [vp, c_int, vp, vp, vp]
    lib.sg_precond_apply_noalloc.argtypes = [vp, c_int, vp, vp, vp]
    lib.sg_rhs.argtypes = [vp, c_int, vp, vp]
    lib.sg_gmres_solve.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                   ctypes.POINTER(sg_solve_info), vp]
    lib.sg_export.argtypes = [vp, c_int, c_int, vp, ctypes.c_size_t]
    lib.sg_tune_plan.argtypes = [c_int, c_int, c_int, c_int, c_int, ctypes.c_longlong,
                                 ctypes.POINTER(ctypes.c_longlong)]
    lib.sg_tune_plan.restype = c_int
    lib.sg_fg_splits.argtypes = [c_int, c_int, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]
    lib.sg_fg_splits.restype = c_int
    lib.sg_op_info.argtypes = [vp, c_int, ctypes.POINTER(ctypes.c_longlong), ctypes.c_char_p, c_int]
    lib.sg_op_info.restype = c_int
    lib.sg_probe_fma.argtypes = [c_int, ctypes.POINTER(ctypes.c_double)]
    lib.sg_probe_fma.restype = c_int
    lib.sg_launch_count.argtypes = []
    lib.sg_launch_count.restype = ctypes.c_longlong
    lib.sg_timing_start.argtypes = [vp, c_int]
    lib.sg_timing_stop.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    lib.sg_free.argtypes = [vp]
    lib.sg_free.restype = None
    fp = ctypes.POINTER(ctypes.c_float)
    lib.sgnet_create.argtypes = [c_int, c_int, c_int, c_int, c_int, c_int, ctypes.c_ulonglong,
                                 ctypes.POINTER(vp)]
    lib.sgnet_set_stats.argtypes = [vp, vp, vp, c_int, vp]
    lib.sgnet_set_basis.argtypes = [vp, vp, c_int, vp]
    lib.sgnet_forward.argtypes = [vp, vp, c_int, vp, vp]
    lib.sgnet_predict.argtypes = [vp, vp, c_int, vp, vp]
    lib.sgnet_loss_grad.argtypes = [vp, vp, vp, c_int, fp, vp]
    lib.sgnet_adam_step.argtypes = [vp, ctypes.c_float, vp]
    lib.sgnet_train_step.argtypes = [vp, vp, vp, c_int, ctypes.c_float, fp, vp]
    lib.sgnet_num_params.argtypes = [vp]
    lib.sgnet_num_params.restype = ctypes.c_longlong
    lib.sgnet_get.argtypes = [vp, c_int, fp, ctypes.c_size_t]
    lib.sgnet_set.argtypes = [vp, c_int, fp, ctypes.c_size_t]
    lib.sgnet_free.argtypes = [vp]
    lib.sgnet_free.restype = None
    for name in ("sgnet_create", "sgnet_set_stats", "sgnet_set_basis", "sgnet_forward", "sgnet_predict",
                 "sgnet_loss_grad", "sgnet_adam_step", "sgnet_train_step", "sgnet_get", "sgnet_set"):
        getattr(lib, name).restype = c_int
    lib.sg_last_error.argtypes = []
    lib.sg_last_error.restype = ctypes.c_char_p
    for name in ("sg_setup", "sg_dims", "sg_nnz", "sg_matvec", "sg_matvec_lowp", "sg_precond_apply",
                 "sg_precond_apply_lowp", "sg_precond_apply_noalloc",
                 "sg_rhs", "sg_gmres_solve", "sg_export", "sg_timing_start", "sg_timing_stop"):
        getattr(lib, name).restype = c_int
    _ = c_dbl
    _lib = lib
    return lib


def _check(rc, allow=()):
    if rc != SG_OK and rc not in allow:
        raise SGError(rc, load_library().sg_last_error().decode())
    return rc


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t, dtype_name):
    import torch
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    want = {"f64": torch.float64, "f32": torch.float32}[dtype_name]
    if t.dtype != want:
        raise ValueError(f"expected {want}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def sg_default_params(**overrides) -> sg_params:
    p = sg_params()
    load_library().sg_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if k in ("precond", "mg_smoother") and isinstance(v, str):
            v = PRECONDS[v]
        if k == "op_kernel" and isinstance(v, str):
            v = OP_KERNELS[v]
        if k == "ilu_order" and isinstance(v, str):
            v = ILU_ORDERS[v]
        if k == "fg_rule" and isinstance(v, str):
            v = FG_RULES[v]
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        setattr(p, k, v)
    return p


class SGHandle:
    """Owns an ``sg_handle*``; frees it on close() or garbage collection."""

    def __init__(self, raw, params):
        self.raw = raw
        self.params = list(params)

    def close(self):
        if self.raw:
            load_library().sg_free(self.raw)
            self.raw = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nsys(self):
        return len(self.params)


def sg_setup(params, stream=None) -> SGHandle:
    if isinstance(params, sg_params):
        params = [params]
    arr = (sg_params * len(params))(*params)
    out = ctypes.c_void_p()
    _check(load_library().sg_setup(arr, len(params), _stream_ptr(stream), ctypes.byref(out)))
    return SGHandle(out, params)


def sg_dims(h: SGHandle, sys: int = 0):
    N, P, L = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load_library().sg_dims(h.raw, sys, ctypes.byref(N), ctypes.byref(P), ctypes.byref(L)))
    return N.value, P.value, L.value


def sg_nnz(h: SGHandle, sys: int = 0):
    a, g = ctypes.c_longlong(), ctypes.c_longlong()
    _check(load_library().sg_nnz(h.raw, sys, ctypes.byref(a), ctypes.byref(g)))
    return a.value, g.value


def sg_matvec(h: SGHandle, sys: int, X, Y, stream=None):
    _check(load_library().sg_matvec(h.raw, sys, _ptr(X, "f64"), _ptr(Y, "f64"), _stream_ptr(stream)))


def sg_matvec_lowp(h: SGHandle, sys: int, X, Y, stream=None):
    _check(load_library().sg_matvec_lowp(h.raw, sys, _ptr(X, "f32"), _ptr(Y, "f32"),
                                         _stream_ptr(stream)))


def sg_precond_apply(h: SGHandle, sys: int, R, Z, stream=None):
    _check(load_library().sg_precond_apply(h.raw, sys, _ptr(R, "f64"), _ptr(Z, "f64"),
                                           _stream_ptr(stream)))


def sg_probe_fma(precision="fp64") -> float:
    """Measured FMA throughput of the current device in GFLOP/s (see include/sg.h)."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    v = ctypes.c_double()
    _check(load_library().sg_probe_fma(precision, ctypes.byref(v)))
    return v.value


def sg_op_info(h: SGHandle, sys: int = 0):
    """Operator kernels of a system: {"fp64": {...}, "fp32": {...}, "msg": str}."""
    info = (ctypes.c_longlong * 8)()
    msg = ctypes.create_string_buffer(512)
    _check(load_library().sg_op_info(h.raw, sys, info, msg, 512))
    names = {0: "none", 1: "pairs", 2: "tile"}
    out = {}
    for i, key in enumerate(("fp64", "fp32")):
        out[key] = {"kernel": names[int(info[4 * i])], "kappa": int(info[4 * i + 1]),
                    "smem": int(info[4 * i + 2]), "chunks": int(info[4 * i + 3])}
    out["msg"] = msg.value.decode()
    return out


def sg_tune_plan(n, M, p, q=0, precision="fp64", smem_max=232448):
    """Host-only plans of the row-tiled operator (see include/sg.h): a list of six dicts with keys
    kappa, ctas, fits, smem, chunks, max_slots, pairs, entries, k_kept, groups, verified, budget,
    visits, s1_steps, s2_steps."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    out = (ctypes.c_longlong * 96)()
    _check(load_library().sg_tune_plan(n, M, p, q, precision, smem_max, out))
    keys = ["kappa", "ctas", "fits", "smem", "chunks", "max_slots", "pairs", "entries", "k_kept",
            "groups", "verified", "budget", "visits", "s1_steps", "s2_steps"]
    return [dict(zip(keys, out[16 * i:16 * i + 15])) for i in range(6)]


def sg_fg_splits(M, p, rule="paper"):
    """Host-only split ranges of the grouped field split (see include/sg.h): [(f0, f1), ...]."""
    if isinstance(rule, str):
        rule = FG_RULES[rule]
    P = math.comb(M + p, p)
    out = (ctypes.c_int * (2 * P))()
    cnt = ctypes.c_int()
    _check(load_library().sg_fg_splits(M, p, rule, out, ctypes.byref(cnt)))
    return [(out[2 * i], out[2 * i + 1]) for i in range(cnt.value)]


def sg_precond_apply_lowp(h: SGHandle, sys: int, R, Z, stream=None):
    _check(load_library().sg_precond_apply_lowp(h.raw, sys, _ptr(R, "f32"), _ptr(Z, "f32"),
                                                _stream_ptr(stream)))


def sg_precond_apply_noalloc(h: SGHandle, sys: int, R, Z, stream=None):
    """Field-split Gauss-Seidel application that allocates nothing (see include/sg.h)."""
    _check(load_library().sg_precond_apply_noalloc(h.raw, sys, _ptr(R, "f64"), _ptr(Z, "f64"),
                                                   _stream_ptr(stream)))


def sg_rhs(h: SGHandle, sys: int, F, stream=None):
    _check(load_library().sg_rhs(h.raw, sys, _ptr(F, "f64"), _stream_ptr(stream)))


def sg_gmres_solve(h: SGHandle, F, X, stream=None, raise_on_error=True):
    """F, X: lists (one per system) of device N x P float64 tensors; X holds x0, receives x."""
    ns = h.nsys
    Fa = (ctypes.c_void_p * ns)(*[_ptr(f, "f64").value for f in F])
    Xa = (ctypes.c_void_p * ns)(*[_ptr(x, "f64").value for x in X])
    info = (sg_solve_info * ns)()
    rc = load_library().sg_gmres_solve(h.raw, Fa, Xa, info, _stream_ptr(stream))
    if raise_on_error:
        _check(rc, allow=(SG_ERR_NOT_CONVERGED,))
    return rc, [i.as_dict() for i in info]


def sg_export(h: SGHandle, sys: int, what: int):
    """Copy an internal array to host numpy (see sg_export in include/sg.h)."""
    import numpy as np
    N, P, L = sg_dims(h, sys)
    nnzA, nnzG = sg_nnz(h, sys)
    spec = {0: (np.float64, nnzA * L), 1: (np.int32, N + 1), 2: (np.int32, nnzA),
            3: (np.float64, h.params[sys].M), 4: (np.float64, nnzA), 5: (np.float64, nnzG * 4)}
    dt, count = spec[what]
    out = np.empty(count, dtype=dt)
    _check(load_library().sg_export(h.raw, sys, what, out.ctypes.data_as(ctypes.c_void_p),
                                    out.nbytes))
    return out


def sg_launch_count() -> int:
    return int(load_library().sg_launch_count())


def sg_timing_start(h: SGHandle, stride: int = 1):
    _check(load_library().sg_timing_start(h.raw, stride))


def sg_timing_stop(h: SGHandle):
    """Returns {class: (ms of timed launches, timed launches, queued launches)}."""
    n = len(K_CLASSES)
    ms, tm, la = (ctypes.c_double * n)(), (ctypes.c_longlong * n)(), (ctypes.c_longlong * n)()
    _check(load_library().sg_timing_stop(h.raw, ms, tm, la))
    return {c: (ms[i], tm[i], la[i]) for i, c in enumerate(K_CLASSES)}


def sg_free(h: SGHandle):
    h.close()


class SGNet:
    """Owns an ``sgnet*`` (include/sgnet.h); methods marshal torch tensors to the C ABI."""

    def __init__(self, in_dim, h1, h2, out_dim, max_batch, bf16=True, seed=1910115050):
        raw = ctypes.c_void_p()
        _check(load_library().sgnet_create(in_dim, h1, h2, out_dim, max_batch, int(bool(bf16)),
                                           seed, ctypes.byref(raw)))
        self.raw = raw
        self.dims = (in_dim, h1, h2, out_dim)
        self.max_batch = max_batch

    def close(self):
        if self.raw:
            load_library().sgnet_free(self.raw)
            self.raw = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self):
        return int(load_library().sgnet_num_params(self.raw))

    def set_basis(self, T, stream=None):
        """Output layer from the training targets' span, then kept fixed (include/sgnet.h)."""
        _check(load_library().sgnet_set_basis(self.raw, _ptr(T, "f32"), T.shape[0],
                                              _stream_ptr(stream)))

    def set_stats(self, Z, T, stream=None):
        _check(load_library().sgnet_set_stats(self.raw, _ptr(Z, "f32"), _ptr(T, "f32"), Z.shape[0],
                                              _stream_ptr(stream)))

    def forward(self, Z, Y, stream=None):
        _check(load_library().sgnet_forward(self.raw, _ptr(Z, "f32"), Z.shape[0], _ptr(Y, "f32"),
                                            _stream_ptr(stream)))

    def predict(self, Z, X, stream=None):
        _check(load_library().sgnet_predict(self.raw, _ptr(Z, "f32"), Z.shape[0], _ptr(X, "f64"),
                                            _stream_ptr(stream)))

    def loss_grad(self, Z, T, stream=None, want_loss=True):
        loss = ctypes.c_float()
        _check(load_library().sgnet_loss_grad(self.raw, _ptr(Z, "f32"), _ptr(T, "f32"), Z.shape[0],
                                              ctypes.byref(loss) if want_loss else None,
                                              _stream_ptr(stream)))
        return loss.value if want_loss else None

    def adam_step(self, lr, stream=None):
        _check(load_library().sgnet_adam_step(self.raw, ctypes.c_float(lr), _stream_ptr(stream)))

    def train_step(self, Z, T, lr, stream=None, want_loss=False):
        loss = ctypes.c_float()
        _check(load_library().sgnet_train_step(self.raw, _ptr(Z, "f32"), _ptr(T, "f32"), Z.shape[0],
                                               ctypes.c_float(lr),
                                               ctypes.byref(loss) if want_loss else None,
                                               _stream_ptr(stream)))
        return loss.value if want_loss else None

    def get(self, what):
        import numpy as np
        count = self.num_params if what in (0, 1) else 2 * self.dims[0]
        out = np.empty(count, dtype=np.float32)
        _check(load_library().sgnet_get(self.raw, what,
                                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), count))
        return out

    def set(self, what, values):
        import numpy as np
        arr = np.ascontiguousarray(values, dtype=np.float32)
        _check(load_library().sgnet_set(self.raw, what,
                                        arr.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), arr.size))
