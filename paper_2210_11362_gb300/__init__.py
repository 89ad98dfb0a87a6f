"""Python binding of libtrals: tensor-ring ALS (Yu & Li, arXiv 2210.11362) on one GB300 GPU.

Argument marshalling only: every step of the computation runs in the CUDA kernels of
``libtrals.so`` (built in-tree by ``paper_2210_11362_gb300.build``).  There is no CPU
fallback: if the library is missing or no GPU is present, the calls raise.

Functions carry the names of the C ABI in ``include/trals.h``.  Device buffers are torch
CUDA tensors (flat, holding column-major data); host buffers are numpy arrays.  Cores are
passed as numpy arrays of shape (R_n, I_n, R_{n+1}) (any memory order; the binding hands
column-major copies to the library and writes results back in place).
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtrals.so")

# trals_status
OK, E_ARG, E_OOM, E_CUDA, E_NOT_SPD, E_NONFINITE, E_TIMEOUT, E_REJECTED, E_PENDING = range(9)
STATUS_NAMES = {0: "OK", 1: "E_ARG", 2: "E_OOM", 3: "E_CUDA", 4: "E_NOT_SPD", 5: "E_NONFINITE",
                6: "E_TIMEOUT", 7: "E_REJECTED", 8: "E_PENDING"}
# trals_xtype
X_F64, X_F32, X_BF16, X_BF16PAIR = 0, 1, 2, 3
# trals_mode
MODE_FP64, MODE_FP32, MODE_BF16, MODE_BF16X3, MODE_BF16X2 = 0, 1, 2, 3, 4
MODE_NAMES = {"fp64": MODE_FP64, "fp32": MODE_FP32, "bf16": MODE_BF16, "bf16x3": MODE_BF16X3, "bf16x2": MODE_BF16X2}
# trals_solver / trals_gram
SOLVE_CHOL, SOLVE_QR, SOLVE_QRNE, SOLVE_QR_COMPRESSED = 0, 1, 2, 3
GRAM_STRUCTURED, GRAM_EXPLICIT = 0, 1

EXPORTED = [
    "trals_version", "trals_create", "trals_destroy", "trals_last_error", "trals_decompose",
    "trals_plan_create", "trals_plan_destroy", "trals_plan_set_cores", "trals_plan_get_cores",
    "trals_plan_run", "trals_plan_residuals", "trals_plan_mttsp", "trals_plan_time_mttsp", "trals_plan_core_dev",
    "trals_plan_explicit_residual", "trals_plan_footprint", "trals_plan_bytes",
    "trals_plan_launches_per_sweep", "trals_plan_mttsp_path",
    "trals_gamma", "trals_coef_matrix", "trals_coef_matrix_explicit", "trals_qr_r_factor", "trals_mttsp", "trals_mttsp_noalloc", "trals_mttsp_path", "trals_last_mttsp_path", "trals_testing_mttsp_withheld_copy", "trals_solve_chol", "trals_check_pivot_rsqrt", "trals_reconstruct",
    "trals_residual_explicit", "trals_quantize_bf16",
    "trals_server_create", "trals_server_destroy", "trals_server_submit", "trals_server_poll",
    "trals_server_wait", "trals_server_stats", "trals_server_last_error", "trals_server_set_group_limit",
    "trals_testing_server_withhold_steps",
]


class TralsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("solver", ctypes.c_int), ("gram", ctypes.c_int),
                ("explicit_residual", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("I", ctypes.c_void_p), ("R", ctypes.c_void_p), ("X", ctypes.c_void_p),
                ("xt", ctypes.c_int), ("x_on_host", ctypes.c_int), ("init_cores", ctypes.c_void_p),
                ("sweeps", ctypes.c_int), ("opts", Opts)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("sweeps", ctypes.c_int), ("submit_s", ctypes.c_double),
                ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double), ("footprint_bytes", ctypes.c_size_t)]


class ServerInfo(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int), ("active", ctypes.c_int), ("completed", ctypes.c_uint64),
                ("used_bytes", ctypes.c_size_t), ("peak_used_bytes", ctypes.c_size_t),
                ("peak_active", ctypes.c_int), ("host_start_s", ctypes.c_double),
                ("grouped_completed", ctypes.c_uint64), ("grouped_steps", ctypes.c_uint64)]


_lib = None
_vp = ctypes.c_void_p
_i32, _i64, _dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double


def lib() -> ctypes.CDLL:
    """Load libtrals.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2210_11362_gb300.build.build() "
                           "(nvcc, sm_103a); there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "trals_version": (ctypes.c_char_p, []),
        "trals_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _vp]),
        "trals_destroy": (None, [_vp]),
        "trals_last_error": (ctypes.c_char_p, [_vp]),
        "trals_decompose": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp,
                                           ctypes.c_int, _vp, _vp]),
        "trals_plan_create": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
        "trals_plan_destroy": (None, [_vp]),
        "trals_plan_set_cores": (ctypes.c_int, [_vp, _vp]),
        "trals_plan_get_cores": (ctypes.c_int, [_vp, _vp]),
        "trals_plan_run": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
        "trals_plan_residuals": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "trals_plan_mttsp": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
        "trals_plan_explicit_residual": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double)]),
        "trals_plan_footprint": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int, _vp,
                                                ctypes.POINTER(ctypes.c_size_t)]),
        "trals_plan_bytes": (ctypes.c_size_t, [_vp]),
        "trals_plan_time_mttsp": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                                 ctypes.POINTER(ctypes.c_float)]),
        "trals_plan_core_dev": (_vp, [_vp, ctypes.c_int]),
        "trals_plan_launches_per_sweep": (ctypes.c_int, [_vp]),
        "trals_plan_mttsp_path": (ctypes.c_int, [_vp, ctypes.c_int]),
        "trals_gamma": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _i64, ctypes.c_int, _vp]),
        "trals_coef_matrix": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _vp]),
        "trals_qr_r_factor": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int, _vp]),
        "trals_coef_matrix_explicit": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int,
                                                      _vp]),
        "trals_mttsp": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp,
                                       ctypes.c_int, _vp]),
        "trals_mttsp_path": (ctypes.c_int, [ctypes.c_int, _vp, _vp, ctypes.c_int, ctypes.c_int]),
        "trals_last_mttsp_path": (ctypes.c_int, [_vp]),
        "trals_testing_mttsp_withheld_copy": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int, _vp,
                                                             ctypes.c_int, _vp, ctypes.c_longlong]),
        "trals_mttsp_noalloc": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]),
        "trals_solve_chol": (ctypes.c_int, [_vp, ctypes.c_int, _i64, ctypes.c_int, _vp, _vp, _vp]),
        "trals_check_pivot_rsqrt": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp]),
        "trals_reconstruct": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.c_int]),
        "trals_residual_explicit": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int, _vp,
                                                   ctypes.POINTER(_dbl), ctypes.POINTER(_dbl)]),
        "trals_quantize_bf16": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _i64, _vp, _vp]),
        "trals_server_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_size_t, ctypes.c_int]),
        "trals_server_destroy": (None, [_vp]),
        "trals_server_submit": (ctypes.c_int, [_vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
        "trals_server_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(Result), _vp, _vp]),
        "trals_server_wait": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(Result), _vp,
                                             _vp]),
        "trals_server_stats": (ctypes.c_int, [_vp, ctypes.POINTER(ServerInfo)]),
        "trals_server_last_error": (ctypes.c_char_p, [_vp]),
        "trals_server_set_group_limit": (ctypes.c_int, [_vp, ctypes.c_int64]),
        "trals_testing_server_withhold_steps": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_longlong]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


# ------------------------------------------------------------------ marshalling helpers
def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _xtype(x) -> int:
    import torch
    if isinstance(x, np.ndarray):
        return {np.dtype(np.float64): X_F64, np.dtype(np.float32): X_F32}[x.dtype]
    return {torch.float64: X_F64, torch.float32: X_F32, torch.bfloat16: X_BF16}[x.dtype]


def _shape(I, R):
    N = len(I)
    Ia = (_i64 * N)(*[int(v) for v in I])
    Ra = (_i32 * N)(*[int(v) for v in R])
    return N, Ia, Ra


def _ptr_array(ptrs: Sequence[int]):
    return (_vp * len(ptrs))(*ptrs)


def _opts(mode=MODE_FP64, solver=SOLVE_CHOL, gram=GRAM_STRUCTURED, explicit_residual=False) -> Opts:
    if isinstance(mode, str):
        mode = MODE_NAMES[mode]
    return Opts(int(mode), int(solver), int(gram), int(bool(explicit_residual)))


def make_opts(mode=MODE_FP64, solver=SOLVE_CHOL, gram=GRAM_STRUCTURED, explicit_residual=False) -> Opts:
    return _opts(mode, solver, gram, explicit_residual)


class Context:
    """A libtrals context (device + stream)."""

    def __init__(self, device: int = 0, stream=None):
        h = _vp()
        s = _ptr_stream(stream)
        st = lib().trals_create(ctypes.byref(h), int(device), s)
        if st != OK:
            raise TralsError(st, f"trals_create(device={device}) failed (is a CUDA GPU present?)")
        self.handle = h
        self.device = device

    def check(self, st: int, what: str = ""):
        if st != OK:
            raise TralsError(st, f"{what}: {trals_last_error(self)}")

    def close(self):
        if getattr(self, "handle", None):
            lib().trals_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr_stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------ C ABI mirrors
def trals_version() -> str:
    return lib().trals_version().decode()


def trals_create(device: int = 0, stream=None) -> Context:
    return Context(device, stream)


def trals_destroy(ctx: Context) -> None:
    ctx.close()


def trals_last_error(ctx: Context) -> str:
    return lib().trals_last_error(ctx.handle).decode()


def cores_to_fortran(cores: Sequence[np.ndarray]) -> List[np.ndarray]:
    return [np.asfortranarray(np.asarray(G, dtype=np.float64)) for G in cores]


def trals_decompose(ctx: Context, I, R, X, cores: List[np.ndarray], sweeps: int, opts: Optional[Opts] = None,
                    ) -> np.ndarray:
    """Fit TR cores to X (numpy host array or torch CUDA tensor, column-major contents).

    ``cores`` (numpy, shapes (R_n, I_n, R_{n+1})) hold the initial cores and receive the result.
    Returns the relative residual after each sweep.
    """
    N, Ia, Ra = _shape(I, R)
    on_host = isinstance(X, np.ndarray) or not getattr(X, "is_cuda", True)
    if isinstance(X, np.ndarray):
        Xh = np.asarray(X).reshape(-1, order="F") if X.ndim > 1 else np.ascontiguousarray(X)
        xptr = Xh.ctypes.data
    else:
        xptr = X.data_ptr()  # a torch tensor (CUDA, or pinned host memory) holding column-major data
    fc = cores_to_fortran(cores)
    res = np.zeros(max(sweeps, 1))
    st = lib().trals_decompose(ctx.handle, N, ctypes.addressof(Ia), ctypes.addressof(Ra), xptr, _xtype(X),
                               int(on_host), _ptr_array([G.ctypes.data for G in fc]), int(sweeps),
                               ctypes.addressof(opts) if opts is not None else None, res.ctypes.data)
    ctx.check(st, "trals_decompose")
    for G, Gf in zip(cores, fc):
        G[...] = Gf
    return res[:sweeps]


class Plan:
    """A resident plan (trals_plan_*)."""

    def __init__(self, ctx: Context, I, R, X_dev, opts: Optional[Opts] = None):
        self.ctx = ctx
        self.I = tuple(int(v) for v in I)
        self.R = tuple(int(v) for v in R)
        self.N = len(self.I)
        self._X = X_dev  # keep the caller's tensor alive
        N, Ia, Ra = _shape(self.I, self.R)
        h = _vp()
        st = lib().trals_plan_create(ctx.handle, N, ctypes.addressof(Ia), ctypes.addressof(Ra), X_dev.data_ptr(),
                                     _xtype(X_dev), ctypes.addressof(opts) if opts is not None else None,
                                     ctypes.byref(h))
        ctx.check(st, "trals_plan_create")
        self.handle = h

    def set_cores(self, cores: Sequence[np.ndarray]) -> None:
        fc = cores_to_fortran(cores)
        self.ctx.check(lib().trals_plan_set_cores(self.handle, _ptr_array([G.ctypes.data for G in fc])),
                       "trals_plan_set_cores")

    def get_cores(self) -> List[np.ndarray]:
        out = [np.zeros((self.R[n], self.I[n], self.R[(n + 1) % self.N]), order="F") for n in range(self.N)]
        self.ctx.check(lib().trals_plan_get_cores(self.handle, _ptr_array([G.ctypes.data for G in out])),
                       "trals_plan_get_cores")
        return out

    def run(self, sweeps: int, use_graph: bool = True) -> None:
        self.ctx.check(lib().trals_plan_run(self.handle, int(sweeps), int(bool(use_graph))), "trals_plan_run")

    def residuals(self, cap: int = 1 << 14) -> np.ndarray:
        buf = np.zeros(cap)
        cnt = ctypes.c_int(0)
        self.ctx.check(lib().trals_plan_residuals(self.handle, buf.ctypes.data, cap, ctypes.byref(cnt)),
                       "trals_plan_residuals")
        return buf[:cnt.value].copy()

    def mttsp(self, n: int, M_dev=None) -> None:
        self.ctx.check(lib().trals_plan_mttsp(self.handle, int(n), _ptr(M_dev)), "trals_plan_mttsp")

    def explicit_residual(self) -> float:
        """|X - TR(cores)|_F / |X|_F of the current cores by one explicit pass over X."""
        v = ctypes.c_double()
        self.ctx.check(lib().trals_plan_explicit_residual(self.handle, ctypes.byref(v)),
                       "trals_plan_explicit_residual")
        return float(v.value)

    def nbytes(self) -> int:
        return int(lib().trals_plan_bytes(self.handle))

    def time_mttsp(self, n: int):
        """(main contraction kernel ms, whole MTTSP step ms) of one enqueue of mode n."""
        k, t = ctypes.c_float(), ctypes.c_float()
        self.ctx.check(lib().trals_plan_time_mttsp(self.handle, int(n), ctypes.byref(k), ctypes.byref(t)),
                       "trals_plan_time_mttsp")
        return float(k.value), float(t.value)

    def core_dev(self, n: int) -> int:
        return lib().trals_plan_core_dev(self.handle, int(n))

    def mttsp_path(self, n: int) -> int:
        return lib().trals_plan_mttsp_path(self.handle, int(n))

    def launches_per_sweep(self) -> int:
        return lib().trals_plan_launches_per_sweep(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            lib().trals_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def trals_plan_create(ctx: Context, I, R, X_dev, opts: Optional[Opts] = None) -> Plan:
    return Plan(ctx, I, R, X_dev, opts)


def trals_gamma(ctx: Context, G_dev, Rn: int, In: int, Rn1: int, Gamma_dev) -> None:
    ctx.check(lib().trals_gamma(ctx.handle, _ptr(G_dev), int(Rn), int(In), int(Rn1), _ptr(Gamma_dev)), "trals_gamma")


def trals_coef_matrix(ctx: Context, R, gammas_dev: Sequence, n: int, S_dev) -> None:
    N = len(R)
    Ra = (_i32 * N)(*[int(v) for v in R])
    ctx.check(lib().trals_coef_matrix(ctx.handle, N, ctypes.addressof(Ra), _ptr_array([_ptr(g) for g in gammas_dev]),
                                      int(n), _ptr(S_dev)), "trals_coef_matrix")


def trals_coef_matrix_explicit(ctx: Context, I, R, cores_dev: Sequence, n: int, S_dev, fp64: bool = True) -> None:
    N, Ia, Ra = _shape(I, R)
    ctx.check(lib().trals_coef_matrix_explicit(ctx.handle, N, ctypes.addressof(Ia), ctypes.addressof(Ra),
                                               _ptr_array([_ptr(c) for c in cores_dev]), int(n), int(bool(fp64)),
                                               _ptr(S_dev)), "trals_coef_matrix_explicit")


def trals_qr_r_factor(ctx: Context, I, R, cores_dev: Sequence, n: int, R_dev) -> None:
    N, Ia, Ra = _shape(I, R)
    ctx.check(lib().trals_qr_r_factor(ctx.handle, N, ctypes.addressof(Ia), ctypes.addressof(Ra),
                                      _ptr_array([_ptr(c) for c in cores_dev]), int(n), _ptr(R_dev)),
              "trals_qr_r_factor")


def trals_mttsp(ctx: Context, I, R, X_dev, mode, cores_dev: Sequence, n: int, M_dev, xt: Optional[int] = None) -> None:
    """M_n of X_dev; xt overrides the element type taken from the tensor (X_BF16PAIR for a hi/lo pair)."""
    N, Ia, Ra = _shape(I, R)
    if isinstance(mode, str):
        mode = MODE_NAMES[mode]
    ctx.check(lib().trals_mttsp(ctx.handle, N, ctypes.addressof(Ia), ctypes.addressof(Ra), _ptr(X_dev),
                                _xtype(X_dev) if xt is None else int(xt), int(mode),
                                _ptr_array([_ptr(c) for c in cores_dev]), int(n), _ptr(M_dev)),
              "trals_mttsp")


def trals_mttsp_noalloc(ctx: Context, I, R, X_dev, cores_dev: Sequence, n: int, M_dev) -> None:
    """FP64 MTTSP of mode n with no device allocation (static scratch; see include/trals.h)."""
    N, Ia, Ra = _shape(I, R)
    ctx.check(lib().trals_mttsp_noalloc(ctx.handle, N, ctypes.addressof(Ia), ctypes.addressof(Ra), _ptr(X_dev),
                                        _ptr_array([_ptr(c) for c in cores_dev]), int(n), _ptr(M_dev)),
              "trals_mttsp_noalloc")


MTTSP_PATHS = {0: "cuda-cores", 1: "tc-kmajor-left", 2: "tc-kmajor-right", 3: "tc-mnmajor", 4: "tc-mnmajor-left",
               5: "two-stage-gemm"}


def trals_last_mttsp_path(ctx: Context) -> int:
    """Kernel the last successful trals_mttsp on ctx ran (MTTSP_PATHS codes; -1 if none)."""
    return lib().trals_last_mttsp_path(ctx.handle)


def trals_testing_mttsp_withheld_copy(ctx: Context, I, R, X_dev, mode, cores_dev: Sequence, n: int, M_dev,
                                      spin_cycles: int) -> None:
    """Fault injection (include/trals_testing.h): the tensor-core MTTSP with its first copy withheld and
    every wait bounded by spin_cycles; raises TralsError(E_TIMEOUT) as the kernel reports."""
    N, Ia, Ra = _shape(I, R)
    if isinstance(mode, str):
        mode = MODE_NAMES[mode]
    ctx.check(lib().trals_testing_mttsp_withheld_copy(ctx.handle, N, ctypes.addressof(Ia), ctypes.addressof(Ra),
                                                      _ptr(X_dev), int(mode),
                                                      _ptr_array([_ptr(c) for c in cores_dev]), int(n),
                                                      _ptr(M_dev), int(spin_cycles)),
              "trals_testing_mttsp_withheld_copy")


def trals_mttsp_path(I, R, n: int, mode) -> int:
    """Kernel the MTTSP of mode n uses in `mode` (0 = CUDA cores, 1-3 = tensor-core variants)."""
    N, Ia, Ra = _shape(I, R)
    if isinstance(mode, str):
        mode = MODE_NAMES[mode]
    return lib().trals_mttsp_path(N, ctypes.addressof(Ia), ctypes.addressof(Ra), int(n), int(mode))


def trals_solve_chol(ctx: Context, Rn: int, In: int, Rn1: int, S_dev, M_dev, G_dev) -> None:
    ctx.check(lib().trals_solve_chol(ctx.handle, int(Rn), int(In), int(Rn1), _ptr(S_dev), _ptr(M_dev), _ptr(G_dev)),
              "trals_solve_chol")


def trals_check_pivot_rsqrt(ctx: Context, d_dev, out_dev, ref_dev) -> None:
    """Verification hook: out = the Cholesky pivots' reciprocal square root of d, ref = CUDA's rsqrt(d)."""
    ctx.check(lib().trals_check_pivot_rsqrt(ctx.handle, _ptr(d_dev), int(d_dev.numel()), _ptr(out_dev), _ptr(ref_dev)),
              "trals_check_pivot_rsqrt")


def trals_reconstruct(ctx: Context, I, R, cores_dev: Sequence, out_dev) -> None:
    N, Ia, Ra = _shape(I, R)
    ctx.check(lib().trals_reconstruct(ctx.handle, N, ctypes.addressof(Ia), ctypes.addressof(Ra),
                                      _ptr_array([_ptr(c) for c in cores_dev]), _ptr(out_dev), _xtype(out_dev)),
              "trals_reconstruct")


def trals_residual_explicit(ctx: Context, I, R, X_dev, cores_dev: Sequence):
    N, Ia, Ra = _shape(I, R)
    r2, x2 = _dbl(0), _dbl(0)
    ctx.check(lib().trals_residual_explicit(ctx.handle, N, ctypes.addressof(Ia), ctypes.addressof(Ra), _ptr(X_dev),
                                            _xtype(X_dev), _ptr_array([_ptr(c) for c in cores_dev]),
                                            ctypes.byref(r2), ctypes.byref(x2)), "trals_residual_explicit")
    return r2.value, x2.value


def trals_quantize_bf16(ctx: Context, src_dev, hi_dev, lo_dev=None) -> None:
    ctx.check(lib().trals_quantize_bf16(ctx.handle, _ptr(src_dev), _xtype(src_dev), int(src_dev.numel()),
                                        _ptr(hi_dev), _ptr(lo_dev)), "trals_quantize_bf16")


# ------------------------------------------------------------------ torch helpers (plumbing)
def core_to_device(G: np.ndarray, device="cuda"):
    """A core (R_n, I_n, R_{n+1}) as a flat column-major float64 CUDA tensor."""
    import torch
    return torch.from_numpy(np.asarray(G, dtype=np.float64).reshape(-1, order="F").copy()).to(device)


def core_from_device(t, Rn: int, In: int, Rn1: int) -> np.ndarray:
    return t.detach().cpu().numpy().reshape((Rn, In, Rn1), order="F")


def tensor_to_device(X: np.ndarray, dtype=None, device="cuda"):
    """A dense tensor as a flat column-major CUDA tensor (float64 unless dtype is given)."""
    import torch
    flat = torch.from_numpy(np.asarray(X, dtype=np.float64).reshape(-1, order="F").copy())
    if dtype is not None:
        flat = flat.to(dtype)
    return flat.to(device)


def trals_plan_destroy(plan: Plan) -> None:
    plan.close()


def trals_plan_set_cores(plan: Plan, cores: Sequence[np.ndarray]) -> None:
    plan.set_cores(cores)


def trals_plan_get_cores(plan: Plan) -> List[np.ndarray]:
    return plan.get_cores()


def trals_plan_run(plan: Plan, sweeps: int, use_graph: bool = True) -> None:
    plan.run(sweeps, use_graph)


def trals_plan_residuals(plan: Plan) -> np.ndarray:
    return plan.residuals()


def trals_plan_mttsp(plan: Plan, n: int, M_dev=None) -> None:
    plan.mttsp(n, M_dev)


def trals_plan_explicit_residual(plan: Plan) -> float:
    return plan.explicit_residual()


def trals_plan_bytes(plan: Plan) -> int:
    return plan.nbytes()


def trals_plan_footprint(ctx: Context, I, R, X_dev, opts: Optional[Opts] = None) -> int:
    """Device workspace bytes a plan for these arguments would allocate (host-side count)."""
    N, Ia, Ra = _shape(I, R)
    b = ctypes.c_size_t()
    ctx.check(lib().trals_plan_footprint(ctx.handle, N, ctypes.addressof(Ia), ctypes.addressof(Ra), _ptr(X_dev),
                                         _xtype(X_dev), ctypes.addressof(opts) if opts is not None else None,
                                         ctypes.byref(b)), "trals_plan_footprint")
    return int(b.value)


def trals_plan_time_mttsp(plan: Plan, n: int):
    return plan.time_mttsp(n)


def trals_plan_core_dev(plan: Plan, n: int) -> int:
    return plan.core_dev(n)


def trals_plan_mttsp_path(plan: Plan, n: int) -> int:
    return plan.mttsp_path(n)


def trals_plan_launches_per_sweep(plan: Plan) -> int:
    return plan.launches_per_sweep()


# ------------------------------------------------------------------ serving
class Server:
    """The serving loop (trals_server_*): continuous batching of decompositions on one GPU."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 64 << 30, max_slots: int = 8):
        h = _vp()
        st = lib().trals_server_create(ctypes.byref(h), int(device), int(hbm_budget_bytes), int(max_slots))
        if st != OK:
            raise TralsError(st, "trals_server_create failed")
        self.handle = h
        self._pending = {}   # ticket -> (X, shapes): X must stay alive until the request is done

    def _err(self, st, what):
        raise TralsError(st, f"{what}: {lib().trals_server_last_error(self.handle).decode()}")

    def submit(self, I, R, X, init_cores: Sequence[np.ndarray], sweeps: int, opts: Optional[Opts] = None) -> int:
        N, Ia, Ra = _shape(I, R)
        on_host = isinstance(X, np.ndarray) or not getattr(X, "is_cuda", True)
        if isinstance(X, np.ndarray) and X.ndim > 1:
            X = np.asarray(X).reshape(-1, order="F").copy()   # column-major contents, kept alive below
        fc = cores_to_fortran(init_cores)
        ptrs = _ptr_array([G.ctypes.data for G in fc])
        q = Request(N, ctypes.addressof(Ia), ctypes.addressof(Ra), _ptr(X), _xtype(X), int(on_host),
                    ctypes.addressof(ptrs), int(sweeps), opts if opts is not None else _opts())
        t = ctypes.c_uint64()
        st = lib().trals_server_submit(self.handle, ctypes.byref(q), ctypes.byref(t))
        if st != OK:
            self._err(st, "trals_server_submit")
        self._pending[t.value] = (X, tuple(int(v) for v in I), tuple(int(v) for v in R), int(sweeps))
        return t.value

    def _take(self, ticket, fn, *extra):
        if ticket not in self._pending:
            raise TralsError(E_ARG, f"unknown or already taken ticket {ticket}")
        X, I, R, sweeps = self._pending[ticket]
        N = len(I)
        out = [np.zeros(R[n] * I[n] * R[(n + 1) % N]) for n in range(N)]
        res = np.zeros(max(sweeps, 1))
        r = Result()
        st = fn(self.handle, ctypes.c_uint64(ticket), *extra, ctypes.byref(r), _ptr_array([o.ctypes.data for o in out]),
                res.ctypes.data)
        if st == E_PENDING:
            return None
        if st != OK:
            self._err(st, "trals_server_poll")
        del self._pending[ticket]
        cores = [o.reshape((R[n], I[n], R[(n + 1) % N]), order="F") for n, o in enumerate(out)]
        info = {"status": r.status, "sweeps": r.sweeps, "submit_s": r.submit_s, "admit_s": r.admit_s,
                "done_s": r.done_s, "footprint_bytes": r.footprint_bytes}
        if r.status != OK:
            info["error"] = lib().trals_server_last_error(self.handle).decode()
        return info, cores, res[:sweeps]

    def poll(self, ticket: int):
        """None while pending, else (info dict, fitted cores, per-sweep residuals)."""
        return self._take(ticket, lib().trals_server_poll)

    def wait(self, ticket: int, timeout: float = -1.0):
        return self._take(ticket, lib().trals_server_wait, ctypes.c_double(timeout))

    def set_group_limit(self, max_elems: int) -> None:
        """Requests submitted from now on with at most max_elems entries (and otherwise small) join the
        grouped step engine; 0 sends every request to a plan."""
        st = lib().trals_server_set_group_limit(self.handle, int(max_elems))
        if st != OK:
            self._err(st, "trals_server_set_group_limit")

    def testing_withhold_steps(self, steps: int, spin_cycles: int) -> None:
        """Fault injection (include/trals_testing.h): the next `steps` grouped steps run without their
        descriptor table, so their bounded wait gives up and their requests report TRALS_E_TIMEOUT."""
        st = lib().trals_testing_server_withhold_steps(self.handle, int(steps), int(spin_cycles))
        if st != OK:
            self._err(st, "trals_testing_server_withhold_steps")

    def stats(self) -> dict:
        s = ServerInfo()
        st = lib().trals_server_stats(self.handle, ctypes.byref(s))
        if st != OK:
            self._err(st, "trals_server_stats")
        return {f: getattr(s, f) for f, _ in ServerInfo._fields_}

    def close(self):
        if getattr(self, "handle", None):
            lib().trals_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def trals_server_create(device: int = 0, hbm_budget_bytes: int = 64 << 30, max_slots: int = 8) -> Server:
    return Server(device, hbm_budget_bytes, max_slots)


def trals_server_destroy(server: Server) -> None:
    server.close()


def trals_server_submit(server: Server, I, R, X, init_cores, sweeps: int, opts: Optional[Opts] = None) -> int:
    return server.submit(I, R, X, init_cores, sweeps, opts)


def trals_server_poll(server: Server, ticket: int):
    return server.poll(ticket)


def trals_server_wait(server: Server, ticket: int, timeout: float = -1.0):
    return server.wait(ticket, timeout)


def trals_server_stats(server: Server) -> dict:
    return server.stats()


def trals_server_last_error(server: Server) -> str:
    return lib().trals_server_last_error(server.handle).decode()


def trals_server_set_group_limit(server: Server, max_elems: int) -> None:
    server.set_group_limit(max_elems)


def trals_testing_server_withhold_steps(server: Server, steps: int, spin_cycles: int) -> None:
    server.testing_withhold_steps(steps, spin_cycles)
