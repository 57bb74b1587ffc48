"""ctypes binding of the HIF-IE C ABI (``include/hif.h``).

Argument marshalling only: every array is handed to the library as a raw
pointer (torch CUDA tensors as device pointers, numpy arrays or CPU tensors
as host pointers; the library tells them apart), and every step of the
computation runs inside the library's CUDA kernels.  If the shared library is
missing the import fails loudly -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libhif.so")

HIF_OK, HIF_EINVAL, HIF_ENOMEM, HIF_ESINGULAR, HIF_ENUMERIC, HIF_ECUDA, HIF_ETIMEOUT, HIF_ENOTCONV = range(8)


class hif_options(C.Structure):
    _fields_ = [
        ("dim", C.c_int),
        ("leaf_occupancy", C.c_int),
        ("second_kind", C.c_int),
        ("precision", C.c_int),
        ("fractional_levels", C.c_int),
        ("skip_levels", C.c_int),
        ("proxy_points", C.c_int),
        ("proxy_radius", C.c_double),
        ("proxy_dirs", C.c_void_p),
        ("fp32_tol_floor", C.c_double),
        ("root_lo", C.c_double * 3),
        ("root_width", C.c_double),
        ("stream", C.c_void_p),
        ("direct_precision", C.c_int),
        ("use_graphs", C.c_int),
        ("autotune", C.c_int),
        ("symmetric", C.c_int),
        ("wavenumber", C.c_double),
        ("ldl", C.c_int),
    ]


class hif_profile_entry(C.Structure):
    _fields_ = [
        ("name", C.c_char_p),
        ("ranges", C.c_int64),
        ("ms", C.c_double),
        ("flops", C.c_double),
        ("bytes", C.c_double),
    ]


class hif_problem(C.Structure):
    _fields_ = [
        ("points", C.c_void_p),
        ("N", C.c_int64),
        ("weights", C.c_void_p),
        ("a", C.c_void_p),
        ("b", C.c_void_p),
        ("c", C.c_void_p),
    ]


class hif_stats_t(C.Structure):
    _fields_ = [
        ("N", C.c_int64),
        ("dim", C.c_int),
        ("levels", C.c_int),
        ("sublevels", C.c_int),
        ("top_size", C.c_int64),
        ("factor_bytes", C.c_int64),
        ("skeletons", C.c_int64 * 64),
        ("redundant", C.c_int64 * 64),
        ("boxes", C.c_int64 * 64),
        ("kinds", C.c_int * 64),
        ("max_box", C.c_int * 64),
        ("factor_seconds", C.c_double),
        ("flops", C.c_double),
        ("kernel_evals", C.c_double),
        ("proxy_rows", C.c_int64),
        ("symmetric_problems", C.c_int),
        ("ldl_boxes", C.c_int64),
        ("ldl_fallbacks", C.c_int64),
    ]


class hif_gemm_problem(C.Structure):
    _fields_ = [
        ("A", C.c_void_p),
        ("B", C.c_void_p),
        ("C", C.c_void_p),
        ("lda", C.c_int64),
        ("ldb", C.c_int64),
        ("ldc", C.c_int64),
        ("m", C.c_int32),
        ("n", C.c_int32),
        ("k", C.c_int32),
        ("trans_a", C.c_int32),
        ("trans_b", C.c_int32),
        ("alpha", C.c_float),
        ("beta", C.c_int32),
    ]


EXPORTS = {
    "hif_options_default": (C.c_int, [C.c_int, C.POINTER(hif_options)]),
    "hif_factor": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                             C.c_int, C.c_double, C.POINTER(hif_options), C.POINTER(C.c_void_p)]),
    "hif_factor_batched": (C.c_int, [C.c_int, C.c_void_p, C.c_int, C.c_double, C.POINTER(hif_options),
                                     C.POINTER(C.c_void_p)]),
    "hif_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64]),
    "hif_apply_transpose": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64]),
    "hif_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64]),
    "hif_solve_transpose": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64]),
    "hif_matvec": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64]),
    "hif_matvec_digits": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64]),
    "hif_solve_refined": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64,
                                    C.c_double, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "hif_adjoint_gradients": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p,
                                        C.c_void_p, C.c_void_p]),
    "hif_eliminated_dofs": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "hif_error_estimates": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_double),
                                      C.POINTER(C.c_int)]),
    "hif_stats": (C.c_int, [C.c_void_p, C.POINTER(hif_stats_t)]),
    "hif_destroy": (C.c_int, [C.c_void_p]),
    "hif_status_string": (C.c_char_p, [C.c_int]),
    "hif_last_error": (C.c_char_p, []),
    "hif_kernel_launches": (C.c_uint64, []),
    "hif_kernel_timing": (C.c_int, [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "hif_kernel_profile": (C.c_int, [C.c_int, C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "hif_kernel_block": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                   C.c_void_p]),
    "hif_id_batched": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hif_gemm_batched_f32": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p]),
    "hif_id_batched_noalloc": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libhif.so (raises OSError with a clear message if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"HIF-IE CUDA library not built: {path} is missing "
                      "(run paper_1307_2666_gb300.build.build())")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class HIFError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.hif_status_string(status).decode()
        detail = lib.hif_last_error().decode()
        super().__init__(f"{where}: {msg}" + (f" ({detail})" if detail else ""))
        self.status = status


def _check(status: int, where: str, allow=()):
    if status != HIF_OK and status not in allow:
        raise HIFError(status, where)
    return status


def _ptr(a):
    """Raw data pointer of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        return C.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported array type {type(a)}")


def _ld(a):
    """Leading dimension of an N x nrhs column-major array (torch or numpy)."""
    if a.ndim == 1:
        return a.shape[0], 1
    if hasattr(a, "stride") and callable(a.stride):
        s0, s1 = a.stride()
        if a.shape[1] == 1:                     # one column: its stride is meaningless
            if s0 != 1 and a.shape[0] > 1:
                raise ValueError("vectors must be column-major (stride 1 along rows)")
            return a.shape[0], 1
        if s0 != 1:
            raise ValueError("vectors must be column-major (stride 1 along rows)")
        return s1, a.shape[1]
    if not a.flags["F_CONTIGUOUS"]:
        raise ValueError("vectors must be Fortran-ordered (column-major)")
    return a.shape[0], a.shape[1]


def hif_options_default(dim: int) -> hif_options:
    o = hif_options()
    _check(load().hif_options_default(dim, C.byref(o)), "hif_options_default")
    return o


def hif_factor(points, weights, a, b, c, kernel_id: int, eps: float, opt: hif_options | None = None):
    lib = load()
    N = points.shape[0]
    h = C.c_void_p()
    st = lib.hif_factor(_ptr(points), N, _ptr(weights), _ptr(a), _ptr(b), _ptr(c), int(kernel_id), float(eps),
                        C.byref(opt) if opt is not None else None, C.byref(h))
    _check(st, "hif_factor")
    return h


def hif_factor_batched(problems, kernel_id: int, eps: float, opt: hif_options | None = None):
    """problems: sequence of (points, weights, a, b, c) array tuples."""
    lib = load()
    arr = (hif_problem * len(problems))()
    for q, (pts, w, a, b, c) in enumerate(problems):
        arr[q] = hif_problem(_ptr(pts).value, pts.shape[0], _ptr(w).value, _ptr(a).value, _ptr(b).value,
                             _ptr(c).value)
    h = C.c_void_p()
    st = lib.hif_factor_batched(len(problems), C.cast(arr, C.c_void_p), int(kernel_id), float(eps),
                                C.byref(opt) if opt is not None else None, C.byref(h))
    _check(st, "hif_factor_batched")
    return h


def _vec_call(name, h, x, y):
    ld, nrhs = _ld(x)
    ldy, nrhs_y = _ld(y)
    if ldy != ld or nrhs_y != nrhs:
        raise ValueError("input and output must have the same shape and leading dimension")
    _check(getattr(load(), name)(h, _ptr(x), _ptr(y), nrhs, ld), name)
    return y


def hif_apply(h, x, y):
    return _vec_call("hif_apply", h, x, y)


def hif_apply_transpose(h, x, y):
    return _vec_call("hif_apply_transpose", h, x, y)


def hif_solve(h, b, x):
    return _vec_call("hif_solve", h, b, x)


def hif_solve_transpose(h, b, x):
    return _vec_call("hif_solve_transpose", h, b, x)


def hif_matvec(h, trans: int, x, y):
    ld, nrhs = _ld(x)
    _check(load().hif_matvec(h, int(trans), _ptr(x), _ptr(y), nrhs, ld), "hif_matvec")
    return y


def hif_matvec_digits(h, trans: int, classes: int, x, y):
    ld, nrhs = _ld(x)
    _check(load().hif_matvec_digits(h, int(trans), int(classes), _ptr(x), _ptr(y), nrhs, ld), "hif_matvec_digits")
    return y


def hif_solve_refined(h, trans: int, f, u, tol: float = 1e-10, maxit: int = 50, method: int = 0):
    ld, nrhs = _ld(f)
    it = C.c_int(0)
    rr = C.c_double(0.0)
    st = load().hif_solve_refined(h, int(trans), _ptr(f), _ptr(u), nrhs, ld, float(tol), int(maxit), int(method),
                                  C.byref(it), C.byref(rr))
    _check(st, "hif_solve_refined", allow=(HIF_ENOTCONV,))
    return st, it.value, rr.value


def hif_adjoint_gradients(h, u, lam, ga, gb, gc):
    """Coefficient gradients of the adjoint method into ga, gb, gc (N each)."""
    ld, nrhs = _ld(u)
    ld2, nrhs2 = _ld(lam)
    if (ld, nrhs) != (ld2, nrhs2):
        raise ValueError("u and lam must have the same shape and leading dimension")
    _check(load().hif_adjoint_gradients(h, _ptr(u), _ptr(lam), nrhs, ld, _ptr(ga), _ptr(gb), _ptr(gc)),
           "hif_adjoint_gradients")


def hif_eliminated_dofs(h, sublevel: int) -> np.ndarray:
    """The DOFs eliminated at one sublevel (the last index: the top block)."""
    lib = load()
    n = C.c_int64(0)
    _check(lib.hif_eliminated_dofs(h, int(sublevel), None, 0, C.byref(n)), "hif_eliminated_dofs")
    out = np.empty(n.value, dtype=np.int32)
    _check(lib.hif_eliminated_dofs(h, int(sublevel), _ptr(out), n.value, C.byref(n)), "hif_eliminated_dofs")
    return out


def hif_error_estimates(h, v0, rtol: float = 1e-2, maxit: int = 200):
    """((|A|, |A - F|, |I - A F^{-1}|), (steps,) * 3, converged) by power
    iteration from v0 (Sec. 5); e_a = norms[1] / norms[0], e_s = norms[2]."""
    norms = (C.c_double * 3)()
    its = (C.c_int * 3)()
    st = load().hif_error_estimates(h, _ptr(v0), float(rtol), int(maxit), norms, its)
    _check(st, "hif_error_estimates", allow=(HIF_ENOTCONV,))
    return tuple(norms), tuple(its), st == HIF_OK


def hif_stats(h) -> dict:
    s = hif_stats_t()
    _check(load().hif_stats(h, C.byref(s)), "hif_stats")
    n = s.sublevels
    kind = {0: "cell", 1: "face", 2: "edge"}
    return {
        "N": s.N, "dim": s.dim, "levels": s.levels, "sublevels": n, "top_size": s.top_size,
        "factor_bytes": s.factor_bytes, "factor_seconds": s.factor_seconds, "flops": s.flops,
        "kernel_evals": s.kernel_evals, "proxy_rows": s.proxy_rows, "symmetric_problems": s.symmetric_problems,
        "ldl_boxes": s.ldl_boxes, "ldl_fallbacks": s.ldl_fallbacks,
        "per_sublevel": [dict(kind=kind[s.kinds[i]], boxes=s.boxes[i], skeletons=s.skeletons[i],
                              redundant=s.redundant[i], max_box=s.max_box[i]) for i in range(n)],
    }


def hif_kernel_launches() -> int:
    return int(load().hif_kernel_launches())


def hif_kernel_profile(enable: bool) -> dict:
    """Per kernel family since the previous call: {name: {ranges, ms, flops,
    bytes}}; then turns per-family event recording on or off."""
    arr = (hif_profile_entry * 32)()
    cnt = C.c_int(0)
    _check(load().hif_kernel_profile(1 if enable else 0, C.cast(arr, C.c_void_p), 32, C.byref(cnt)),
           "hif_kernel_profile")
    return {arr[k].name.decode(): dict(ranges=int(arr[k].ranges), ms=float(arr[k].ms), flops=float(arr[k].flops),
                                       bytes=float(arr[k].bytes)) for k in range(min(cnt.value, 32))}


def hif_kernel_timing(enable: bool) -> tuple[float, int]:
    """(device ms, launches) of the tensor-core direct sum since the previous
    call; then turns event recording on or off."""
    ms = C.c_double(0.0)
    n = C.c_int64(0)
    _check(load().hif_kernel_timing(1 if enable else 0, C.byref(ms), C.byref(n)), "hif_kernel_timing")
    return ms.value, n.value


def hif_destroy(h):
    if h:
        _check(load().hif_destroy(h), "hif_destroy")


def hif_kernel_block(points, weights, a, b, c, kernel_id: int, rows, cols, out, stream=None):
    N, dim = points.shape
    ldo = out.stride()[1] if hasattr(out, "stride") and callable(out.stride) else out.shape[0]
    _check(load().hif_kernel_block(_ptr(points), N, dim, _ptr(weights), _ptr(a), _ptr(b), _ptr(c), int(kernel_id),
                                   _ptr(rows), len(rows), _ptr(cols), len(cols), _ptr(out), ldo, stream),
           "hif_kernel_block")
    return out


def hif_id_batched(mats, off, m, n, tol, k, perm, poff, T, toff, stream=None):
    _check(load().hif_id_batched(len(m), _ptr(mats), _ptr(off), _ptr(m), _ptr(n), _ptr(tol), _ptr(k), _ptr(perm),
                                 _ptr(poff), _ptr(T), _ptr(toff), stream), "hif_id_batched")


def hif_id_batched_noalloc(mats, off, m, n, tol, k, perm, poff, T, toff, stream=None):
    """Batched ID whose work space is a fixed device array: no allocation.
    All arrays must be device tensors.  Returns the status code (HIF_OK, or
    HIF_EINVAL when the input exceeds the fixed work space)."""
    return _check(load().hif_id_batched_noalloc(len(m), _ptr(mats), _ptr(off), _ptr(m), _ptr(n), _ptr(tol), _ptr(k),
                                                _ptr(perm), _ptr(poff), _ptr(T), _ptr(toff), stream),
                  "hif_id_batched_noalloc", allow=(HIF_EINVAL,))


def hif_gemm_batched_f32(problems, stream=None):
    """C = beta C + alpha op(A) op(B) for each problem, FP32 on the tensor
    cores.  problems: a sequence of dicts with keys A, B, C (device tensors
    or raw pointers), lda, ldb, ldc, m, n, k, trans_a, trans_b, alpha, beta."""
    arr = (hif_gemm_problem * max(1, len(problems)))()
    for i, q in enumerate(problems):
        raw = lambda x: None if x is None else (x if isinstance(x, int) else _ptr(x).value)
        arr[i] = hif_gemm_problem(raw(q["A"]), raw(q["B"]), raw(q["C"]), int(q["lda"]), int(q["ldb"]),
                                  int(q["ldc"]), int(q["m"]), int(q["n"]), int(q["k"]), int(q.get("trans_a", 0)),
                                  int(q.get("trans_b", 0)), float(q.get("alpha", 1.0)), int(q.get("beta", 0)))
    return _check(load().hif_gemm_batched_f32(len(problems), C.cast(arr, C.c_void_p), stream),
                  "hif_gemm_batched_f32", allow=(HIF_EINVAL,))
