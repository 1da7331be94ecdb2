"""ctypes binding of the C ABI in include/plam.h (argument marshalling only).

Every function here forwards to the identically named C entry point of
lib/libplam.so; all computation happens in the CUDA kernels behind it.  The
library is loaded on first use and a missing or unloadable library raises
immediately: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libplam.so")

PLAM_OK = 0
PLAM_ERR_INVALID = 1
PLAM_ERR_NOT_CONVERGED = 2
PLAM_ERR_DIVERGED = 3
PLAM_ERR_CHOLESKY = 4
PLAM_ERR_TIMEOUT = 5
PLAM_ERR_CUDA = 6
PLAM_ERR_NOMEM = 7
PLAM_ERR_UNSUPPORTED = 8
STATUS_NAMES = {0: "PLAM_OK", 1: "PLAM_ERR_INVALID", 2: "PLAM_ERR_NOT_CONVERGED",
                3: "PLAM_ERR_DIVERGED", 4: "PLAM_ERR_CHOLESKY", 5: "PLAM_ERR_TIMEOUT",
                6: "PLAM_ERR_CUDA", 7: "PLAM_ERR_NOMEM", 8: "PLAM_ERR_UNSUPPORTED"}

PLAM_VARIANT_PLAM, PLAM_VARIANT_PCAL, PLAM_VARIANT_MOPTQR = 0, 1, 2
PLAM_TC_SINGLE_CTA = 8
PLAM_LAMBDA1, PLAM_LAMBDA2, PLAM_LAMBDA_DA = 0, 1, 2
PLAM_ETA_ABB, PLAM_ETA_BB1, PLAM_ETA_BB2, PLAM_ETA_CONST, PLAM_ETA_DIFF = 0, 1, 2, 3, 4
PLAM_PREC_FP64, PLAM_PREC_FP32 = 0, 1
PLAM_OBJ_DENSE, PLAM_OBJ_HARTREE1D, PLAM_OBJ_STENCIL3D, PLAM_OBJ_CALLBACK, PLAM_OBJ_QAP = 0, 1, 2, 3, 4
PLAM_ENGINE_AUTO, PLAM_ENGINE_GRAPH, PLAM_ENGINE_RESIDENT = 0, 1, 2


class plam_params_t(C.Structure):
    _fields_ = [("variant", C.c_int), ("lambda_rule", C.c_int), ("beta", C.c_double),
                ("eta_rule", C.c_int), ("eta0", C.c_double), ("eta_gamma", C.c_double),
                ("tol", C.c_double), ("maxit", C.c_int), ("precision", C.c_int),
                ("final_orth", C.c_int), ("graph_iters", C.c_int), ("engine", C.c_int),
                ("tensor_cores", C.c_int), ("refine_switch", C.c_double), ("feas_max", C.c_double),
                ("orth_metrics", C.c_int), ("eta_min", C.c_double), ("eta_max", C.c_double)]


# int grad(void* ctx, const void* X, int64_t ldx, void* G, int64_t ldg, double* f, void* stream)
plam_grad_fn = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                           C.c_void_p, C.c_void_p)


class plam_objective_t(C.Structure):
    _fields_ = [("kind", C.c_int), ("A", C.c_void_p), ("lda", C.c_int64), ("alpha", C.c_double),
                ("quad_scale", C.c_double), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("V", C.c_void_p), ("grad", plam_grad_fn), ("grad_ctx", C.c_void_p),
                ("xc", C.c_double), ("block", C.c_int64), ("lin", C.c_void_p),
                ("ldlin", C.c_int64), ("Bq", C.c_void_p), ("ldbq", C.c_int64)]


# int allgather(void* ctx, const double* send, double* recv, int64_t count, void* stream)
plam_allgather_fn = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p)
# int exchange(void* ctx, const void* send_lo, const void* send_hi, void* recv_lo, void* recv_hi,
#              int64_t count, void* stream)
plam_exchange_fn = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_int64, C.c_void_p)


class plam_comm_t(C.Structure):
    _fields_ = [("rank", C.c_int), ("size", C.c_int), ("row0", C.c_int64), ("n_global", C.c_int64),
                ("allgather", plam_allgather_fn), ("exchange", plam_exchange_fn),
                ("ctx", C.c_void_p)]


class plam_batch_problem_t(C.Structure):
    _fields_ = [("n", C.c_int64), ("p", C.c_int64), ("A", C.c_void_p), ("lda", C.c_int64),
                ("X", C.c_void_p), ("ldx", C.c_int64), ("Q", C.c_void_p), ("ldq", C.c_int64)]


class plam_info_t(C.Structure):
    _fields_ = [("iters", C.c_int), ("status", C.c_int), ("converged", C.c_int), ("pad_", C.c_int),
                ("f", C.c_double), ("kkt_rel", C.c_double), ("feas", C.c_double),
                ("eta", C.c_double), ("K0", C.c_double), ("eta0", C.c_double),
                ("f_orth", C.c_double), ("kkt_orth", C.c_double), ("feas_orth", C.c_double),
                ("ms_iterations", C.c_double), ("ms_orth", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


SIGNATURES = {
    "plam_default_params": (C.c_int, [C.POINTER(plam_params_t)]),
    "plam_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int64, C.c_int64,
                              C.POINTER(plam_objective_t), C.POINTER(plam_params_t), C.c_void_p]),
    "plam_create_sharded": (C.c_int, [C.POINTER(C.c_void_p), C.c_int64, C.c_int64,
                                      C.POINTER(plam_objective_t), C.POINTER(plam_params_t),
                                      C.POINTER(plam_comm_t), C.c_void_p]),
    "plam_destroy": (C.c_int, [C.c_void_p]),
    "plam_reset": (C.c_int, [C.c_void_p]),
    "plam_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(plam_info_t)]),
    "pcal_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(plam_info_t)]),
    "plam_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                             C.POINTER(plam_info_t)]),
    "plam_orthonormalize": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                      C.c_int, C.POINTER(C.c_double)]),
    "plam_energy_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                   C.POINTER(C.c_double)]),
    "plam_energy": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "plam_energy_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                       C.c_int64]),
    "plam_grams": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                             C.c_void_p, C.c_void_p]),
    "plam_grams_noalloc": (C.c_int, [C.c_int64, C.c_int64, C.c_int, C.c_void_p, C.c_int64,
                                     C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "plam_time_kernels": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int,
                                    C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    "plam_history": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_int)]),
    "plam_last_iteration": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                      C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "plam_kernel_launches": (C.c_int64, [C.c_void_p]),
    "plam_state_bytes": (C.c_size_t, [C.c_void_p]),
    "plam_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "plam_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "plam_solve_engine": (C.c_int, [C.c_void_p]),
    "plam_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(plam_batch_problem_t), C.c_int,
                                    C.POINTER(plam_params_t), C.c_void_p]),
    "plam_batch_solve": (C.c_int, [C.c_void_p, C.POINTER(plam_info_t)]),
    "plam_batch_autotune": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int),
                                      C.POINTER(C.c_double)]),
    "plam_batch_set_tile": (C.c_int, [C.c_void_p, C.c_int]),
    "plam_batch_destroy": (C.c_int, [C.c_void_p]),
    "plam_last_error": (C.c_char_p, []),
    "plam_version": (C.c_int, []),
}

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libplam.so (once) and declare every signature.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
    try:
        import torch  # noqa: F401  (share torch's CUDA runtime when it is present)
    except Exception:
        pass
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class PlamError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load().plam_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} {msg}".strip())
        self.status = status


def check(status: int, where: str, ok=(PLAM_OK,)) -> int:
    if status not in ok:
        raise PlamError(status, where)
    return status


# ---------------------------------------------------------------- same-name wrappers

def plam_default_params() -> plam_params_t:
    prm = plam_params_t()
    check(load().plam_default_params(C.byref(prm)), "plam_default_params")
    return prm


def plam_create(n: int, p: int, obj: plam_objective_t, prm: plam_params_t, stream: int = 0) -> C.c_void_p:
    h = C.c_void_p()
    check(load().plam_create(C.byref(h), n, p, C.byref(obj), C.byref(prm), C.c_void_p(stream)),
          "plam_create")
    return h


def plam_create_sharded(n_local: int, p: int, obj: plam_objective_t, prm: plam_params_t,
                        comm: plam_comm_t, stream: int = 0) -> C.c_void_p:
    h = C.c_void_p()
    check(load().plam_create_sharded(C.byref(h), n_local, p, C.byref(obj), C.byref(prm),
                                     C.byref(comm), C.c_void_p(stream)), "plam_create_sharded")
    return h


def plam_destroy(h) -> int:
    return load().plam_destroy(h)


def plam_reset(h) -> int:
    return check(load().plam_reset(h), "plam_reset")


def plam_step(h, X: int, ldx: int):
    info = plam_info_t()
    st = load().plam_step(h, C.c_void_p(X), ldx, C.byref(info))
    return st, info


def pcal_step(h, X: int, ldx: int):
    info = plam_info_t()
    st = load().pcal_step(h, C.c_void_p(X), ldx, C.byref(info))
    return st, info


def plam_solve(h, X: int, ldx: int, Xout: int | None, ldo: int):
    info = plam_info_t()
    st = load().plam_solve(h, C.c_void_p(X), ldx, C.c_void_p(Xout or 0), ldo, C.byref(info))
    return st, info


def plam_orthonormalize(h, X: int, ldx: int, Xout: int, ldo: int, passes: int = 1, want_feas=True):
    feas = C.c_double(float("nan"))
    st = load().plam_orthonormalize(h, C.c_void_p(X), ldx, C.c_void_p(Xout), ldo, passes,
                                    C.byref(feas) if want_feas else None)
    return st, feas.value


def plam_energy(h, X: int, ldx: int, f_dev: int):
    return load().plam_energy(h, C.c_void_p(X), ldx, C.c_void_p(f_dev))


def plam_energy_backward(h, X: int, ldx: int, scale_dev, G: int, ldg: int):
    return load().plam_energy_backward(h, C.c_void_p(X), ldx,
                                       C.c_void_p(scale_dev) if scale_dev else None,
                                       C.c_void_p(G), ldg)


def plam_energy_grad(h, X: int, ldx: int, G: int, ldg: int, want_f=True):
    f = C.c_double(float("nan"))
    st = load().plam_energy_grad(h, C.c_void_p(X), ldx, C.c_void_p(G), ldg,
                                 C.byref(f) if want_f else None)
    return st, f.value


def plam_grams(h, X: int, ldx: int, G: int | None, ldg: int, B: int, Cm: int | None):
    return load().plam_grams(h, C.c_void_p(X), ldx, C.c_void_p(G or 0), ldg, C.c_void_p(B),
                             C.c_void_p(Cm or 0))


def plam_grams_noalloc(n: int, p: int, precision: int, X: int, ldx: int, G: int | None, ldg: int,
                       B: int, Cm: int | None, stream: int = 0):
    return load().plam_grams_noalloc(n, p, precision, C.c_void_p(X), ldx, C.c_void_p(G or 0), ldg,
                                     C.c_void_p(B), C.c_void_p(Cm or 0), C.c_void_p(stream))


KERNEL_GROUPS = ("objective", "gram_partial", "gram_finalize", "update", "step_size", "primal_update")


def plam_time_kernels(h, X: int, ldx: int, iters: int):
    ms = (C.c_double * 6)()
    done = C.c_int(0)
    st = load().plam_time_kernels(h, C.c_void_p(X), ldx, iters, ms, C.byref(done))
    return st, dict(zip(KERNEL_GROUPS, list(ms))), done.value


def plam_last_iteration(h, R: int | None, ldr: int, M: int | None, p: int):
    """(status, colsums[3p], bb[3]) of the latest evaluated iterate; R and M are device
    pointers (or None) that receive the residual and the update matrix."""
    import numpy as np
    cols = (C.c_double * (3 * p))()
    bb = (C.c_double * 3)()
    st = load().plam_last_iteration(h, C.c_void_p(R or 0), ldr, C.c_void_p(M or 0), cols, bb)
    return st, np.array(cols[:]), np.array(bb[:])


def plam_history(h, cap: int):
    import numpy as np
    buf = (C.c_double * (5 * max(cap, 1)))()
    cnt = C.c_int(0)
    check(load().plam_history(h, buf, cap, C.byref(cnt)), "plam_history")
    return np.frombuffer(buf, dtype=np.float64, count=5 * cnt.value).reshape(cnt.value, 5).copy()


def plam_kernel_launches(h) -> int:
    return int(load().plam_kernel_launches(h))


def plam_version() -> int:
    return int(load().plam_version())


def plam_batch_create(problems, params, stream):
    arr = (plam_batch_problem_t * len(problems))(*problems)
    h = C.c_void_p()
    check(load().plam_batch_create(C.byref(h), arr, len(problems), C.byref(params),
                                   C.c_void_p(stream)), "plam_batch_create")
    return h


def plam_batch_solve(h, count: int):
    infos = (plam_info_t * count)()
    st = load().plam_batch_solve(h, infos)
    return st, list(infos)


def plam_batch_autotune(h, iters: int):
    tile = C.c_int()
    ms = C.c_double()
    st = load().plam_batch_autotune(h, iters, C.byref(tile), C.byref(ms))
    return st, tile.value, ms.value


def plam_batch_set_tile(h, tile_rows: int):
    return load().plam_batch_set_tile(h, tile_rows)


def plam_batch_destroy(h):
    return load().plam_batch_destroy(h)
