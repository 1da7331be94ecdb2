"""GB300 (sm_103a) PLAM / PCAL hot path (arXiv:1810.03930).

The computation lives in lib/libplam.so (C ABI: include/plam.h).  `_lib`
forwards the C entry points under the same names; `Solver` marshals torch
device tensors (column-major n x p matrices stored as (p, ld) row-major
tensors) into those calls.  PyTorch provides device memory and streams only.
"""
from __future__ import annotations

import numpy as np

from . import _lib
from ._lib import (PLAM_ETA_ABB, PLAM_ETA_BB1, PLAM_ETA_BB2, PLAM_ETA_CONST, PLAM_ETA_DIFF,  # noqa: F401
                   PLAM_LAMBDA1, PLAM_LAMBDA2, PLAM_OBJ_CALLBACK, PLAM_OBJ_DENSE,
                   PLAM_OBJ_HARTREE1D, PLAM_OBJ_STENCIL3D, PLAM_PREC_FP32, PLAM_PREC_FP64,
                   PLAM_VARIANT_PCAL, PLAM_VARIANT_PLAM, PlamError, check, pcal_step, plam_create,
                   plam_default_params, plam_destroy, plam_energy, plam_energy_backward,
                   plam_energy_grad, plam_grams, plam_history, plam_kernel_launches,
                   plam_orthonormalize, plam_reset, plam_solve, plam_step, plam_time_kernels)

_RULES = {"abb": PLAM_ETA_ABB, "bb1": PLAM_ETA_BB1, "bb2": PLAM_ETA_BB2, "const": PLAM_ETA_CONST,
          "diff": PLAM_ETA_DIFF}


def _torch():
    import torch
    return torch


def storage_dtype(precision: str):
    torch = _torch()
    return torch.float64 if precision == "fp64" else torch.float32


def colmajor_to_device(M: np.ndarray, dtype, device="cuda", ld: int | None = None):
    """An n x p (or n-vector) host array as a device tensor of shape (p, ld) holding it column-major."""
    torch = _torch()
    M = np.asarray(M)
    if M.ndim == 1:
        return torch.as_tensor(np.ascontiguousarray(M), device=device).to(dtype)
    n, p = M.shape
    ld = ld or n
    t = torch.zeros((p, ld), dtype=dtype, device=device)
    t[:, :n] = torch.as_tensor(np.ascontiguousarray(M.T), device=device).to(dtype)
    return t


class _DeviceBuffer:
    """A raw device buffer exposed through __cuda_array_interface__ (zero copy)."""

    def __init__(self, ptr: int, shape, strides, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "strides": tuple(strides),
                                         "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3}


def _colmajor_view(ptr: int, n: int, p: int, ld: int, dtype):
    """The n x p column-major matrix at device address ptr as an (n, p) tensor view."""
    torch = _torch()
    esz = 8 if dtype == torch.float64 else 4
    buf = _DeviceBuffer(ptr, (n, p), (esz, ld * esz), "<f8" if esz == 8 else "<f4")
    return torch.as_tensor(buf, device="cuda")


def _energy_function():
    """torch.autograd.Function over a Solver's built-in objective: the forward kernels give
    f(X) on the device, the backward kernels grad_out * grad f(X) (plam_energy and
    plam_energy_backward).  X is a (p, ld) tensor holding the column-major n x p matrix."""
    torch = _torch()

    class EnergyFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, X, solver):
            if X.dim() != 2 or X.stride(1) != 1 or X.shape[0] != solver.p or X.shape[1] < solver.n:
                raise ValueError("X must be a (p, ld >= n) tensor with unit stride along ld")
            f = torch.empty((1,), dtype=torch.float64, device=X.device)
            check(plam_energy(solver.h, X.data_ptr(), X.stride(0), f.data_ptr()), "plam_energy")
            ctx.save_for_backward(X)
            ctx.solver = solver
            return f[0]

        @staticmethod
        def backward(ctx, grad_out):
            (X,) = ctx.saved_tensors
            solver = ctx.solver
            G = torch.zeros_like(X)
            s = grad_out.detach().to(torch.float64).reshape(1).contiguous()
            check(plam_energy_backward(solver.h, X.data_ptr(), X.stride(0), s.data_ptr(),
                                       G.data_ptr(), G.stride(0)), "plam_energy_backward")
            return G, None

    return EnergyFn


_ENERGY_FN = None


def device_to_colmajor(t, n: int) -> np.ndarray:
    """Inverse of colmajor_to_device: an n x p float64 host array (Fortran order)."""
    return np.asfortranarray(t[:, :n].double().cpu().numpy().T)


class Solver:
    """One plam_handle_t with its objective; inputs and outputs are torch device tensors.

    Matrices are torch tensors of shape (p, ld) whose memory is the column-major
    n x p matrix (ld = leading dimension >= n).

    kind: "dense" (A), "qap" (A and the p x p B of Problem 4, f = 1/2 tr(A^T X B X^T)),
    "hartree1d" (alpha, quad_scale, xc; block = rows per Dirichlet block
    of L, 0 for one block; lin = the linear term G_lin of Problem 2, n x p), "stencil3d"
    (grid = (nx, ny, nz), V) or "callback" (energy = a torch function of the (n, p) iterate).
    The other keywords are the fields of plam_params_t (include/plam.h).
    """

    def __init__(self, n, p, kind, *, A=None, B=None, alpha=1.0, quad_scale=0.25, xc=0.0, block=0, lin=None,
                 grid=None, V=None,
                 variant="pcal", lambda_rule="lambda2", beta=1.0, eta_rule="abb", eta0=0.0,
                 eta_gamma=0.0, tol=1e-8, maxit=3000, precision="fp64", final_orth=1,
                 graph_iters=16, engine="auto", tensor_cores="auto", refine_switch=1e-3,
                 energy=None, orth_metrics=True, stream=None, shard=None, feas_max=1e6,
                 eta_min=0.0, eta_max=0.0):
        torch = _torch()
        self.n, self.p = int(n), int(p)
        self.precision = precision
        self.dtype = storage_dtype(precision)
        prm = plam_default_params()
        prm.variant = {"plam": PLAM_VARIANT_PLAM, "pcal": PLAM_VARIANT_PCAL,
                       "moptqr": _lib.PLAM_VARIANT_MOPTQR}[variant]
        prm.lambda_rule = {"lambda1": PLAM_LAMBDA1, "lambda2": PLAM_LAMBDA2, "da": 2}[lambda_rule]
        prm.beta = float(beta)
        prm.eta_rule = _RULES[eta_rule]
        prm.eta0 = float(eta0)
        prm.eta_gamma = float(eta_gamma)
        prm.tol = float(tol)
        prm.maxit = int(maxit)
        prm.precision = PLAM_PREC_FP64 if precision == "fp64" else PLAM_PREC_FP32
        prm.final_orth = int(final_orth)
        prm.graph_iters = int(graph_iters)
        prm.engine = {"auto": 0, "graph": 1, "resident": 2}[engine]
        prm.tensor_cores = {"auto": -1, "off": 0, "on": 1, "tf32": 1, "3xtf32": 2,
                            "tf32-single": 1 | _lib.PLAM_TC_SINGLE_CTA,
                            "3xtf32-single": 2 | _lib.PLAM_TC_SINGLE_CTA}[tensor_cores]
        prm.refine_switch = float(refine_switch)
        prm.orth_metrics = 1 if orth_metrics else 0
        prm.feas_max = float(feas_max)
        prm.eta_min = float(eta_min)
        prm.eta_max = float(eta_max)
        self.params = prm
        obj = _lib.plam_objective_t()
        self._keep = []
        if kind in ("dense", "qap"):
            At = A if isinstance(A, torch.Tensor) else colmajor_to_device(A, self.dtype)
            self._keep.append(At)
            obj.kind, obj.A, obj.lda = PLAM_OBJ_DENSE, At.data_ptr(), At.stride(0)
            if kind == "qap":
                Bt = B if isinstance(B, torch.Tensor) else colmajor_to_device(B, self.dtype)
                self._keep.append(Bt)
                obj.kind, obj.Bq, obj.ldbq = _lib.PLAM_OBJ_QAP, Bt.data_ptr(), Bt.stride(0)
        elif kind == "hartree1d":
            obj.kind, obj.alpha, obj.quad_scale = PLAM_OBJ_HARTREE1D, float(alpha), float(quad_scale)
            obj.xc = float(xc)
            obj.block = int(block)
            if lin is not None:
                Lt = lin if isinstance(lin, torch.Tensor) else colmajor_to_device(lin, self.dtype)
                self._keep.append(Lt)
                obj.lin, obj.ldlin = Lt.data_ptr(), Lt.stride(0)
        elif kind == "stencil3d":
            nx, ny, nz = grid
            obj.kind, obj.nx, obj.ny, obj.nz = PLAM_OBJ_STENCIL3D, nx, ny, nz
            if V is not None:
                Vt = V if isinstance(V, torch.Tensor) else colmajor_to_device(V, self.dtype)
                self._keep.append(Vt)
                obj.V = Vt.data_ptr()
        elif kind == "callback":
            if energy is None:
                raise ValueError("kind='callback' needs energy=callable(X) -> scalar tensor")
            self._cb_error = None
            self._cb = _lib.plam_grad_fn(self._make_callback(energy))
            obj.kind, obj.grad = PLAM_OBJ_CALLBACK, self._cb
        else:
            raise ValueError(kind)
        self.objective = obj
        self.stream = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        if shard is not None:
            # a row-sharded handle (plam_create_sharded): n is this rank's row count and the
            # objective describes its rows; shard = (comm struct, its Python callbacks)
            self.comm, self._comm_keep = shard
            self.h = _lib.plam_create_sharded(self.n, self.p, obj, prm, self.comm, self.stream)
        else:
            self.h = plam_create(self.n, self.p, obj, prm, self.stream)

    def _make_callback(self, energy):
        """The C gradient callback of a user energy: f = energy(X) on an (n, p) view of X,
        grad f by torch.autograd, both written as stream-ordered device work."""
        torch = _torch()
        n, p, dtype = self.n, self.p, self.dtype

        def cb(ctx, Xp, ldx, Gp, ldg, fp, stream):
            try:
                s = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
                with torch.cuda.stream(s):
                    X = _colmajor_view(Xp, n, p, ldx, dtype).detach().requires_grad_(True)
                    with torch.enable_grad():
                        f = energy(X)
                        (g,) = torch.autograd.grad(f, X)
                    _colmajor_view(Gp, n, p, ldg, dtype).copy_(g)
                    fo = torch.as_tensor(_DeviceBuffer(fp, (1,), (8,), "<f8"), device="cuda")
                    fo.copy_(f.detach().to(torch.float64).reshape(1))
                return 0
            except Exception as e:       # reported by the C entry point as PLAM_ERR_CUDA
                self._cb_error = e
                return 1

        return cb

    def energy(self, X):
        """f(X) as a differentiable 0-dim tensor (built-in objectives; backward = grad f)."""
        global _ENERGY_FN
        if _ENERGY_FN is None:
            _ENERGY_FN = _energy_function()
        return _ENERGY_FN.apply(X, self)

    def close(self):
        if getattr(self, "h", None) is not None:
            plam_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def new_matrix(self, dtype=None, ld=None):
        torch = _torch()
        return torch.zeros((self.p, ld or self.n), dtype=dtype or self.dtype, device="cuda")

    def step(self, X, variant=None):
        variant = variant or ("pcal" if self.params.variant == PLAM_VARIANT_PCAL else "plam")
        fn = pcal_step if variant == "pcal" else plam_step
        st, info = fn(self.h, X.data_ptr(), X.stride(0))
        check(st, f"{variant}_step", ok=(0, 3))
        return st, info

    def solve(self, X, Xout=None):
        st, info = plam_solve(self.h, X.data_ptr(), X.stride(0),
                              Xout.data_ptr() if Xout is not None else None,
                              Xout.stride(0) if Xout is not None else 0)
        check(st, "plam_solve", ok=(0, 2, 3))
        return st, info

    def orthonormalize(self, X, Xout, passes=1):
        st, feas = plam_orthonormalize(self.h, X.data_ptr(), X.stride(0), Xout.data_ptr(),
                                       Xout.stride(0), passes)
        check(st, "plam_orthonormalize")
        return feas

    def energy_grad(self, X, G):
        st, f = plam_energy_grad(self.h, X.data_ptr(), X.stride(0), G.data_ptr(), G.stride(0))
        check(st, "plam_energy_grad")
        return f

    def grams(self, X, G=None):
        torch = _torch()
        B = torch.empty((self.p, self.p), dtype=torch.float64, device="cuda")
        Cm = torch.empty((self.p, self.p), dtype=torch.float64, device="cuda") if G is not None else None
        st = plam_grams(self.h, X.data_ptr(), X.stride(0), G.data_ptr() if G is not None else None,
                        G.stride(0) if G is not None else 0, B.data_ptr(),
                        Cm.data_ptr() if Cm is not None else None)
        check(st, "plam_grams")
        # (p, p) row-major tensors holding column-major matrices: transpose back
        return B.t().contiguous(), (Cm.t().contiguous() if Cm is not None else None)

    def time_kernels(self, X, iters):
        """Average per-launch milliseconds of each kernel group over up to `iters` iterations."""
        st, ms, done = plam_time_kernels(self.h, X.data_ptr(), X.stride(0), iters)
        check(st, "plam_time_kernels")
        return ms, done

    def last_iteration(self):
        """The latest evaluated iterate's residual R (a (p, n) tensor), update matrix M (p x p,
        as a (p, p) tensor holding it column-major: M is symmetric), reduced column dots
        (3p: ||X_i||^2, <X_i, R_i>, ||R_i||^2) and Barzilai-Borwein dots (<S,S>, <S,Y>, <Y,Y>)."""
        torch = _torch()
        R = torch.empty((self.p, self.n), dtype=self.dtype, device="cuda")
        M = torch.empty((self.p, self.p), dtype=self.dtype, device="cuda")
        st, cols, bb = _lib.plam_last_iteration(self.h, R.data_ptr(), self.n, M.data_ptr(), self.p)
        check(st, "plam_last_iteration")
        return R, M, cols, bb

    def get_state(self) -> bytes:
        """The run's iteration state (plam_get_state) as bytes: a checkpoint that, with the X of
        the same iterate, lets plam_step / pcal_step continue the run exactly."""
        nb = _lib.load().plam_state_bytes(self.h)
        buf = (_lib.C.c_char * nb)()
        check(_lib.load().plam_get_state(self.h, buf, nb), "plam_get_state")
        return bytes(buf)

    def set_state(self, state: bytes):
        buf = (_lib.C.c_char * len(state)).from_buffer_copy(state)
        check(_lib.load().plam_set_state(self.h, buf, len(state)), "plam_set_state")

    def history(self):
        return plam_history(self.h, self.params.maxit + 2)

    def reset(self):
        plam_reset(self.h)

    def engine(self):
        """'resident', 'graph' or 'direct': what solve() runs on this handle."""
        e = _lib.load().plam_solve_engine(self.h)
        return {2: "resident", 1: "graph"}.get(e, "direct")

    def kernel_launches(self):
        return plam_kernel_launches(self.h)


class BatchSolver:
    """Many independent dense trace problems f_b = 1/2 tr(X_b^T A_b X_b) (p_b <= 64) solved in one
    persistent launch (plam_batch_*).  As, X0s: sequences of n_b x n_b and n_b x p_b host arrays
    (or (p, ld) device tensors from colmajor_to_device).  FP32 storage; FP64 outputs Q_b."""

    def __init__(self, As, X0s, *, variant="pcal", lambda_rule="lambda2", beta=1.0, eta_rule="abb",
                 eta0=0.0, eta_gamma=0.0, tol=1e-6, maxit=3000, orthonormalize=True, stream=None,
                 eta_min=0.0, eta_max=0.0):
        torch = _torch()
        prm = plam_default_params()
        prm.variant = PLAM_VARIANT_PCAL if variant == "pcal" else PLAM_VARIANT_PLAM
        prm.lambda_rule = PLAM_LAMBDA2 if lambda_rule == "lambda2" else PLAM_LAMBDA1
        prm.beta, prm.eta_rule = float(beta), _RULES[eta_rule]
        prm.eta0, prm.eta_gamma = float(eta0), float(eta_gamma)
        prm.tol, prm.maxit = float(tol), int(maxit)
        prm.eta_min, prm.eta_max = float(eta_min), float(eta_max)
        prm.precision = PLAM_PREC_FP32
        self.A, self.X, self.Q, probs = [], [], [], []
        for A, X0 in zip(As, X0s):
            At = A if isinstance(A, torch.Tensor) else colmajor_to_device(A, torch.float32)
            Xt = X0 if isinstance(X0, torch.Tensor) else colmajor_to_device(X0, torch.float32)
            p, n = Xt.shape[0], (X0.shape[0] if not isinstance(X0, torch.Tensor) else At.shape[0])
            Qt = torch.zeros((p, n), dtype=torch.float64, device="cuda") if orthonormalize else None
            self.A.append(At)
            self.X.append(Xt)
            self.Q.append(Qt)
            probs.append(_lib.plam_batch_problem_t(n, p, At.data_ptr(), At.stride(0), Xt.data_ptr(),
                                                   Xt.stride(0), Qt.data_ptr() if Qt is not None else None,
                                                   Qt.stride(0) if Qt is not None else 0))
        self.count = len(probs)
        self.stream = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        self.h = _lib.plam_batch_create(probs, prm, self.stream)

    def solve(self):
        st, infos = _lib.plam_batch_solve(self.h, self.count)
        check(st, "plam_batch_solve")
        return infos

    def autotune(self, iters=20):
        st, tile, ms = _lib.plam_batch_autotune(self.h, int(iters))
        check(st, "plam_batch_autotune")
        return tile, ms

    def set_tile(self, tile_rows):
        check(_lib.plam_batch_set_tile(self.h, int(tile_rows)), "plam_batch_set_tile")

    def close(self):
        if getattr(self, "h", None) is not None:
            _lib.plam_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
