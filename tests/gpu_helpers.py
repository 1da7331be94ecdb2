"""Helpers for the GPU parity tests: build a GPU solver and the matching oracle objective
from one workloads.Workload, and move column-major matrices between host and device."""
import numpy as np

from oracle import objectives as oo


def gpu_solver(w, precision="fp64", **kw):
    from paper_1810_03930_gb300 import Solver
    if w.kind == "dense":
        return Solver(w.n, w.p, "dense", A=w.A, precision=precision, **kw)
    if w.kind == "hartree1d":
        return Solver(w.n, w.p, "hartree1d", alpha=w.alpha, quad_scale=w.quad_scale, xc=w.xc,
                      block=w.block, lin=w.lin, precision=precision, **kw)
    if w.kind == "stencil3d":
        return Solver(w.n, w.p, "stencil3d", grid=(w.m, w.m, w.m), V=w.V, precision=precision, **kw)
    raise ValueError(w.kind)


def oracle_objective(w):
    return oo.objective_for(w)


def to_dev(M, solver, ld=None):
    from paper_1810_03930_gb300 import colmajor_to_device
    return colmajor_to_device(M, solver.dtype, ld=ld)


def to_host(t, n):
    from paper_1810_03930_gb300 import device_to_colmajor
    return device_to_colmajor(t, n)


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
