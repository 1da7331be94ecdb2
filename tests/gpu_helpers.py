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


# Entry-wise tolerance factor for iterates after several iterations, against an earlier bound on
# their relative Frobenius-norm error: accumulated rounding is noise-like, and the largest of
# N ~ 1e4..1e5 such errors exceeds their RMS by about sqrt(2 ln N) ~ 4.3..4.8.  A single wrong
# entry (a boundary row, a ragged tile), off by far more than the noise, still fails.
ITER_FACTOR = 5.0


def column_rms(ref):
    """Per-column root mean square of an n x p array (the scale of that column's entries)."""
    ref = np.asarray(ref, dtype=np.float64)
    if ref.ndim == 1:
        return np.sqrt(np.mean(ref * ref))
    return np.sqrt(np.mean(ref * ref, axis=0))[None, :]


def assert_entrywise(got, ref, rtol, scale=None, what=""):
    """Every entry: |got - ref| <= rtol (|ref| + scale), scale the per-column RMS of ref unless
    given (the local magnitude an entry's rounding error is proportional to, so that entries
    near zero by cancellation are not held to a relative bound).  A single wrong entry (a
    boundary row, a ragged tile) fails, which a Frobenius-norm comparison would hide."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    if scale is None:
        scale = column_rms(ref)
    bound = rtol * (np.abs(ref) + scale)
    diff = np.abs(got - ref)
    ratio = np.where(bound > 0, diff / np.where(bound > 0, bound, 1.0), np.where(diff > 0, np.inf, 0.0))
    worst = np.unravel_index(int(np.argmax(ratio)), ratio.shape)
    assert np.all(np.isfinite(got)), f"{what}: non-finite entries"
    assert ratio[worst] <= 1.0, (f"{what}: entry {tuple(int(i) for i in worst)} differs by "
                                 f"{diff[worst]:.3e} from {ref[worst]:.6e} (bound {bound[worst]:.3e}, "
                                 f"{ratio[worst]:.2f}x the tolerance rtol={rtol:g})")
    return float(ratio[worst])
