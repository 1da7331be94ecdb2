"""Row-sharded solves (plam_create_sharded) on one GPU: P ranks emulated by host threads
(dist.LocalComm), each with its own handle and stream on its own rows, meeting only at the
library's all-gathers and halo exchanges (host barriers; no kernel waits for another rank's).

Against the single-handle solve of the same problem from the same start: the step sizes and
KKT values of the first iterations (the rank-order sums change only the summation order of the
Grams and dots, so FP64 agrees to ~1e-12 and the Barzilai-Borwein sequence to 1e-9), the
converged objective (against Ky Fan's optimum from the oracle), and the orthonormalised output
assembled from the ranks' rows against the single handle's, entry by entry."""
import threading

import numpy as np
import pytest

from oracle import objectives as oo
from tests.gpu_helpers import to_dev, to_host
from workloads import orthonormal_start, rng_for, workload_block_hartree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _run_ranks(size, fn):
    """fn(rank) on `size` threads; returns their results (re-raises the first failure)."""
    out, errs = [None] * size, []

    def work(r):
        try:
            torch.cuda.set_device(0)
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                out[r] = fn(r, s)
            s.synchronize()
        except Exception as e:          # noqa: BLE001  reported below
            errs.append((r, e))

    ts = [threading.Thread(target=work, args=(r,)) for r in range(size)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if errs:
        raise errs[0][1]
    return out


def _stencil_case(m, p, seed):
    rng = rng_for(30, 0, sub=seed)
    V = rng.uniform(0.0, 1.0, m ** 3)
    X0 = orthonormal_start(m ** 3, p, rng_for(30, 1, sub=seed))
    return V, X0


def _single_stencil(m, p, V, X0, precision, **kw):
    from paper_1810_03930_gb300 import Solver
    s = Solver(m ** 3, p, "stencil3d", grid=(m, m, m), V=V, precision=precision, **kw)
    Xd = to_dev(X0, s)
    Qd = s.new_matrix(dtype=torch.float64)
    st, info = s.solve(Xd, Qd)
    out = (st, info, s.history(), to_host(Qd, m ** 3))
    s.close()
    return out


def _sharded_stencil(size, m, p, V, X0, precision, **kw):
    from paper_1810_03930_gb300 import colmajor_to_device, storage_dtype
    from paper_1810_03930_gb300.dist import LocalComm, ShardedStencil, sharded_solver
    comm = LocalComm(size)
    dtype = storage_dtype(precision)

    def rank(r, stream):
        sl = ShardedStencil((m, m, m), r, size)
        rows = slice(sl.row0, sl.row0 + sl.n_local)
        Vr = torch.as_tensor(np.ascontiguousarray(V[rows]), device="cuda").to(dtype)
        s = sharded_solver(comm.member(r), "stencil3d", sl.n_local, p, sl.row0, sl.n_global,
                           grid=(m, m, sl.nz_local), V=Vr, precision=precision,
                           stream=stream.cuda_stream, **kw)
        buf, X = sl.new_x(p, dtype)
        X[:, :sl.n_local] = colmajor_to_device(X0[rows], dtype)
        Q = torch.zeros((p, sl.n_local), dtype=torch.float64, device="cuda")
        st, info = s.solve(X, Q)
        torch.cuda.current_stream().synchronize()
        res = (st, info, s.history(), Q.cpu().numpy().T.copy(), sl.row0)
        s.close()
        return res

    return _run_ranks(size, rank)


@pytest.mark.parametrize("size", [2, 3])
def test_sharded_stencil_solve_matches_the_single_handle_fp64(size):
    """20^3 grid (8000 rows; 3 ranks hold 7, 7 and 6 z-planes), p = 12, FP64 PCAL to KKT 1e-9."""
    m, p = 20, 12
    V, X0 = _stencil_case(m, p, size)
    beta = 12.0 + V.max() + 0.1
    kw = dict(variant="pcal", beta=beta, tol=1e-9, maxit=5000, final_orth=1)
    st1, info1, h1, Q1 = _single_stencil(m, p, V, X0, "fp64", orth_metrics=False, **kw)
    ranks = _sharded_stencil(size, m, p, V, X0, "fp64", **kw)
    assert st1 == 0
    # every rank took identical decisions: the same history, bit for bit
    for st, info, h, _, _ in ranks:
        assert st == 0 and info.iters == ranks[0][1].iters
        assert np.array_equal(h, ranks[0][2], equal_nan=True)
    h = ranks[0][2]
    k = min(20, len(h), len(h1))
    np.testing.assert_allclose(h[:k, 4], h1[:k, 4], rtol=1e-9)      # eta
    np.testing.assert_allclose(h[:k, 2], h1[:k, 2], rtol=1e-8)      # relative KKT
    assert abs(ranks[0][1].iters - info1.iters) <= max(5, 0.25 * info1.iters)
    # the orthonormalised output, assembled from the ranks' rows
    Q = np.zeros_like(Q1)
    for _, _, _, Qr, row0 in ranks:
        Q[row0:row0 + Qr.shape[0]] = Qr
    obj = oo.Stencil3DObjective(m, V)
    fstar, _ = oo.trace_min_optimum(obj.H, p)
    assert abs(obj.value(Q) - fstar) <= 1e-10 * abs(fstar)
    assert np.abs(Q.T @ Q - np.eye(p)).max() <= 1e-13
    # the subspaces agree (the spectrum has a gap at p on this instance)
    assert np.linalg.norm(Q - Q1 @ (Q1.T @ Q), 2) <= 1e-6


def test_sharded_stencil_first_iterations_fp32():
    """FP32 storage, 3 ranks on a 24^3 grid, p = 16: the first 10 step sizes and KKT values as the
    single handle's to FP32 rounding."""
    m, p = 24, 16
    V, X0 = _stencil_case(m, p, 7)
    kw = dict(variant="pcal", beta=1.0, tol=0.0, maxit=10, final_orth=0)
    _, _, h1, _ = _single_stencil(m, p, V, X0, "fp32", orth_metrics=False, engine="graph",
                                  graph_iters=0, **kw)
    ranks = _sharded_stencil(3, m, p, V, X0, "fp32", **kw)
    h = ranks[0][2]
    np.testing.assert_allclose(h[:10, 4], h1[:10, 4], rtol=2e-4)
    np.testing.assert_allclose(h[:, 2], h1[:, 2], rtol=2e-4)


def test_sharded_block_hartree_matches_the_single_handle():
    """Section 5.4's Problem 1 (blocks of 5 rows, alpha = 1) at n = 2000, p = 20 on 2 ranks,
    FP64 to KKT 1e-9: the blocks never cross ranks, so each rank's gradient is purely local."""
    from paper_1810_03930_gb300 import Solver, colmajor_to_device
    from paper_1810_03930_gb300.dist import LocalComm, shard_rows, sharded_solver
    w = workload_block_hartree(2000, 20)
    kw = dict(variant="pcal", beta=1.0, tol=1e-9, maxit=5000, final_orth=1, precision="fp64")
    s1 = Solver(w.n, w.p, "hartree1d", alpha=w.alpha, quad_scale=w.quad_scale, block=w.block,
                orth_metrics=False, **kw)
    Q1d = s1.new_matrix(dtype=torch.float64)
    st1, info1 = s1.solve(to_dev(w.X0, s1), Q1d)
    h1, Q1 = s1.history(), to_host(Q1d, w.n)
    s1.close()
    size = 2
    comm = LocalComm(size)
    plan = shard_rows(w.n, size, w.block)

    def rank(r, stream):
        row0, nl = plan[r]
        s = sharded_solver(comm.member(r), "hartree1d", nl, w.p, row0, w.n, alpha=w.alpha,
                           quad_scale=w.quad_scale, block=w.block, stream=stream.cuda_stream, **kw)
        X = colmajor_to_device(w.X0[row0:row0 + nl], torch.float64)
        Q = torch.zeros((w.p, nl), dtype=torch.float64, device="cuda")
        st, info = s.solve(X, Q)
        torch.cuda.current_stream().synchronize()
        res = (st, info, s.history(), Q.cpu().numpy().T.copy(), row0)
        s.close()
        return res

    ranks = _run_ranks(size, rank)
    assert st1 == 0 and all(r[0] == 0 for r in ranks)
    h = ranks[0][2]
    k = min(20, len(h), len(h1))
    np.testing.assert_allclose(h[:k, 4], h1[:k, 4], rtol=1e-9)
    np.testing.assert_allclose(h[:k, 1], h1[:k, 1], rtol=1e-12)     # f, with the Hartree partials
    Q = np.zeros_like(Q1)
    for _, _, _, Qr, row0 in ranks:
        Q[row0:row0 + Qr.shape[0]] = Qr
    obj = oo.objective_for(w)
    assert abs(obj.value(Q) - obj.value(Q1)) <= 1e-10 * abs(obj.value(Q1))
    assert np.abs(Q.T @ Q - np.eye(w.p)).max() <= 1e-13


def test_sharded_handles_reject_what_they_cannot_run():
    from paper_1810_03930_gb300 import PlamError
    from paper_1810_03930_gb300.dist import LocalComm, sharded_solver
    comm = LocalComm(2)
    with pytest.raises(PlamError):       # one global Dirichlet L couples every row
        sharded_solver(comm.member(0), "hartree1d", 500, 4, 0, 1000, alpha=1.0, block=0)
    with pytest.raises(PlamError):       # a slab must start on a z-plane
        sharded_solver(comm.member(1), "stencil3d", 8 * 8 * 3, 4, 70, 8 * 8 * 6, grid=(8, 8, 3))
