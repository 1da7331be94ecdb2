"""Tensor-core (tcgen05, kind::tf32) Grams of the FP32 mode against the definition.

TF32 keeps 10 of the 23 mantissa bits of each FP32 operand, so each product
carries a relative error below about 2 * 2^-10 and the entry (i, j) of X^T Y an
absolute error below 2.2 * 2^-10 * (|X|^T |Y|)_ij, plus the FP32 accumulation
error; that elementwise bound is what these tests check.
"""
import numpy as np
import pytest

from tests.gpu_helpers import to_dev
from workloads import Workload, orthonormal_start

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _solver(n, p, tc):
    from paper_1810_03930_gb300 import Solver
    return Solver(n, p, "hartree1d", precision="fp32", tensor_cores=tc)


@pytest.mark.parametrize("n,p", [(4099, 50), (3001, 128), (8192, 256), (2051, 300), (1000, 1),
                                 (6000, 17)])
def test_tensor_core_grams_within_tf32_bound(n, p):
    rng = np.random.default_rng(n * 7 + p)
    X = rng.standard_normal((n, p)).astype(np.float32).astype(np.float64)
    G = rng.standard_normal((n, p)).astype(np.float32).astype(np.float64)
    s = _solver(n, p, "on")
    ld = (n + 31) // 32 * 32          # 16-byte aligned columns: the tensor-core path applies
    Xd, Gd = to_dev(X, s, ld=ld), to_dev(G, s, ld=ld)
    B, Cm = s.grams(Xd, Gd)
    B, Cm = B.cpu().numpy(), Cm.cpu().numpy()
    absX, absG = np.abs(X), np.abs(G)
    tolB = 2.2 * 2.0 ** -10 * (absX.T @ absX) + 1e-5 * np.sqrt(n)
    tolC = 2.2 * 2.0 ** -10 * (absX.T @ absG) + 1e-5 * np.sqrt(n)
    assert np.all(np.abs(B - X.T @ X) <= tolB)
    assert np.all(np.abs(Cm - X.T @ G) <= tolC)
    # the tensor cores really ran: the result differs from exact FP32-product Grams
    # (a TF32 sum over thousands of rows cannot match to the last bit)
    s_off = _solver(n, p, "off")
    B2, C2 = s_off.grams(to_dev(X, s_off), to_dev(G, s_off))
    if n * p > 5000:
        assert not np.array_equal(Cm, C2.cpu().numpy())
    # fixed-order reduction: bitwise reproducible
    B3, C3 = s.grams(Xd, Gd)
    assert np.array_equal(B, B3.cpu().numpy()) and np.array_equal(Cm, C3.cpu().numpy())
    s.close()
    s_off.close()


def test_tensor_core_gram_without_g_and_unaligned_fallback():
    n, p = 5002, 130
    X = orthonormal_start(n, p, np.random.default_rng(1)).astype(np.float32).astype(np.float64)
    s = _solver(n, p, "on")
    Xd = to_dev(X, s, ld=n + 1)          # leading dimension 5003, not a multiple of 4: CUDA-core fallback
    B, _ = s.grams(Xd)
    assert np.abs(B.cpu().numpy() - X.T @ X).max() <= 2e-6 * np.sqrt(n)
    Xa = to_dev(X, s, ld=n + 2)          # 5004, a multiple of 4: tensor cores
    B2, _ = s.grams(Xa)
    bound = 2.2 * 2.0 ** -10 * (np.abs(X).T @ np.abs(X)) + 1e-5
    assert np.all(np.abs(B2.cpu().numpy() - X.T @ X) <= bound)
    s.close()


@pytest.mark.parametrize("n,p", [(8192, 256), (3001, 130), (6000, 17)])
def test_compensated_tensor_core_grams(n, p):
    """3xTF32 (hi*hi + hi*lo + lo*hi with round-to-nearest splits): each product carries about
    2^-21 relative error, so the Grams agree with the definition to near-FP32 accuracy."""
    from paper_1810_03930_gb300 import Solver
    rng = np.random.default_rng(n + 3 * p)
    X = rng.standard_normal((n, p)).astype(np.float32).astype(np.float64)
    G = rng.standard_normal((n, p)).astype(np.float32).astype(np.float64)
    s = Solver(n, p, "hartree1d", precision="fp32", tensor_cores="3xtf32")
    ld = (n + 31) // 32 * 32
    B, Cm = s.grams(to_dev(X, s, ld=ld), to_dev(G, s, ld=ld))
    absX, absG = np.abs(X), np.abs(G)
    tolB = 4 * 2.0 ** -21 * (absX.T @ absX) + 2e-6 * np.sqrt(n)
    tolC = 4 * 2.0 ** -21 * (absX.T @ absG) + 2e-6 * np.sqrt(n)
    assert np.all(np.abs(B.cpu().numpy() - X.T @ X) <= tolB)
    assert np.all(np.abs(Cm.cpu().numpy() - X.T @ G) <= tolC)
    s.close()


def test_tf32_rounding_is_unbiased():
    """Round-to-nearest conversion: the diagonal of X^T X for unit columns is not pulled low by the
    truncating FP32 -> TF32 read of the tensor cores (a bias of about 7e-4 before rounding)."""
    n, p = 8192, 128
    X = orthonormal_start(n, p, np.random.default_rng(5)).astype(np.float32).astype(np.float64)
    s = _solver(n, p, "on")
    B, _ = s.grams(to_dev(X, s, ld=n))
    d = np.diag(B.cpu().numpy()) - np.sum(X * X, axis=0)
    assert abs(d.mean()) < 2e-5
    s.close()


def test_compensated_grams_have_no_accumulation_drift():
    """The accumulator of tcgen05.mma truncates; summing each 32-row segment from zero and
    adding the segments with round-to-nearest FP32 keeps the drift of a long same-signed sum
    (a diagonal of X^T X) at a few 1e-7, where one accumulation over the whole chunk drifted
    by about -8e-6 at this size."""
    n, p = 65536, 128
    X = np.random.default_rng(9).standard_normal((n, p)).astype(np.float32).astype(np.float64)
    from paper_1810_03930_gb300 import Solver
    s = Solver(n, p, "hartree1d", precision="fp32", tensor_cores="3xtf32")
    B, _ = s.grams(to_dev(X, s, ld=n))
    ref = np.sum(X * X, axis=0)
    d = (np.diag(B.cpu().numpy()) - ref) / ref
    assert abs(d.mean()) < 1e-6
    assert np.abs(d).max() < 2e-6
    s.close()


@pytest.mark.parametrize("p,tc", [(64, "tf32"), (130, "tf32"), (64, "3xtf32")])
def test_tensor_core_solve_reaches_eigenvalue_sum(p, tc):
    """PCAL in FP32 with tensor-core Grams (TF32, compensated below the switch, or
    compensated throughout) on the 3D Laplacian plus potential: after the final FP64
    Cholesky-QR the objective equals half the sum of the p smallest eigenvalues to 1e-6
    relative and the columns are orthonormal to 1e-12."""
    import scipy.sparse.linalg as sla
    from oracle import objectives as oo
    from tests.gpu_helpers import gpu_solver, to_host
    from workloads import workload_stencil3d
    w = workload_stencil3d(m=20, p=p)
    obj = oo.Stencil3DObjective(w.m, w.V)
    ev = sla.eigsh(obj.H.tocsc(), k=p, sigma=-1.0, which="LM", return_eigenvectors=False)
    fstar = 0.5 * np.sort(ev)[:p].sum()
    beta = obj.hess_norm_bound() + 0.1
    s = gpu_solver(w, "fp32", variant="pcal", beta=beta, tol=1e-5, maxit=5000, final_orth=1,
                   tensor_cores=tc, engine="graph")
    Xd = to_dev(w.X0, s)
    Qd = s.new_matrix(dtype=torch.float64)
    st, info = s.solve(Xd, Qd)
    assert st == 0 and info.converged
    Q = to_host(Qd, w.n)
    assert abs(obj.value(Q) - fstar) <= 1e-6 * abs(fstar)
    assert np.linalg.norm(Q.T @ Q - np.eye(p)) <= 1e-12
    s.close()


# ---------------------------------------------------------------- tensor-core update GEMM


def _dense_case(n, p, seed):
    from workloads import workload_dense_trace
    w = workload_dense_trace(n, p)
    X0 = w.X0 + 0.02 * np.random.default_rng(seed).standard_normal(w.X0.shape)   # infeasible start
    return w, X0


@pytest.mark.parametrize("n,p", [(3001, 130), (2048, 256), (2900, 300), (1000, 40), (777, 1)])
@pytest.mark.parametrize("variant", ["plam", "pcal"])
@pytest.mark.parametrize("tc,tol", [("3xtf32", 2e-5), ("tf32", 4e-3), ("3xtf32-single", 2e-5)])
def test_tensor_core_update_three_iterations(n, p, variant, tc, tol):
    """Three FP32 iterations with the tcgen05 update GEMM R = G - X M (eq. S1) and its epilogue
    dots (column norms for PCAL's closed form, the Barzilai-Borwein sums of Section 5.1, the KKT
    residual of Section 3.3) against the FP64 oracle: the steps X^3 - X^0 and the step sizes
    eta^0..2 agree to the accuracy of the operand rounding (TF32: 2^-11; compensated 3xTF32: FP32
    level), the relative KKT values to TF32 level (its correction term X E is plain TF32).  Row
    blocks of 128 with a ragged tail, column tiles of 128 with a ragged tail (p = 130), a single
    column (p = 1); from p = 256 on CTA pairs take 256-row tiles (n = 2900: 23 row blocks, so
    the second CTA of the last pair lies past n; p = 300: the second CTA's half of the last
    column tile lies past p), and "-single" keeps one CTA per tile."""
    from oracle import objectives as oo
    from oracle import plam as op
    from tests.gpu_helpers import ITER_FACTOR, assert_entrywise, gpu_solver, to_host
    w, X0 = _dense_case(n, p, 17)
    obj = oo.TraceObjective(w.A)
    beta = 1.5
    ref = op.solve(obj, X0, variant=variant, beta=beta, tol=0.0, maxit=3)
    s = gpu_solver(w, "fp32", variant=variant, beta=beta, tol=0.0, maxit=3, final_orth=0,
                   tensor_cores=tc, refine_switch=0.0, engine="graph")
    Xd = to_dev(X0, s, ld=(n + 31) // 32 * 32)
    st, info = s.solve(Xd)
    hist = s.history()
    X3 = to_host(Xd, n)
    X0f = X0.astype(np.float32).astype(np.float64)
    assert_entrywise(X3 - X0f, ref.X - X0, ITER_FACTOR * 5 * tol, what="X^3 - X^0")
    eta_ref = np.array([h.eta for h in ref.history[:3]])
    kkt_ref = np.array([h.kkt for h in ref.history])
    np.testing.assert_allclose(hist[:3, 4], eta_ref, rtol=5 * tol)
    np.testing.assert_allclose(hist[:, 2], kkt_ref, rtol=max(5 * tol, 1e-3))
    s.close()


def test_tensor_core_update_replaces_the_cuda_core_update():
    """With tensor cores on, one iteration launches the TF32 split of M and the tcgen05 update
    in place of the CUDA-core update kernel (one launch more than the CUDA-core sequence)."""
    from tests.gpu_helpers import gpu_solver
    w, X0 = _dense_case(1024, 128, 3)
    counts = {}
    for tc in ("off", "tf32"):
        s = gpu_solver(w, "fp32", variant="pcal", beta=1.5, tol=0.0, maxit=1, tensor_cores=tc,
                       engine="graph")
        Xd = to_dev(X0, s, ld=1024)
        s.step(Xd)
        counts[tc] = s.kernel_launches()
        s.close()
    assert counts["tf32"] == counts["off"] + 1


@pytest.mark.parametrize("m,p", [(30, 256), (34, 130)])
@pytest.mark.parametrize("tc,tol", [("3xtf32", 2e-5), ("tf32", 4e-3), ("tf32-single", 4e-3)])
def test_tensor_core_update_persistent_tiles(m, p, tc, tol):
    """The persistent update kernel walks several 128 x 128 tiles per CTA (27000 or 39304 rows:
    hundreds of tiles on 152 SMs), alternating its two tensor-memory accumulator buffers and the
    two-slot epilogue ring; three PCAL iterations on the 3D stencil against the FP64 oracle."""
    from oracle import objectives as oo
    from oracle import plam as op
    from tests.gpu_helpers import ITER_FACTOR, assert_entrywise, gpu_solver, to_host
    from workloads import workload_stencil3d
    w = workload_stencil3d(m=m, p=p)
    obj = oo.Stencil3DObjective(w.m, w.V.astype(np.float32).astype(np.float64))
    X0 = w.X0 + 0.02 * np.random.default_rng(5).standard_normal(w.X0.shape)
    ref = op.solve(obj, X0, variant="pcal", beta=1.0, tol=0.0, maxit=3)
    s = gpu_solver(w, "fp32", variant="pcal", beta=1.0, tol=0.0, maxit=3, final_orth=0,
                   tensor_cores=tc, refine_switch=0.0, engine="graph")
    n = w.n
    Xd = to_dev(X0, s, ld=(n + 31) // 32 * 32)
    st, info = s.solve(Xd)
    hist = s.history()
    X3 = to_host(Xd, n)
    X0f = X0.astype(np.float32).astype(np.float64)
    assert_entrywise(X3 - X0f, ref.X - X0, ITER_FACTOR * 5 * tol, what="X^3 - X^0")
    # eta^2 = <Y,Y>/|<S,Y>| (BB2) divides differences of residuals, Y = R^2 - R^1: the TF32 error
    # of R is amplified by |R| / |Y| (up to ~10% here), so plain TF32 is held to eta^0, eta^1
    ne = 3 if tc == "3xtf32" else 2
    np.testing.assert_allclose(hist[:ne, 4], [h.eta for h in ref.history[:ne]], rtol=5 * tol)
    # K = R - X E with E = Psi(C) - M in plain TF32 (2^-12 relative to X E, which is not small
    # at an infeasible start): the KKT value carries that error in both modes
    np.testing.assert_allclose(hist[:, 2], [h.kkt for h in ref.history], rtol=max(5 * tol, 1e-3))
    s.close()
