"""MOptQR on the GPU (PLAM_VARIANT_MOPTQR: the projected gradient from the update kernel with
M = C^T, MOptQR's own Barzilai-Borwein sums, the Cholesky retraction in FP64 arithmetic every
iteration; Table "cost", Sections 5.3-5.4) against the oracle's MOptQR: the step sizes and KKT
values of the first iterations, the converged objective, and feasibility of every iterate.
Problem 2's linear term (Section 5.4's tridiagonal A with a random G_lin) makes X^T G
unsymmetric, so a transposed C^T in the update would show."""
import numpy as np
import pytest

from oracle import moptqr as om
from oracle import objectives as oo
from tests.gpu_helpers import gpu_solver, to_dev, to_host
from workloads import workload_dense_trace, workload_tridiag_linear

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("make", ["dense", "tridiag_linear"])
def test_moptqr_fp64_matches_oracle(make):
    w = workload_dense_trace(200, 8) if make == "dense" else workload_tridiag_linear(1000, 20)
    obj = oo.objective_for(w)
    ref = om.solve(obj, w.X0, tol=1e-9, maxit=5000)
    assert ref.converged
    s = gpu_solver(w, "fp64", variant="moptqr", tol=1e-9, maxit=5000, final_orth=1)
    Xd = to_dev(w.X0, s)
    Qd = s.new_matrix(dtype=torch.float64)
    st, info = s.solve(Xd, Qd)
    assert st == 0 and info.converged, info.as_dict()
    hist = s.history()
    k = min(20, len(hist), len(ref.history))
    np.testing.assert_allclose(hist[:k, 4], [h.eta for h in ref.history[:k]], rtol=1e-9)
    np.testing.assert_allclose(hist[:k, 2], [h.kkt for h in ref.history[:k]], rtol=1e-8)
    # every iterate is feasible: the retraction keeps ||X^T X - I||_F at rounding level
    assert np.all(hist[:, 3] <= 1e-12)
    assert abs(info.iters - ref.iters) <= max(5, 0.25 * ref.iters)
    X = to_host(Xd, w.n)
    assert abs(obj.value(X) - ref.f_orth) <= 1e-10 * abs(ref.f_orth)
    if make == "dense":
        fstar = 0.5 * np.linalg.eigvalsh(w.A)[:w.p].sum()
        assert abs(obj.value(X) - fstar) <= 1e-10 * abs(fstar)
    s.close()


@pytest.mark.parametrize("p,tc", [(20, "off"), (130, "auto")])
def test_moptqr_fp32_first_iterations_and_solve(p, tc):
    """FP32 storage (CUDA-core update at p = 20; tensor-core Grams and update at p = 130, whose
    C^T is not symmetric here): the first step sizes as the oracle's to the products' accuracy,
    then the solve to relative KKT 1e-5 and its objective against the oracle's."""
    w = workload_tridiag_linear(2000, p)
    X0f = w.X0.astype(np.float32).astype(np.float64)
    lin = w.lin.astype(np.float32).astype(np.float64)
    obj = oo.HartreeObjective(w.n, w.alpha, w.quad_scale, 0.0, 0, lin)
    ref = om.solve(obj, X0f, tol=1e-5, maxit=5000)
    s = gpu_solver(w, "fp32", variant="moptqr", tol=1e-5, maxit=5000, final_orth=1, tensor_cores=tc,
                   refine_switch=1e-3)
    Qd = s.new_matrix(dtype=torch.float64)
    Xd = to_dev(w.X0, s)
    st, info = s.solve(Xd, Qd)
    assert st == 0 and info.converged, info.as_dict()
    hist = s.history()
    tol = 1e-4 if tc == "off" else 5e-3
    np.testing.assert_allclose(hist[:4, 4], [h.eta for h in ref.history[:4]], rtol=tol)
    # the last iterate, feasible to FP32 storage (the device's own ||X^T X - I||_F comes from
    # the Grams of the iteration: TF32 ones, ~1e-3, until the compensated phase)
    X = to_host(Xd, w.n)
    assert np.linalg.norm(X.T @ X - np.eye(p)) <= 1e-5
    assert np.all(hist[:, 3] <= (1e-5 if tc == "off" else 2e-3))
    assert abs(obj.value(to_host(Qd, w.n)) - ref.f_orth) <= 1e-6 * abs(ref.f_orth)
    s.close()


def test_moptqr_kernel_groups_include_the_retraction():
    """plam_time_kernels on a MOptQR handle: the last group is the retraction (the copies, the
    step, the FP64 Gram of V, the Cholesky factor and V R^{-1}) and it is not free."""
    w = workload_tridiag_linear(4000, 64)
    s = gpu_solver(w, "fp64", variant="moptqr", tol=0.0, maxit=100, final_orth=0)
    ms, done = s.time_kernels(to_dev(w.X0, s), 5)
    assert done == 5 and ms["primal_update"] > 0.0
    s.close()
