"""Problem 4 (Section 5.2, eq. QAP), f = 1/2 tr(A^T X B X^T), as a built-in objective
(PLAM_OBJ_QAP: the dense kernel's A X, then the right-multiply kernel's (A X) B): the gradient
and energy against the oracle entry by entry (ragged 64-row and 64-column tiles), the
autograd pair (forward energy, backward kernels), and PCAL solves against the oracle's and
against the closed-form minimum for a diagonal B."""
import numpy as np
import pytest

from oracle import objectives as oo
from oracle import plam as op
from tests.gpu_helpers import assert_entrywise, to_dev, to_host
from workloads import gaussian_symmetric, orthonormal_start, paper_p4_matrices, rng_for

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _solver(A, B, precision, **kw):
    from paper_1810_03930_gb300 import Solver
    n, p = A.shape[0], B.shape[0]
    return Solver(n, p, "qap", A=A, B=B, precision=precision, **kw)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,p", [(333, 7), (200, 65), (130, 64)])
def test_qap_gradient_and_energy_match_oracle(precision, n, p):
    A, B = paper_p4_matrices(n, p, rng_for(24, 0, sub=n + p))
    X = orthonormal_start(n, p, rng_for(24, 1, sub=n)) + 0.01 * rng_for(24, 2).standard_normal((n, p))
    if precision == "fp32":
        A, B, X = (M.astype(np.float32).astype(np.float64) for M in (A, B, X))
    obj = oo.QAPObjective(A, B)
    s = _solver(A, B, precision)
    Gd = s.new_matrix()
    f = s.energy_grad(to_dev(X, s), Gd)
    # FP32: two chained single-precision products (n + p terms)
    tol = 1e-12 if precision == "fp64" else 1e-5
    assert_entrywise(to_host(Gd, n), obj.grad(X), tol, what="A X B")
    assert abs(f - obj.value(X)) <= 10 * tol * max(1.0, abs(obj.value(X)))
    # the autograd pair: forward kernels give f, backward kernels grad_out * A X B
    Xt = to_dev(X, s).requires_grad_(True)
    e = s.energy(Xt)
    (g,) = torch.autograd.grad(2.5 * e, Xt)
    assert abs(e.item() - obj.value(X)) <= 10 * tol * max(1.0, abs(obj.value(X)))
    assert_entrywise(to_host(g, n), 2.5 * obj.grad(X), tol, what="backward")
    s.close()


def test_qap_pcal_reaches_the_closed_form_minimum():
    """B = diag(3, 2, 1): min over X^T X = I is 1/2 sum_i b_i lambda_i(A), the largest b_i with
    the smallest eigenvalues (the oracle pins the same value); FP64 PCAL to KKT 1e-10."""
    n, p = 40, 3
    A = gaussian_symmetric(n, rng_for(23, 0))
    b = np.array([3.0, 2.0, 1.0])
    obj = oo.QAPObjective(A, np.diag(b))
    fstar = 0.5 * float(b @ np.linalg.eigvalsh(A)[:p])
    s = _solver(A, np.diag(b), "fp64", variant="pcal", beta=obj.hess_norm_bound() + 0.1, tol=1e-10,
                maxit=20000, final_orth=1)
    Qd = s.new_matrix(dtype=torch.float64)
    st, info = s.solve(to_dev(orthonormal_start(n, p, rng_for(23, 1)), s), Qd)
    assert st == 0 and info.converged
    Q = to_host(Qd, n)
    assert abs(obj.value(Q) - fstar) <= 1e-10 * abs(fstar)
    assert abs(info.f_orth - fstar) <= 1e-10 * abs(fstar)
    assert info.feas_orth <= 1e-12
    s.close()


@pytest.mark.parametrize("variant", ["plam", "pcal"])
def test_qap_solve_matches_oracle_run(variant):
    """Problem 4's generator (A, B symmetrised Gaussians), n = 300, p = 10, beta = s + 0.1, FP64
    to relative KKT 1e-8: the first 20 step sizes and KKT values as the oracle's, and the
    orthonormalised objective."""
    n, p = 300, 10
    A, B = paper_p4_matrices(n, p, rng_for(24, 3))
    obj = oo.QAPObjective(A, B)
    X0 = orthonormal_start(n, p, rng_for(24, 4))
    beta = obj.hess_norm_bound() + 0.1
    ref = op.solve(obj, X0, variant=variant, beta=beta, tol=1e-8, maxit=20000)
    s = _solver(A, B, "fp64", variant=variant, beta=beta, tol=1e-8, maxit=20000, final_orth=1)
    Qd = s.new_matrix(dtype=torch.float64)
    st, info = s.solve(to_dev(X0, s), Qd)
    hist = s.history()
    k = min(20, len(ref.history), len(hist))
    np.testing.assert_allclose(hist[:k, 4], [h.eta for h in ref.history[:k]], rtol=1e-9)
    np.testing.assert_allclose(hist[:k, 2], [h.kkt for h in ref.history[:k]], rtol=1e-8)
    assert st == 0 and ref.converged
    assert abs(info.iters - ref.iters) <= max(5, 0.25 * ref.iters)
    assert abs(obj.value(to_host(Qd, n)) - ref.f_orth) <= 1e-9 * abs(ref.f_orth)
    s.close()
