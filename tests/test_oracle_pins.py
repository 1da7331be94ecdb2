"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each expected value comes from a
closed form, a brute-force dense eigensolve, a hand computation, a finite
difference, or an inequality the paper proves (Lemma 2).  Together they are
chosen so that a dropped term, a wrong sign or index, or a transposed operand
in the oracle fails at least one of them (tests/test_oracle_mutations.py plants
such mistakes and checks that they are caught).
"""
import math

import numpy as np
import pytest

from oracle import kernels as ok
from oracle import objectives as oo
from oracle import plam as op
from workloads import (gaussian_symmetric, orthonormal_start, paper_p2_linear, paper_p3_operator,
                       parameter_study_problems, rng_for, workload_dense_trace)

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---------------------------------------------------------------- trace problem


@pytest.fixture(scope="module")
def c1():
    w = workload_dense_trace(500, 20)
    obj = oo.TraceObjective(w.A)
    evals, evecs = np.linalg.eigh(w.A)   # brute-force dense eigensolve (LAPACK syevd)
    sol = {v: op.solve(obj, w.X0, variant=v, beta=1.0, tol=1e-8, maxit=3000) for v in ("plam", "pcal")}
    return w, obj, evals, evecs, sol


@pytest.mark.parametrize("variant", ["plam", "pcal"])
def test_trace_objective_equals_eigen_sum(c1, variant):
    """Problem 3: min 1/2 tr(X^T A X) over the Stiefel manifold = 1/2 sum of the p smallest eigenvalues."""
    w, obj, evals, _, sol = c1
    r = sol[variant]
    assert r.converged and r.kkt_stop < 1e-8
    fstar = 0.5 * evals[: w.p].sum()
    assert abs(r.f_orth - fstar) <= 1e-10 * abs(fstar)
    # 2f = tr(X^T A X) = sum lambda_i, also before the final orthonormalisation to KKT accuracy
    assert abs(r.f_stop - fstar) <= 1e-7 * abs(fstar)


@pytest.mark.parametrize("variant", ["plam", "pcal"])
def test_trace_multiplier_spectrum_and_subspace(c1, variant):
    """At a KKT point Lambda = X^T A X has the p smallest eigenvalues of A; span(X) is their eigenspace."""
    w, obj, evals, evecs, sol = c1
    r = sol[variant]
    Xo = r.X_orth
    Lam = op.psi(Xo.T @ (w.A @ Xo))
    lam_x = np.linalg.eigvalsh(Lam)
    np.testing.assert_allclose(lam_x, evals[: w.p], rtol=0, atol=1e-7 * abs(evals).max())
    # principal angles between span(X) and the exact eigenspace (Davis-Kahan: sin <= ||KKT|| / gap)
    U = evecs[:, : w.p]
    sin_max = np.linalg.norm(Xo - U @ (U.T @ Xo), 2)   # ||(I - U U^T) X||_2 = sin of the largest angle
    gap = evals[w.p] - evals[w.p - 1]
    kkt_abs = r.kkt_orth * r.K0
    assert sin_max <= 2 * kkt_abs / gap + 1e-12


@pytest.mark.parametrize("variant", ["plam", "pcal"])
def test_unsymmetrised_multiplier_is_symmetric_at_stationarity(variant):
    """Section 2.2, eq. (closed-multi): Lambda = grad f^T X at a stationary point, so the unsymmetrised
    X^T grad f becomes symmetric.  Problem 2 (quadratic + linear term) is used because there X^T grad f
    is not symmetric away from stationarity (for pure trace objectives it always is)."""
    n, p = 100, 5
    A, _ = paper_p3_operator(n, rng_for(6, 0), theta=1.01, xi=1.0)
    Gl = paper_p2_linear(n, p, rng_for(6, 2))
    obj = oo.QuadLinearObjective(A, Gl)
    X0 = orthonormal_start(n, p, rng_for(6, 1))
    C0 = X0.T @ obj.grad(X0)
    assert np.linalg.norm(C0 - C0.T) / np.linalg.norm(C0) > 1e-2
    r = op.solve(obj, X0, variant=variant, beta=3.0, tol=1e-10, maxit=20000)
    assert r.converged
    C = r.C_last
    assert np.linalg.norm(C - C.T) / np.linalg.norm(C) < 1e-8


@pytest.mark.parametrize("variant", ["plam", "pcal"])
def test_final_orthonormalisation(c1, variant):
    """Section 5.3, Table 'orth step': the post-process drives feasibility to ~1e-14 and leaves KKT unchanged."""
    _, obj, _, _, sol = c1
    r = sol[variant]
    assert r.feas_orth <= 1e-12
    assert r.feas_stop > r.feas_orth
    assert r.kkt_orth <= 1.2 * r.kkt_stop + 1e-12
    assert r.kkt_orth >= 0.5 * r.kkt_stop
    lam_norm = np.linalg.norm(r.Lambda)
    assert abs(r.f_orth - r.f_stop) <= lam_norm * r.feas_stop + r.K0 * r.kkt_stop


def test_pcal_iterates_have_unit_columns(c1):
    """Algorithm 3: every PCAL iterate has unit-norm columns (the redundant sphere constraints)."""
    w, obj, _, _, _ = c1
    norms = []

    def cb(k, X, G, R, eta):
        norms.append(np.abs(np.linalg.norm(X, axis=0) - 1.0).max())

    op.solve(obj, w.X0, variant="pcal", beta=1.0, tol=1e-6, maxit=50, callback=cb)
    assert len(norms) > 10
    assert max(norms[1:]) < 1e-13


def test_kkt_forms_agree_at_solution(c1):
    """eq. (kkt) and eq. (kkt2) both vanish at the solution; Psi form of Section 3.3 is close to eq. (kkt2)."""
    w, obj, _, _, sol = c1
    X = sol["pcal"].X_orth
    G = obj.grad(X)
    r_full = np.linalg.norm(G - X @ (G.T @ X))
    r_psi = np.linalg.norm(op.kkt_residual(G, X))
    assert r_full / sol["pcal"].K0 < 1e-7
    assert abs(r_full - r_psi) <= 1e-7 * sol["pcal"].K0


def test_paper_p3_generator_closed_form():
    """Problem 2/3 generator with xi = 1: spectrum exactly {theta^(1-i)}, so
    min 1/2 tr(X^T A X) = 1/2 sum_{i=n-p+1}^{n} theta^(1-i)."""
    n, p, theta = 120, 6, 1.01
    A, lam = paper_p3_operator(n, rng_for(7, 0), theta=theta, xi=1.0)
    ev = np.sort(np.linalg.eigvalsh(A))
    np.testing.assert_allclose(ev, np.sort(theta ** (1.0 - np.arange(1, n + 1))), rtol=1e-12)
    X0 = orthonormal_start(n, p, rng_for(7, 1))
    r = op.solve(oo.TraceObjective(A), X0, variant="pcal", beta=1.0, tol=1e-10, maxit=20000)
    fstar = 0.5 * sum(theta ** (1.0 - i) for i in range(n - p + 1, n + 1))
    assert r.converged
    assert abs(r.f_orth - fstar) <= 1e-9 * fstar


# ---------------------------------------------------------------- Hartree problem


def _green(n):
    """Closed-form inverse of tridiag(-1,2,-1) (Dirichlet): min(i,j)(n+1-max(i,j))/(n+1), 1-based."""
    i = np.arange(1, n + 1)
    return np.minimum.outer(i, i) * (n + 1 - np.maximum.outer(i, i)) / (n + 1.0)


def test_hartree_inverse_laplacian():
    obj2 = oo.HartreeObjective(2)
    # hand value: L = [[2,-1],[-1,2]], L^{-1} = (1/3)[[2,1],[1,2]]
    np.testing.assert_allclose(obj2.hartree_potential(np.array([1.0, 0.0])), [2 / 3, 1 / 3], rtol=1e-15)
    np.testing.assert_allclose(obj2.hartree_potential(np.array([0.0, 1.0])), [1 / 3, 2 / 3], rtol=1e-15)
    n = 300
    obj = oo.HartreeObjective(n)
    rho = np.random.default_rng(3).random(n)
    np.testing.assert_allclose(obj.hartree_potential(rho), _green(n) @ rho, rtol=1e-12)


def test_hartree_energy_hand_value():
    """X = [e_1 .. e_p]: tr(X^T L X) = 2p and rho^T L^{-1} rho = sum_{i,j<=p} min(i,j)(n+1-max(i,j))/(n+1)."""
    n, p, alpha, q = 40, 5, 1.3, 0.25
    X = np.zeros((n, p))
    X[np.arange(p), np.arange(p)] = 1.0
    h = 0.0
    for i in range(1, p + 1):
        for j in range(1, p + 1):
            h += min(i, j) * (n + 1 - max(i, j)) / (n + 1)
    expect = q * 2 * p + 0.25 * alpha * h
    assert abs(oo.HartreeObjective(n, alpha, q).value(X) - expect) <= 1e-13 * expect


def test_hartree_alpha0_reduces_to_laplacian_eigenproblem():
    """alpha = 0: min q tr(X^T L X) = q sum_{k<=p} (2 - 2 cos(k pi/(n+1)))."""
    n, p, q = 80, 4, 0.25
    obj = oo.HartreeObjective(n, alpha=0.0, quad_scale=q)
    X0 = orthonormal_start(n, p, rng_for(8, 1))
    r = op.solve(obj, X0, variant="pcal", beta=1.0, tol=1e-10, maxit=20000)
    fstar = q * sum(2 - 2 * math.cos(k * math.pi / (n + 1)) for k in range(1, p + 1))
    assert r.converged
    assert abs(r.f_orth - fstar) <= 1e-9 * fstar


def test_block_laplacian_spectrum_and_inverse():
    """Section 5.4's block-diagonal L (blocks of b rows, a ragged last block): the matrix that
    laplacian_1d_apply assembles column by column has the union of the blocks' Dirichlet spectra
    {2 - 2 cos(k pi/(m+1)) : k <= m} and no coupling across block edges, and the banded solve
    L^{-1} rho equals the blocks' closed-form Green's functions min(u,v)(m+1-max(u,v))/(m+1)
    (the b = 2 block is (1/3)[[2,1],[1,2]])."""
    n, b = 23, 5
    Ld = oo.laplacian_1d_apply(np.eye(n), b)
    sizes = [b] * (n // b) + ([n % b] if n % b else [])
    ev = sorted(2 - 2 * math.cos(k * math.pi / (m + 1)) for m in sizes for k in range(1, m + 1))
    np.testing.assert_allclose(np.linalg.eigvalsh(Ld), ev, atol=1e-13)
    for e in range(b, n, b):                 # rows e-1 and e sit in different blocks
        assert Ld[e - 1, e] == 0.0 and Ld[e, e - 1] == 0.0
    obj = oo.HartreeObjective(n, block=b)
    rho = np.random.default_rng(4).random(n)
    y = obj.hartree_potential(rho)
    start = 0
    for m in sizes:
        np.testing.assert_allclose(y[start:start + m], _green(m) @ rho[start:start + m], rtol=1e-13)
        start += m
    y2 = oo.HartreeObjective(6, block=2).hartree_potential(np.array([1.0, 0.0, 0.0, 3.0, 0.0, 0.0]))
    np.testing.assert_allclose(y2, [2 / 3, 1 / 3, 1.0, 2.0, 0.0, 0.0], rtol=1e-15)


def test_block_hartree_linear_energy_hand_value():
    """X = [e_1 .. e_p] with blocks of b rows and a linear term: tr(X^T L X) = 2p, rho is the
    indicator of the first p rows, so rho^T L^{-1} rho adds the Green's function entries of the
    pairs of those rows inside one block, and tr(G_lin^T X) = sum_i G_lin[i, i]."""
    n, p, b, alpha, q = 30, 7, 4, 1.1, 0.5
    lin = np.random.default_rng(9).standard_normal((n, p))
    X = np.zeros((n, p))
    X[np.arange(p), np.arange(p)] = 1.0
    h = 0.0
    for i in range(p):
        for j in range(p):
            if i // b == j // b:
                u, v = i % b + 1, j % b + 1
                h += min(u, v) * (b + 1 - max(u, v)) / (b + 1)
    expect = q * 2 * p + 0.25 * alpha * h + float(np.trace(lin[:p, :]))
    got = oo.HartreeObjective(n, alpha, q, block=b, lin=lin).value(X)
    assert abs(got - expect) <= 1e-13 * abs(expect)


def test_block_laplacian_trace_problem_reaches_ky_fan():
    """alpha = 0 with blocks of 5 rows: min q tr(X^T L X) = q times the sum of the p smallest
    eigenvalues of the union of the blocks' spectra (the Section 5.4 Problem 1 operator)."""
    n, p, b, q = 60, 6, 5, 0.5
    obj = oo.HartreeObjective(n, alpha=0.0, quad_scale=q, block=b)
    X0 = orthonormal_start(n, p, rng_for(19, 1))
    r = op.solve(obj, X0, variant="pcal", beta=2.1, tol=1e-10, maxit=20000)
    ev = sorted(2 - 2 * math.cos(k * math.pi / (b + 1)) for _ in range(n // b) for k in range(1, b + 1))
    fstar = q * sum(ev[:p])
    assert r.converged
    assert abs(r.f_orth - fstar) <= 1e-9 * fstar


def test_problem4_special_cases():
    """Problem 4 (Section 5.2, eq. QAP): with B = I it is Problem 3 (the same value and gradient as
    f = 1/2 tr(X^T A X)); with B = diag(3, 2, 1) its minimum over X^T X = I is
    1/2 sum_i b_i lambda_i(A), the largest b_i paired with the smallest eigenvalues of A (the
    rearrangement behind Ky Fan's principle), which the oracle's PCAL reaches."""
    n, p = 40, 3
    A = gaussian_symmetric(n, rng_for(23, 0))
    X = np.random.default_rng(2).standard_normal((n, p))
    q, t = oo.QAPObjective(A, np.eye(p)), oo.TraceObjective(A)
    assert abs(q.value(X) - t.value(X)) <= 1e-12 * abs(t.value(X))
    np.testing.assert_allclose(q.grad(X), t.grad(X), rtol=1e-13, atol=1e-13)
    b = np.array([3.0, 2.0, 1.0])
    obj = oo.QAPObjective(A, np.diag(b))
    lam = np.linalg.eigvalsh(A)
    fstar = 0.5 * float(b @ lam[:p])
    r = op.solve(obj, orthonormal_start(n, p, rng_for(23, 1)), variant="pcal",
                 beta=obj.hess_norm_bound() + 0.1, tol=1e-10, maxit=20000)
    assert r.converged
    assert abs(r.f_orth - fstar) <= 1e-10 * abs(fstar)


def _fd_check(obj, X, seed=0, h=1e-6):
    E = np.random.default_rng(seed).standard_normal(X.shape)
    fd = (obj.value(X + h * E) - obj.value(X - h * E)) / (2 * h)
    an = float(np.sum(obj.grad(X) * E))
    return fd, an


@pytest.mark.parametrize("kind", ["dense", "hartree", "stencil", "quadlin", "dense_hartree",
                                  "block_hartree_lin_xc", "qap"])
def test_gradient_finite_difference(kind):
    """Central differences <grad f, E> = (f(X+hE) - f(X-hE)) / 2h for every oracle objective."""
    rng = np.random.default_rng(11)
    if kind == "dense":
        n = 60
        obj = oo.TraceObjective(gaussian_symmetric(n, rng))
    elif kind == "hartree":
        n = 70
        obj = oo.HartreeObjective(n, alpha=1.0, quad_scale=0.25)
    elif kind == "stencil":
        m = 4
        n = m ** 3
        obj = oo.Stencil3DObjective(m, rng.random(n))
    elif kind == "block_hartree_lin_xc":
        n = 63
        obj = oo.HartreeObjective(n, alpha=1.3, quad_scale=0.5, xc=0.7, block=5,
                                  lin=rng.standard_normal((n, 5)))
    elif kind == "qap":
        n = 45
        B0 = rng.standard_normal((5, 5))
        obj = oo.QAPObjective(gaussian_symmetric(n, rng), 0.5 * (B0 + B0.T))
    elif kind == "quadlin":
        n = 50
        obj = oo.QuadLinearObjective(gaussian_symmetric(n, rng), rng.standard_normal((n, 5)))
    else:
        n = 40
        obj = oo.DenseHartreeObjective(gaussian_symmetric(n, rng), alpha=1.0, quad_scale=0.5)
    X = rng.standard_normal((n, 5))
    fd, an = _fd_check(obj, X)
    assert abs(fd - an) <= 1e-7 * max(1.0, abs(an))


# ---------------------------------------------------------------- 3D stencil


def test_stencil3d_operator_brute_force():
    """L3 + V against a dense matrix assembled point by point from the 7-point rule (m = 3)."""
    _stencil_brute_force((3, 3, 3))


def test_stencil3d_operator_brute_force_non_cubic():
    """The same on a slab whose three axes all differ (2 x 3 x 4), as the oracle's timed sample
    of the 128^3 workload (its first z-planes) uses."""
    _stencil_brute_force((2, 3, 4))


def _stencil_brute_force(grid):
    nx, ny, nz = grid
    n = nx * ny * nz
    V = np.random.default_rng(5).random(n)
    H = np.zeros((n, n))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = x + nx * y + nx * ny * z
                H[i, i] = 6.0 + V[i]
                for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    xx, yy, zz = x + dx, y + dy, z + dz
                    if 0 <= xx < nx and 0 <= yy < ny and 0 <= zz < nz:
                        H[i, xx + nx * yy + nx * ny * zz] = -1.0
    obj = oo.Stencil3DObjective(nx if nx == ny == nz else grid, V)
    X = np.random.default_rng(6).standard_normal((n, 3))
    np.testing.assert_allclose(obj.grad(X), H @ X, rtol=1e-14, atol=1e-14)


def test_stencil3d_constant_potential_closed_form():
    """V = c: eigenvalues sum_{t in (a,b,c)} (2 - 2 cos(pi t/(m+1))) + c; p = 4 sits at a spectral gap.
    beta = s + 0.1 with s = 12 + c >= ||grad^2 f(0)||_2 (the parameter-study setting of Section 5.3)."""
    m, p, c = 6, 4, 0.37
    obj = oo.Stencil3DObjective(m, np.full(m ** 3, c))
    one = [2 - 2 * math.cos(math.pi * t / (m + 1)) for t in range(1, m + 1)]
    ev = sorted(one[a] + one[b] + one[d] + c for a in range(m) for b in range(m) for d in range(m))
    assert ev[p] - ev[p - 1] > 0.1
    X0 = orthonormal_start(m ** 3, p, rng_for(9, 1))
    r = op.solve(obj, X0, variant="pcal", beta=obj.hess_norm_bound() + 0.1, tol=1e-10, maxit=20000)
    fstar = 0.5 * sum(ev[:p])
    assert r.converged
    assert abs(r.f_orth - fstar) <= 1e-9 * fstar


# ---------------------------------------------------------------- Lemma 2 and single steps


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lemma2_feasibility_bound(seed):
    """Lemma 2: beta > (||grad f||_2 ||X||_2 + delta) / sigma_min(X)^2 implies
    ||X^T X - I||_F <= ||X||_2 / delta * ||grad_X L_beta(X, Psi(grad f^T X))||_F."""
    rng = np.random.default_rng(seed)
    n, p = 80, 6
    obj = oo.TraceObjective(gaussian_symmetric(n, rng))
    X = orthonormal_start(n, p, rng) + 0.05 * rng.standard_normal((n, p))
    G = obj.grad(X)
    sv = np.linalg.svd(X, compute_uv=False)
    # a delta large against ||grad f||_2 ||X||_2 makes the bound nearly tight, so it pins the penalty term
    delta = 50.0 * np.linalg.norm(G, 2) * sv[0]
    beta = 1.001 * (np.linalg.norm(G, 2) * sv[0] + delta) / sv[-1] ** 2
    B = X.T @ X
    R = op.lagrangian_grad(G, X, B, op.multiplier_lambda1(G, X), beta)
    lhs = np.linalg.norm(B - np.eye(p))
    rhs = sv[0] / delta * np.linalg.norm(R)
    assert lhs <= rhs
    assert lhs > 0.4 * rhs   # the bound is not vacuous here (ratio ~ sigma_min^2/sigma_max^2)


def test_single_step_matches_definitions():
    """One PLAM and one PCAL step agree with the closed forms (eq. PLAM-main, Algorithm 3's column formula)."""
    rng = np.random.default_rng(21)
    n, p, beta = 40, 3, 2.5
    obj = oo.TraceObjective(gaussian_symmetric(n, rng))
    X0 = orthonormal_start(n, p, rng) + 0.01 * rng.standard_normal((n, p))
    G = obj.grad(X0)
    steps = {}

    def cb(k, X, Gk, R, eta):
        steps[k] = (R.copy(), eta)

    for variant, rule in (("plam", "lambda1"), ("pcal", "lambda2"), ("pcal", "lambda1")):
        steps.clear()
        r = op.solve(obj, X0, variant=variant, beta=beta, lambda_rule=rule, tol=0.0, maxit=1,
                     record=False, callback=cb)
        R, eta = steps[0]
        # eq. (PLAM-main) written out: G - X Psi(G^T X) + beta X (X^T X - I)
        Lam = 0.5 * (G.T @ X0 + X0.T @ G)
        if variant == "pcal" and rule == "lambda2":
            R0 = G - X0 @ Lam + beta * X0 @ (X0.T @ X0 - np.eye(p))
            Lam = Lam + np.diag(np.einsum("ij,ij->j", X0, R0))
        Rexp = G - X0 @ Lam + beta * X0 @ (X0.T @ X0 - np.eye(p))
        np.testing.assert_allclose(R, Rexp, rtol=1e-13, atol=1e-13)
        V = X0 - Rexp / eta
        Xexp = V if variant == "plam" else V / np.sqrt(np.einsum("ij,ij->j", V, V))
        np.testing.assert_allclose(r.X, Xexp, rtol=1e-13, atol=1e-13)
        assert abs(eta - (np.linalg.norm(G) / np.linalg.norm(X0) + beta)) <= 1e-13 * eta


def test_lambda2_diagonal_is_sphere_multiplier():
    """eq. (kkt3): at a point where every column is a unit eigenvector, R0 = 0 and the lambda2 correction vanishes;
    for a radial perturbation the correction equals the radial component."""
    rng = np.random.default_rng(4)
    n, p = 30, 3
    A = gaussian_symmetric(n, rng)
    ev, U = np.linalg.eigh(A)
    X = U[:, :p].copy()
    obj = oo.TraceObjective(A)
    G = obj.grad(X)
    L0, d, Lam, M = ok.multiplier(X, G, beta=1.0)
    np.testing.assert_allclose(d, 0, atol=1e-12)
    np.testing.assert_allclose(np.diag(Lam), ev[:p], rtol=1e-12)
    # scale column 0 by s: X^T grad_X L(X, Psi) picks up the radial derivative of the penalty
    s = 1.1
    Xs = X.copy()
    Xs[:, 0] *= s
    Gs = obj.grad(Xs)
    _, d2, _, _ = ok.multiplier(Xs, Gs, beta=1.0)
    # column 0: grad = lam s u, Psi entry lam s^2, R0_0 = lam s u - lam s^3 u + beta s u (s^2 - 1)
    lam0 = ev[0]
    expect = s * (lam0 * s - lam0 * s ** 3 + 1.0 * s * (s * s - 1))
    assert abs(d2[0] - expect) <= 1e-12 * max(1.0, abs(expect))
    np.testing.assert_allclose(d2[1:], 0, atol=1e-12)


def test_flop_table():
    """Table 'cost' per-iteration totals: PLAM and PCAL 7np^2 + O(np): X^T X (np^2), grad f^T X (2np^2),
    X(X^T X - I) and X Psi(.) (2np^2 each)."""
    from paper_1810_03930_gb300.flops import iteration_flops
    n, p = 10000, 1000
    f = iteration_flops(n, p)
    assert f["gram_xx"] == n * p * p
    assert f["gram_xg"] == 2 * n * p * p
    assert f["update"] == 2 * n * p * p
    assert f["kkt_product"] == 2 * n * p * p
    assert f["total"] == 7 * n * p * p


def _read_orth_table():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "orth_step_table.txt")
    rows = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        solver, stage, f, kkt, feas = line.split()
        rows[(solver, stage)] = (float(f), float(kkt), float(feas))
    return rows


@pytest.mark.parametrize("variant", ["plam", "pcal"])
def test_orth_step_table_pattern(variant):
    """Table 'orth step' (Section 5.3) on a synthetic Problem 1 of the same size: the paper's printed
    pattern (f unchanged to ~1e-10 relative, KKT unchanged to two digits, feasibility to ~1e-14)."""
    table = _read_orth_table()
    f_s, k_s, x_s = table[(variant.upper(), "stop")]
    f_o, k_o, x_o = table[(variant.upper(), "orth")]
    assert abs(f_o - f_s) / abs(f_s) < 1e-9 and x_o < 1e-13 and abs(k_o - k_s) <= 0.01 * k_s
    n, p = 1000, 20
    L = gaussian_symmetric(n, rng_for(11, 0))
    obj = oo.DenseHartreeObjective(L, alpha=1.0, quad_scale=0.5)
    X0 = orthonormal_start(n, p, rng_for(11, 1))
    beta = obj.hess_norm_bound() if variant == "plam" else 1.0   # Section 5.1 defaults
    r = op.solve(obj, X0, variant=variant, beta=beta, tol=1e-5, maxit=3000)
    assert r.converged
    assert r.feas_orth < 1e-13
    assert abs(r.f_orth - r.f_stop) / abs(r.f_stop) < 1e-7
    assert abs(r.kkt_orth - r.kkt_stop) <= 0.05 * r.kkt_stop


def test_trace_min_optimum_against_dense_eigensolve_and_closed_form():
    """oracle.objectives.trace_min_optimum (shift-invert Lanczos) against (i) a dense LAPACK
    eigensolve of a random-potential 3D stencil and (ii) the closed-form spectrum of the
    constant-potential Dirichlet Laplacian, 2 - 2 cos(pi t / (m + 1)) summed over three axes."""
    rng = np.random.default_rng(42)
    m, p = 7, 12
    V = rng.uniform(0.0, 1.0, m ** 3)
    H = oo.Stencil3DObjective(m, V).H
    f, ev = oo.trace_min_optimum(H, p)
    ev_dense = np.linalg.eigvalsh(H.toarray())
    np.testing.assert_allclose(ev, ev_dense[:p], rtol=1e-11, atol=1e-11)
    assert abs(f - 0.5 * ev_dense[:p].sum()) <= 1e-11 * abs(f)
    c = 0.3
    one = [2 - 2 * math.cos(math.pi * t / (m + 1)) for t in range(1, m + 1)]
    closed = sorted(one[a] + one[b] + one[d] + c for a in range(m) for b in range(m) for d in range(m))
    f2, _ = oo.trace_min_optimum(oo.Stencil3DObjective(m, np.full(m ** 3, c)).H, p)
    assert abs(f2 - 0.5 * sum(closed[:p])) <= 1e-11 * f2


def test_separable_potential_optimum_against_dense_eigensolve_and_closed_form():
    """oracle.objectives.separable_trace_min_optimum (three tridiagonal eigensolves and the
    Kronecker-sum spectrum) against (i) a dense LAPACK eigensolve of the assembled operator on
    a non-cubic grid, assembled point by point from the generator's V (so a potential laid out
    with another axis fastest, or a dropped axis term, would move the spectrum), and (ii) the
    constant-potential closed form, v_k = c / 3."""
    from workloads import separable_potential
    rng = np.random.default_rng(11)
    nx, ny, nz, p = 7, 5, 6, 17
    V, vx, vy, vz = separable_potential(nx, ny, nz, rng)
    import scipy.sparse as sp

    def second_difference(m):
        return sp.diags([-np.ones(m - 1), 2 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1])

    Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    # point by point: index x + nx (y + ny z), x fastest
    H = (sp.kron(Iz, sp.kron(Iy, second_difference(nx))) +
         sp.kron(Iz, sp.kron(second_difference(ny), Ix)) +
         sp.kron(second_difference(nz), sp.kron(Iy, Ix)) + sp.diags(V)).toarray()
    for z, y, x in ((0, 0, 1), (3, 2, 6), (5, 4, 0)):
        assert abs(V[x + nx * (y + ny * z)] - (vx[x] + vy[y] + vz[z])) <= 1e-15
    ev_dense = np.linalg.eigvalsh(H)
    f, ev = oo.separable_trace_min_optimum(vx, vy, vz, p)
    np.testing.assert_allclose(ev, ev_dense[:p + 1], rtol=1e-13, atol=1e-13)
    assert abs(f - 0.5 * ev_dense[:p].sum()) <= 1e-13 * abs(f)
    m, c = 9, 0.45
    one = [2 - 2 * math.cos(math.pi * t / (m + 1)) for t in range(1, m + 1)]
    closed = sorted(one[a] + one[b] + one[d] + c for a in range(m) for b in range(m) for d in range(m))
    f3, ev3 = oo.separable_trace_min_optimum(*(np.full(m, c / 3.0),) * 3, 30)
    assert abs(f3 - 0.5 * sum(closed[:30])) <= 1e-13 * f3
    np.testing.assert_allclose(ev3, closed[:31], rtol=1e-13)


@pytest.mark.parametrize("variant", ["plam", "pcal"])
def test_dual_ascent_variants(variant):
    """PLAM-DA / PCAL-DA (Section 5.3): the first step equals the closed-form method's first step
    (Lambda^0 = Psi(G^0^T X^0)); the multiplier then follows Lambda^k = Lambda^{k-1} - beta
    (X^k^T X^k - I) exactly; and PCAL-DA still reaches the trace problem's optimum
    1/2 sum of the p smallest eigenvalues."""
    rng = np.random.default_rng(8)
    n, p, beta = 120, 4, 1.0
    A = gaussian_symmetric(n, rng)
    X0 = orthonormal_start(n, p, rng)
    obj = oo.TraceObjective(A)
    a = op.solve(obj, X0, variant=variant, beta=beta, lambda_rule="da", tol=0.0, maxit=1)
    b = op.solve(obj, X0, variant=variant, beta=beta, lambda_rule="lambda1", tol=0.0, maxit=1)
    assert np.array_equal(a.X, b.X)
    seen = []

    def grab(k, X, G, R, eta):
        B = X.T @ X
        # R = G - X Lambda + beta X (B - I)  =>  X^T (G - R) + beta B (B - I) = B Lambda
        seen.append(np.linalg.solve(B, X.T @ (G - R) + beta * B @ (B - np.eye(p))))

    op.solve(obj, X0, variant=variant, beta=beta, lambda_rule="da", tol=0.0, maxit=4, callback=grab)
    Xs = []
    op.solve(obj, X0, variant=variant, beta=beta, lambda_rule="da", tol=0.0, maxit=4,
             callback=lambda k, X, G, R, eta: Xs.append(X.copy()))
    for k in range(1, 4):
        Bk = Xs[k].T @ Xs[k]
        np.testing.assert_allclose(seen[k], seen[k - 1] - beta * (Bk - np.eye(p)), atol=1e-9)
    if variant == "pcal":
        # PCAL-DA keeps unit columns and reaches the optimum; PLAM-DA at beta = 1 lets X shrink
        # to zero on this problem (the relative KKT value then vanishes without a solution),
        # in line with the paper's finding that dual ascent is the weaker multiplier update
        r = op.solve(obj, X0, variant=variant, beta=beta, lambda_rule="da", tol=1e-8, maxit=20000,
                     record=False)
        assert r.converged
        ev = np.linalg.eigvalsh(A)
        assert abs(r.f_orth - 0.5 * ev[:p].sum()) <= 1e-9 * abs(0.5 * ev[:p].sum())


def test_exchange_term_pins():
    """Problem 6's exchange term -(3 gamma/4) sum rho^{4/3} (Section 5.2): (i) with gamma = 0 the
    objective is the Hartree one exactly; (ii) hand value on X = [e_1 .. e_p] placed on distinct
    rows (rho = their indicator, so sum rho^{4/3} = p); (iii) the gradient -2 gamma rho^{1/3} X
    against central differences."""
    n, p = 40, 3
    gamma = 2.0 * (3.0 / math.pi) ** (1.0 / 3.0)
    rng = np.random.default_rng(12)
    X = rng.standard_normal((n, p)) / math.sqrt(n)
    h0 = oo.HartreeObjective(n, 2.0, 0.5)
    h1 = oo.HartreeObjective(n, 2.0, 0.5, xc=0.0)
    assert h1.value(X) == h0.value(X) and np.array_equal(h1.grad(X), h0.grad(X))
    rows = [3, 17, 30]
    E = np.zeros((n, p))
    for c, r in enumerate(rows):
        E[r, c] = 1.0
    hx = oo.HartreeObjective(n, 2.0, 0.5, xc=gamma)
    # L^{-1} by the Dirichlet Green's function min(i,j)(n+1-max(i,j))/(n+1), 1-based
    ginv = lambda i, j: min(i, j) * (n + 1 - max(i, j)) / (n + 1)
    rr = [r + 1 for r in rows]
    hartree = sum(ginv(i, j) for i in rr for j in rr)
    expect = 0.5 * 2.0 * p + 0.25 * 2.0 * hartree - 0.75 * gamma * p
    assert abs(hx.value(E) - expect) <= 1e-12 * abs(expect)
    D = rng.standard_normal((n, p))
    hstep = 1e-5
    dd = (hx.value(X + hstep * D) - hx.value(X - hstep * D)) / (2 * hstep)
    assert abs(dd - np.sum(hx.grad(X) * D)) <= 1e-7 * max(1.0, abs(dd))


def parameter_study_set():
    """The seeded parameter-study problems and s = the largest ||A||_2 of the set (the Hessian
    norm at 0 of the trace objective)."""
    As, X0s = parameter_study_problems()
    s = max(float(np.max(np.abs(np.linalg.eigvalsh(A)))) for A in As)
    return As, X0s, s


@pytest.mark.parametrize("variant", ["plam", "pcal"])
def test_parameter_study_conclusions_on_trace_problems(variant):
    """Section 5.1's parameter study (Figs. 'eta' and 'beta'), qualitatively, on 12 seeded trace
    problems (n = 200, p = 8, relative KKT 1e-6): with beta = s + 0.1 the alternating BB step
    needs the fewest iterations (median) of ABB, BB1, BB2 and the differential rule, and the
    constant step reaches the tolerance on none within 3000 iterations; a large penalty
    (beta = 10 s + 1) is slower than beta = s + 0.1.  (The paper's divergence of PLAM with a small
    beta shows on its nonlinear problems, not on these.)"""
    As, X0s, s = parameter_study_set()

    def median_iters(beta, rule):
        rs = [op.solve(oo.TraceObjective(A), X0, variant=variant, beta=beta, eta_rule=rule,
                       tol=1e-6, maxit=3000, record=False) for A, X0 in zip(As, X0s)]
        return float(np.median([r.iters for r in rs])), sum(not r.converged for r in rs)

    med = {rule: median_iters(s + 0.1, rule) for rule in ("abb", "bb1", "bb2", "diff", "const")}
    for rule in ("abb", "bb1", "bb2", "diff"):
        assert med[rule][1] == 0, (rule, med[rule])
        if rule != "abb":
            assert med["abb"][0] < med[rule][0], med
    assert med["const"][1] == len(As)
    slow, _ = median_iters(10 * s + 1, "abb")
    assert slow > 1.3 * med["abb"][0]


@pytest.mark.parametrize("variant", ["plam", "pcal"])
def test_parameter_study_conclusion_on_problem4(variant):
    """Section 5.1's step-size study (Fig. "eta") on Problem 4 (8 seeded instances, n = 200,
    p = 8, A and B symmetrised Gaussians, beta = s + 0.1 with s = ||A|| ||B||, relative KKT
    1e-6): ABB converges on every instance with the smallest median iteration count, ahead of
    BB1 and BB2, and the constant step reaches the tolerance within 3000 iterations on none of
    the instances it is run on."""
    from workloads import paper_p4_matrices
    its = {"abb": [], "bb1": [], "bb2": [], "const": []}
    conv_abb = 0
    for i in range(8):
        A, B = paper_p4_matrices(200, 8, rng_for(22, 0, sub=i))
        X0 = orthonormal_start(200, 8, rng_for(22, 1, sub=i))
        obj = oo.QAPObjective(A, B)
        beta = obj.hess_norm_bound() + 0.1
        for rule in ("abb", "bb1", "bb2") + (("const",) if i < 2 else ()):
            r = op.solve(obj, X0, variant=variant, beta=beta, eta_rule=rule, tol=1e-6, maxit=3000,
                         record=False)
            its[rule].append(r.iters if r.converged else 3000)
            conv_abb += int(rule == "abb" and r.converged)
    assert conv_abb == 8
    assert np.median(its["abb"]) < np.median(its["bb1"]) and np.median(its["abb"]) < np.median(its["bb2"])
    assert all(k == 3000 for k in its["const"])


@pytest.mark.parametrize("variant", ["plam", "pcal"])
def test_feasibility_follows_kkt_on_problem1(variant):
    """Section 5.3 (Fig. "feasibility", Lemma 2): on Problem 1 the feasibility violation
    ||X^T X - I||_F decays nonmonotonically with the same tendency as the KKT violation.  From the
    orthonormal start it first rises, then falls with the KKT value: over the run the two logs
    correlate above 0.85 (0.91-0.94 on these instances), and it rises at many iterations."""
    from workloads import multiplier_study_problems
    p1, _ = multiplier_study_problems(count=3)
    for L, X0 in p1:
        obj = oo.DenseHartreeObjective(L, alpha=1.0, quad_scale=0.5)
        r = op.solve(obj, X0, variant=variant, beta=obj.hess_norm_bound() + 0.1, tol=1e-8,
                     maxit=3000)
        assert r.converged
        feas = np.array([h.feas for h in r.history[1:]])
        kkt = np.array([h.kkt for h in r.history[1:]])
        assert np.corrcoef(np.log10(feas), np.log10(kkt))[0, 1] > 0.85
        assert np.sum(np.diff(feas) > 0) >= 10
        assert feas[-1] < 1e-7 < feas.max()


def test_multiplier_study_conclusion_on_problems_1_and_2():
    """Section 5.3 (Fig. "PCAL_multiplier"), qualitatively: the closed-form multiplier update of
    PLAM (eq. Lambda1) and PCAL (eq. lambda2) against dual ascent (PLAM-DA / PCAL-DA, the ALM
    multiplier step of Algorithm 1) on 6 seeded instances each of Problem 1 (dense Gaussian L,
    alpha = 1) and Problem 2 (the Gao et al. generator, default parameters), n = 200, p = 8,
    beta = s + 0.1, relative KKT 1e-6, ABB.  The closed form converges on every instance and
    its median iteration count is well below dual ascent's (which misses 3000 iterations on
    some instances)."""
    from workloads import multiplier_study_problems
    p1, p2 = multiplier_study_problems()
    cases = []
    for L, X0 in p1:
        obj = oo.DenseHartreeObjective(L, alpha=1.0, quad_scale=0.5)
        cases.append(("P1", obj, obj.hess_norm_bound(), X0))
    for A, lam, Gl, X0 in p2:
        cases.append(("P2", oo.QuadLinearObjective(A, Gl), float(np.max(np.abs(lam))), X0))
    for prob in ("P1", "P2"):
        for variant, closed in (("plam", "lambda1"), ("pcal", "lambda2")):
            its = {}
            for rule in (closed, "da"):
                rs = [op.solve(obj, X0, variant=variant, beta=s + 0.1, lambda_rule=rule, tol=1e-6,
                               maxit=3000, record=False)
                      for name, obj, s, X0 in cases if name == prob]
                its[rule] = [r.iters if r.converged else 3000 for r in rs]
                if rule == closed:
                    assert all(r.converged for r in rs), (prob, variant, its)
            assert np.median(its["da"]) >= 2.5 * np.median(its[closed]), (prob, variant, its)


# ---------------------------------------------------------------- MOptQR (Sections 5.3-5.4)


def test_moptqr_retraction_is_the_qr_factor_and_keeps_feasibility():
    """Table "cost"'s Cholesky retraction V L^{-T} (V^T V = L L^T) is the Q factor of V with a
    positive diagonal of R (Householder QR, a different algorithm); the projected gradient
    D = G - X G^T X is tangent (X^T D skew-symmetric) at a feasible X; and every MOptQR iterate
    stays feasible to rounding."""
    from oracle import moptqr as om
    w = workload_dense_trace(200, 8)
    # Problem 2's linear term makes X^T G unsymmetric, so the skew part of X^T D is not zero
    obj = oo.QuadLinearObjective(w.A, np.random.default_rng(9).standard_normal((200, 8)))
    X = w.X0
    G = obj.grad(X)
    D = om.projected_gradient(G, X)
    S = X.T @ D
    assert np.abs(S).max() > 1e-3 * np.abs(X.T @ G).max()
    assert np.abs(S + S.T).max() <= 1e-13 * np.abs(X.T @ G).max()
    V = X - 0.05 * D
    np.testing.assert_allclose(om.cholesky_retraction(V), op.orthonormalize(V), rtol=0, atol=1e-13)
    r = om.solve(obj, X, tol=1e-10, maxit=20)
    assert all(h.feas <= 1e-13 for h in r.history)


def test_moptqr_converges_to_ky_fan_optimum():
    """Problem 3's generator (dense trace), n = 200, p = 8: MOptQR with ABB steps reaches half
    the sum of the 8 smallest eigenvalues (Ky Fan), like PLAM and PCAL do."""
    from oracle import moptqr as om
    w = workload_dense_trace(200, 8)
    obj = oo.TraceObjective(w.A)
    fstar = 0.5 * np.linalg.eigvalsh(w.A)[:8].sum()
    r = om.solve(obj, w.X0, tol=1e-10, maxit=5000)
    assert r.converged and not r.diverged
    assert abs(r.f_orth - fstar) <= 1e-10 * abs(fstar)
    assert r.feas_orth <= 1e-13


def test_moptqr_first_step_by_hand():
    """One iteration written out: eta^0 = ||G||_F / ||X||_F (no penalty), V = X - D / eta^0,
    X^1 = Q of V; and the second step size is BB1 = |<S,Y>| / <S,S> of S = X^1 - X^0,
    Y = D^1 - D^0 (ABB, odd k)."""
    from oracle import moptqr as om
    w = workload_dense_trace(120, 5)
    obj = oo.TraceObjective(w.A)
    X0 = w.X0
    G0 = obj.grad(X0)
    eta0 = np.linalg.norm(G0) / np.linalg.norm(X0)
    D0 = G0 - X0 @ (G0.T @ X0)
    X1 = op.orthonormalize(X0 - D0 / eta0)
    D1 = obj.grad(X1) - X1 @ (obj.grad(X1).T @ X1)
    S, Y = X1 - X0, D1 - D0
    eta1 = abs(np.sum(S * Y)) / np.sum(S * S)
    r = om.solve(obj, X0, tol=0.0, maxit=2)
    assert abs(r.history[0].eta - eta0) <= 1e-13 * eta0
    assert abs(r.history[1].eta - eta1) <= 1e-11 * eta1



def test_penalty_study_conclusion_on_problems_1_to_4():
    """Section 5.1's penalty study (Figs. "beta", "PCAL_beta_sensitive"), beta in {0, 0.01s, 0.1s,
    s + 0.1, 10s + 1}, ABB, relative KKT 1e-6, 6 seeded instances each of Problems 1 (dense
    Gaussian L, alpha = 1), 2 (Gao et al. generator with a linear term), 3 (dense trace) and 4
    (symmetrised Gaussian A and B), n = 200, p = 8: PLAM with a small penalty diverges on some
    instances (Problem 2 at beta = 0 and 0.01s; Problem 4 at beta = 0), PCAL converges on every
    instance for every beta, and the largest beta is the slowest for both (medians).  Measured
    with this oracle (5 of 6 Problem 2 runs and 2 of 6 Problem 4 runs of PLAM diverge)."""
    from workloads import (multiplier_study_problems, paper_p4_matrices, parameter_study_problems)
    p1, p2 = multiplier_study_problems()
    probs = {"P1": [], "P2": [], "P3": [], "P4": []}
    for L, X0 in p1:
        obj = oo.DenseHartreeObjective(L, alpha=1.0, quad_scale=0.5)
        probs["P1"].append((obj, obj.hess_norm_bound(), X0))
    for A, lam, Gl, X0 in p2:
        probs["P2"].append((oo.QuadLinearObjective(A, Gl), float(np.max(np.abs(lam))), X0))
    As, X0s = parameter_study_problems()
    for A, X0 in zip(As[:6], X0s[:6]):
        probs["P3"].append((oo.TraceObjective(A), float(np.max(np.abs(np.linalg.eigvalsh(A)))), X0))
    for i in range(6):
        A, B = paper_p4_matrices(200, 8, rng_for(22, 0, sub=i))
        obj = oo.QAPObjective(A, B)
        probs["P4"].append((obj, obj.hess_norm_bound(), orthonormal_start(200, 8, rng_for(22, 1, sub=i))))
    betas = {"0": lambda s: 0.0, "0.01s": lambda s: 0.01 * s, "0.1s": lambda s: 0.1 * s,
             "s+0.1": lambda s: s + 0.1, "10s+1": lambda s: 10 * s + 1}

    def run(prob, variant, b):
        rs = [op.solve(obj, X0, variant=variant, beta=betas[b](s), tol=1e-6, maxit=3000,
                       record=False) for obj, s, X0 in probs[prob]]
        return rs

    # PLAM with a small penalty: divergence on some instances
    assert sum(r.diverged for r in run("P2", "plam", "0")) >= 3
    assert sum(r.diverged for r in run("P2", "plam", "0.01s")) >= 3
    assert sum(r.diverged for r in run("P4", "plam", "0")) >= 1
    for prob in ("P1", "P2", "P3", "P4"):
        med = {}
        for b in betas:
            rs = run(prob, "pcal", b)
            assert all(r.converged for r in rs), (prob, b)
            med[b] = np.median([r.iters for r in rs])
        assert med["10s+1"] == max(med.values()), (prob, med)
        rs = run(prob, "plam", "10s+1")
        assert all(r.converged for r in rs)
        assert np.median([r.iters for r in rs]) > np.median([r.iters for r in run(prob, "plam", "s+0.1")])


# ---------------------------------------------------------------- single-step definitions


def _orthonormal_block(n, k, seed):
    """An n x k matrix with orthonormal columns (Householder QR of a seeded Gaussian)."""
    Z = np.random.default_rng(seed).standard_normal((n, k))
    return np.linalg.qr(Z)[0]


def test_update_residual_lies_outside_the_range_of_x():
    """R = G - X M with X orthonormal and M = X^T G (not symmetric) is G's component orthogonal
    to range(X): X^T R = 0 and ||R||^2 = ||G||^2 - ||X^T G||^2 (Pythagoras).  K = G - X Psi(C)
    leaves the skew part: X^T K = (C - C^T)/2.  A transposed M or a sign flip breaks either."""
    X = _orthonormal_block(40, 5, 11)
    G = np.random.default_rng(12).standard_normal((40, 5))
    C = X.T @ G
    assert np.linalg.norm(C - C.T) > 0.5
    R, K = ok.update(X, G, C, 0.5 * (C + C.T))
    assert np.abs(X.T @ R).max() <= 1e-13
    assert math.isclose(np.sum(R * R), np.sum(G * G) - np.sum(C * C), rel_tol=1e-12)
    np.testing.assert_allclose(X.T @ K, 0.5 * (C - C.T), atol=1e-13)


def test_column_dots_of_orthogonal_pieces():
    """X = Q diag(a), R = Q diag(b) + W diag(c) with [Q | W] orthonormal: the column dots are
    a^2, a b and b^2 + c^2 exactly (up to rounding)."""
    Q2 = _orthonormal_block(30, 8, 13)
    Q, W = Q2[:, :4], Q2[:, 4:]
    a = np.array([1.0, 2.0, 0.5, 3.0])
    b = np.array([-1.0, 0.25, 2.0, 0.0])
    c = np.array([0.5, 1.5, 0.0, 2.0])
    xx, xr, rr = ok.column_dots(Q * a, Q * b + W * c)
    np.testing.assert_allclose(xx, a * a, rtol=1e-13)
    np.testing.assert_allclose(xr, a * b, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(rr, b * b + c * c, rtol=1e-13)


def test_bb_dots_along_one_direction():
    """X = X_prev + t D and R = R_prev + c D: <S,S> = t^2 |D|^2, <S,Y> = t c |D|^2,
    <Y,Y> = c^2 |D|^2 with S = X - X_prev, Y = R - R_prev (Section 5.1); a reversed difference
    flips the sign of <S,Y>."""
    rng = np.random.default_rng(14)
    Xp, Rp = rng.standard_normal((25, 3)), rng.standard_normal((25, 3))
    D = _orthonormal_block(25, 3, 15) * np.array([1.0, 2.0, 2.0])      # |D|_F^2 = 9
    t, c = 0.75, -1.5
    ss, sy, yy = ok.bb_dots(Xp + t * D, Rp + c * D, Xp, Rp)
    assert math.isclose(ss, t * t * 9.0, rel_tol=1e-12)
    assert math.isclose(sy, t * c * 9.0, rel_tol=1e-12)
    assert math.isclose(yy, c * c * 9.0, rel_tol=1e-12)


def test_primal_update_lands_on_a_chosen_target():
    """PLAM: R = eta (X - Y) gives X - R/eta = Y (eq. PLAM-main).  PCAL: R = eta (X - Y diag(s))
    with Y of unit columns and s > 0 gives Y after the column normalisation (Algorithm 3)."""
    rng = np.random.default_rng(16)
    X = rng.standard_normal((20, 4))
    Y = rng.standard_normal((20, 4))
    eta = 3.5
    np.testing.assert_allclose(ok.primal_update(X, eta * (X - Y), eta, variant="plam"), Y,
                               rtol=1e-13, atol=1e-14)
    Yu = Y / np.linalg.norm(Y, axis=0)
    s = np.array([0.5, 2.0, 7.0, 1.0])
    np.testing.assert_allclose(ok.primal_update(X, eta * (X - Yu * s), eta, variant="pcal"), Yu,
                               rtol=1e-12, atol=1e-13)


def test_cholesky_qr_factor_recovers_a_planted_triangle():
    """X = Q R0 with Q orthonormal and R0 upper triangular with a positive diagonal: R0 is the
    unique Cholesky factor of X^T X, so the factor is R0 (Section 5.3's Cholesky-QR)."""
    Q = _orthonormal_block(50, 6, 17)
    R0 = np.triu(np.random.default_rng(18).standard_normal((6, 6)))
    R0[np.diag_indices(6)] = np.abs(R0[np.diag_indices(6)]) + 0.5
    np.testing.assert_allclose(ok.cholesky_qr_factor(Q @ R0), R0, rtol=1e-12, atol=1e-13)


def test_step_size_interval_of_width_zero_is_the_constant_rule():
    """eta^k clamped to [eta_min, eta_max] with eta_min = eta_max = gamma takes eta = gamma at every
    iteration, eta0 included, whatever the BB rule proposes: the run is the constant rule
    eta_C = gamma of Section 5.1, iterate for iterate."""
    w = workload_dense_trace(120, 6)
    obj = oo.TraceObjective(w.A)
    gamma = 30.0
    for variant in ("plam", "pcal"):
        a = op.solve(obj, w.X0, variant=variant, beta=1.0, eta_rule="abb", tol=0.0, maxit=25,
                     eta_min=gamma, eta_max=gamma)
        b = op.solve(obj, w.X0, variant=variant, beta=1.0, eta_rule="const", gamma=gamma, tol=0.0,
                     maxit=25)
        assert not a.diverged and len(a.history) == 26
        assert np.array_equal(a.X, b.X)
        assert all(h.eta == gamma for h in a.history[:-1])   # the last record takes no step


def test_step_size_interval_bounds_every_step():
    """A lower bound eta_min caps the step 1/eta^k: every recorded eta lies in the interval, and the
    bound binds on some steps of this run (ABB proposes smaller eta there)."""
    w = workload_dense_trace(120, 6)
    obj = oo.TraceObjective(w.A)
    free = op.solve(obj, w.X0, variant="pcal", beta=1.0, tol=0.0, maxit=40)
    etas = np.array([h.eta for h in free.history[:40]])
    lo = float(np.median(etas))
    r = op.solve(obj, w.X0, variant="pcal", beta=1.0, tol=0.0, maxit=40, eta_min=lo)
    got = np.array([h.eta for h in r.history[:40]])
    assert np.all(got >= lo) and np.sum(got == lo) >= 5
