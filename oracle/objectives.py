"""Objectives f(X) and gradients of the paper's test problems, FP64 (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

  TraceObjective     Problem 3 (Section 5.2, eq. RR): f = 1/2 tr(X^T A X), grad = A X.
  HartreeObjective   Problem 1 / Kohn-Sham form (Section 1.1 eq. KS-energy,
                     Section 5.2 eq. nonlinear), optionally with Problem 6's
                     exchange term -(3 gamma/4) sum rho^{4/3}:
                         f = q tr(X^T L X) + (alpha/4) rho^T L^{-1} rho,
                         rho = diag(X X^T),
                     L = tridiag(-1, 2, -1) with Dirichlet ends.  q = 1/4 follows
                     the Kohn-Sham energy (q = 1/2 is Problem 1's scaling).
                     Gradient: 2 q L X + alpha Diag(L^{-1} rho) X, since
                     d rho_i / d X_ij = 2 X_ij and d(rho^T L^{-1} rho)/d rho = 2 L^{-1} rho.
                     L^{-1} rho is a banded LAPACK solve (scipy.linalg.solve_banded).
  Stencil3DObjective f = 1/2 tr(X^T (L3 + Diag(V)) X), L3 the 7-point Dirichlet
                     Laplacian on an m^3 grid (6 on the diagonal, -1 per
                     neighbour), built as a Kronecker sum of 1D tridiagonals;
                     lexicographic index i = x + m y + m^2 z.
                     With `block` L is block-diagonal and `lin` adds Problem 2's
                     linear term tr(G_lin^T X) (Section 5.4's parallel workloads).
  QuadLinearObjective Problem 2 (eq. OCQP): f = 1/2 tr(X^T A X) + tr(G^T X).
  QAPObjective       Problem 4 (eq. QAP): f = 1/2 tr(A^T X B X^T), grad = A X B.
  DenseHartreeObjective Problem 1 exactly (eq. nonlinear): dense symmetric L and
                     its pseudo-inverse L^+ (numpy.linalg.pinv), coefficient q.
  trace_min_optimum  the optimum of a trace problem f = 1/2 tr(X^T H X) over
                     X^T X = I_p: half the sum of the p smallest eigenvalues of H
                     (Ky Fan), by a shift-invert Lanczos eigensolve (ARPACK) of a
                     sparse H.
  separable_trace_min_optimum  the same optimum for H = L3 + Diag(V) with a
                     separable potential V(x, y, z) = v_x(x) + v_y(y) + v_z(z):
                     H is then the Kronecker sum of three 1D operators
                     T_k = tridiag(-1, 2, -1) + Diag(v_k), so its eigenvalues are
                     the sums mu_a + mu_b + mu_c of theirs (three symmetric
                     tridiagonal eigensolves, LAPACK stev), and f* is half the
                     sum of the p smallest such sums (Ky Fan), exact at any size.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


class TraceObjective:
    """f = 1/2 tr(X^T A X) (Problem 3)."""

    def __init__(self, A: np.ndarray):
        self.A = np.asarray(A, dtype=np.float64)
        self.n = self.A.shape[0]

    def value(self, X):
        return 0.5 * float(np.sum(X * (self.A @ X)))

    def grad(self, X):
        return self.A @ X

    def hess_norm_bound(self):
        """s = ||grad^2 f(0)||_2 = ||A||_2 (Section 5.1)."""
        return float(np.max(np.abs(np.linalg.eigvalsh(self.A))))


class QuadLinearObjective:
    """f = 1/2 tr(X^T A X) + tr(G^T X) (Problem 2)."""

    def __init__(self, A: np.ndarray, Glin: np.ndarray):
        self.A = np.asarray(A, dtype=np.float64)
        self.Glin = np.asarray(Glin, dtype=np.float64)
        self.n = self.A.shape[0]

    def value(self, X):
        return 0.5 * float(np.sum(X * (self.A @ X))) + float(np.sum(self.Glin * X))

    def grad(self, X):
        return self.A @ X + self.Glin


class QAPObjective:
    """f = 1/2 tr(A^T X B X^T) with A, B symmetric (Problem 4, Section 5.2 eq. QAP).

    d/dX tr(A^T X B X^T) = A X B^T + A^T X B, so grad f = 1/2 (A X B + A X B) = A X B for
    symmetric A and B.  s = ||A||_2 ||B||_2 bounds the Hessian at 0."""

    def __init__(self, A: np.ndarray, B: np.ndarray):
        self.A = np.asarray(A, dtype=np.float64)
        self.B = np.asarray(B, dtype=np.float64)
        self.n = self.A.shape[0]

    def value(self, X):
        return 0.5 * float(np.sum((self.A @ X) * (X @ self.B)))

    def grad(self, X):
        return self.A @ X @ self.B

    def hess_norm_bound(self):
        return float(np.max(np.abs(np.linalg.eigvalsh(self.A))) * np.max(np.abs(np.linalg.eigvalsh(self.B))))


def laplacian_1d_coupled(n: int, block: int = 0) -> np.ndarray:
    """c[i] = True where rows i and i + 1 are coupled by the off-diagonal -1 of L (length n - 1).

    block = 0: L = tridiag(-1, 2, -1) over all n rows.  block = b > 0: L = Diag(L_1, ..., L_s)
    with every L_j that tridiagonal matrix on b consecutive rows (the last one on the n - (s-1) b
    rows left), the block-diagonal Laplacian of Section 5.4's Problem 1; rows b j - 1 and b j
    are then not coupled."""
    c = np.ones(max(n - 1, 0), dtype=bool)
    if block > 0:
        c[block - 1::block] = False
    return c


def laplacian_1d_banded(n: int, block: int = 0) -> np.ndarray:
    """The 3 x n band storage of L (see laplacian_1d_coupled) for scipy.linalg.solve_banded."""
    c = laplacian_1d_coupled(n, block)
    ab = np.zeros((3, n))
    ab[0, 1:] = np.where(c, -1.0, 0.0)      # superdiagonal: ab[0, j] = L[j-1, j]
    ab[1, :] = 2.0
    ab[2, :-1] = np.where(c, -1.0, 0.0)     # subdiagonal: ab[2, j] = L[j+1, j]
    return ab


def laplacian_1d_apply(X: np.ndarray, block: int = 0) -> np.ndarray:
    """L X for L = tridiag(-1, 2, -1) with zero (Dirichlet) values outside each block."""
    Y = 2.0 * X
    c = laplacian_1d_coupled(X.shape[0], block)
    if X.ndim == 1:
        Y[1:] -= np.where(c, X[:-1], 0.0)
        Y[:-1] -= np.where(c, X[1:], 0.0)
    else:
        Y[1:] -= np.where(c[:, None], X[:-1], 0.0)
        Y[:-1] -= np.where(c[:, None], X[1:], 0.0)
    return Y


class HartreeObjective:
    """f = q tr(X^T L X) + (alpha/4) rho^T L^{-1} rho - (3 xc/4) sum_i rho_i^{4/3} + tr(G_lin^T X),
    rho = diag(X X^T).

    The third term is Problem 6's exchange energy (Section 5.2, gamma = xc); its gradient
    follows from d rho_i / d X_ij = 2 X_ij: -(3 xc/4)(4/3) rho_i^{1/3} 2 X_ij = -2 xc rho_i^{1/3} X_ij.
    `block` makes L block-diagonal (laplacian_1d_coupled) and `lin` adds the linear term of
    Problem 2 (gradient + G_lin): Section 5.4 runs Problem 1 with blocks of 5 rows and Problem 2
    with the tridiagonal A = L and a random G_lin (q = 1/2, alpha = 0)."""

    def __init__(self, n: int, alpha: float = 1.0, quad_scale: float = 0.25, xc: float = 0.0,
                 block: int = 0, lin: np.ndarray | None = None):
        self.n = int(n)
        self.alpha = float(alpha)
        self.q = float(quad_scale)
        self.xc = float(xc)
        self.block = int(block)
        self.lin = None if lin is None else np.asarray(lin, dtype=np.float64)
        self._ab = laplacian_1d_banded(self.n, self.block)

    def density(self, X):
        return np.sum(X * X, axis=1)

    def hartree_potential(self, rho):
        """L^{-1} rho by a banded LU solve (LAPACK gbsv)."""
        return sla.solve_banded((1, 1), self._ab, rho, check_finite=False)

    def value(self, X):
        rho = self.density(X)
        y = self.hartree_potential(rho)
        f = (self.q * float(np.sum(X * laplacian_1d_apply(X, self.block)))
             + 0.25 * self.alpha * float(rho @ y) - 0.75 * self.xc * float(np.sum(np.cbrt(rho) * rho)))
        if self.lin is not None:
            f += float(np.sum(self.lin * X))
        return f

    def grad(self, X):
        rho = self.density(X)
        y = self.hartree_potential(rho)
        G = (2.0 * self.q * laplacian_1d_apply(X, self.block) + self.alpha * (y[:, None] * X)
             - 2.0 * self.xc * (np.cbrt(rho)[:, None] * X))
        if self.lin is not None:
            G = G + self.lin
        return G

    def hess_norm_bound(self):
        """Upper bound of ||grad^2 f(0)||_2 = 2 q ||L||_2 <= 8 q (the Hartree part vanishes at 0)."""
        return 8.0 * self.q


class DenseHartreeObjective:
    """f = q tr(X^T L X) + (alpha/4) rho^T L^+ rho with a dense symmetric L (Problem 1)."""

    def __init__(self, L: np.ndarray, alpha: float = 1.0, quad_scale: float = 0.5):
        self.L = np.asarray(L, dtype=np.float64)
        self.n = self.L.shape[0]
        self.alpha = float(alpha)
        self.q = float(quad_scale)
        self.Lp = np.linalg.pinv(self.L, hermitian=True)

    def value(self, X):
        rho = np.sum(X * X, axis=1)
        return self.q * float(np.sum(X * (self.L @ X))) + 0.25 * self.alpha * float(rho @ (self.Lp @ rho))

    def grad(self, X):
        rho = np.sum(X * X, axis=1)
        return 2.0 * self.q * (self.L @ X) + self.alpha * ((self.Lp @ rho)[:, None] * X)

    def hess_norm_bound(self):
        """s = ||grad^2 f(0)||_2 = 2 q ||L||_2 (Problem 1 states s = ||L||_2 for q = 1/2)."""
        return 2.0 * self.q * float(np.max(np.abs(np.linalg.eigvalsh(self.L))))


def laplacian_3d(m) -> sp.csr_matrix:
    """7-point Dirichlet Laplacian on an m^3 grid (m an int) or an nx x ny x nz grid (m a tuple),
    index x + nx (y + ny z), as I(x)I(x)T_x + I(x)T_y(x)I + T_z(x)I(x)I."""
    nx, ny, nz = (m, m, m) if np.isscalar(m) else tuple(int(t) for t in m)

    def T(k):
        return sp.diags([-np.ones(k - 1), 2.0 * np.ones(k), -np.ones(k - 1)], [-1, 0, 1], format="csr")

    Ix, Iy, Iz = (sp.identity(k, format="csr") for k in (nx, ny, nz))
    return (sp.kron(Iz, sp.kron(Iy, T(nx))) + sp.kron(Iz, sp.kron(T(ny), Ix))
            + sp.kron(T(nz), sp.kron(Iy, Ix))).tocsr()


class Stencil3DObjective:
    """f = 1/2 tr(X^T (L3 + Diag(V)) X) on an m^3 grid (m an int) or an nx x ny x nz grid
    (m a tuple: a slab of z-planes, with Dirichlet ends in every direction)."""

    def __init__(self, m, V: np.ndarray):
        self.grid = (m, m, m) if np.isscalar(m) else tuple(int(t) for t in m)
        self.m = int(m) if np.isscalar(m) else self.grid
        self.n = self.grid[0] * self.grid[1] * self.grid[2]
        self.V = np.asarray(V, dtype=np.float64)
        self.H = (laplacian_3d(self.m) + sp.diags(self.V)).tocsr()

    def value(self, X):
        return 0.5 * float(np.sum(X * (self.H @ X)))

    def grad(self, X):
        return self.H @ X

    def hess_norm_bound(self):
        """||L3 + V||_2 <= 12 + max V (Gershgorin)."""
        return 12.0 + float(np.max(self.V))


def objective_for(w) -> object:
    """Build the oracle objective described by a workloads.Workload."""
    if w.kind == "dense":
        return TraceObjective(w.A)
    if w.kind == "hartree1d":
        return HartreeObjective(w.n, w.alpha, w.quad_scale, getattr(w, "xc", 0.0) or 0.0,
                                getattr(w, "block", 0) or 0, getattr(w, "lin", None))
    if w.kind == "stencil3d":
        return Stencil3DObjective(w.m, w.V)
    raise ValueError(w.kind)


def trace_min_optimum(H, p: int, shift: float | None = None):
    """min { 1/2 tr(X^T H X) : X^T X = I_p } = 1/2 (lambda_1 + ... + lambda_p) for symmetric H
    (Ky Fan's minimum principle), with the p smallest eigenvalues from ARPACK in shift-invert
    mode about `shift` (default: a Gershgorin lower bound of the spectrum, so that the
    eigenvalues nearest the shift are the smallest ones).  Returns (f*, eigenvalues)."""
    import scipy.sparse.linalg as spla
    H = sp.csc_matrix(H)
    if shift is None:
        d = H.diagonal()
        off = np.asarray(abs(H).sum(axis=1)).ravel() - np.abs(d)
        shift = float(np.min(d - off)) - 1e-3
    ev = spla.eigsh(H, k=p, sigma=shift, which="LM", return_eigenvectors=False)
    ev = np.sort(ev)
    return 0.5 * float(ev.sum()), ev


def separable_trace_min_optimum(v_x, v_y, v_z, p: int):
    """(f*, the p + 1 smallest eigenvalues) of H = L3 + Diag(V) on an nx x ny x nz grid with
    V[x + nx (y + ny z)] = v_x[x] + v_y[y] + v_z[z]: H = T_z (x) I (x) I + I (x) T_y (x) I
    + I (x) I (x) T_x with T_k = tridiag(-1, 2, -1) + Diag(v_k) (Dirichlet), whose eigenvalues
    are all sums of one eigenvalue of each T_k; f* = 1/2 (lambda_1 + ... + lambda_p)."""
    mus = []
    for v in (v_x, v_y, v_z):
        v = np.asarray(v, dtype=np.float64)
        mus.append(sla.eigh_tridiagonal(2.0 + v, -np.ones(len(v) - 1), eigvals_only=True))
    mx, my, mz = mus
    sums = (mz[:, None, None] + my[None, :, None] + mx[None, None, :]).ravel()
    k = min(p + 1, sums.size)
    ev = np.sort(np.partition(sums, k - 1)[:k])
    return 0.5 * float(ev[:p].sum()), ev

