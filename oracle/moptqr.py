"""MOptQR, the comparison solver of Sections 5.3-5.4, FP64, step by step.

TEST INFRASTRUCTURE ONLY (see the package docstring).

MOptQR is a Riemannian gradient method on the Stiefel manifold with the QR (projection-like)
retraction; the paper equips it with the same alternating Barzilai-Borwein step as PLAM and
PCAL and lists one iteration's cost in Table "cost" (rows "MOptQR (cholesky LL^T)"):

  G  = grad f(X)
  D  = G - X (G^T X)                        the projected gradient (X^T D is skew-symmetric
                                            at a feasible X)
  V  = X - tau D,  tau = 1 / eta            eta from the rules of Section 5.1 on
                                            S = X^k - X^{k-1}, Y = D^k - D^{k-1}
  V^T V = L L^T  (Cholesky),  X <- V L^{-T} the retraction: the Q factor of V with a positive
                                            diagonal of R = L^T

Every iterate is feasible (to rounding), so no final orthonormalisation is needed.  The
stopping test is the one PLAM and PCAL use, ||G - X Psi(G^T X)||_F / (same at X^0) < tol.
Readings (the paper gives MOptQR no listing): eta at k = 0 is ||G^0||_F / ||X^0||_F (the
PLAM/PCAL rule with beta = 0: MOptQR has no penalty); the safeguards and clamps of
oracle.plam.step_size apply.
"""
from __future__ import annotations

import numpy as np

from .plam import IterRecord, SolveResult, default_eta0, feasibility, fro, kkt_residual, step_size


def projected_gradient(G, X):
    """D = G - X (G^T X) (Table "cost": V := X - tau (grad f(X) - X grad f(X)^T X))."""
    return G - X @ (G.T @ X)


def cholesky_retraction(V):
    """X = V L^{-T} with V^T V = L L^T (Table "cost": V^T V, chol(V^T V) = L L^T, V L^{-T})."""
    L = np.linalg.cholesky(V.T @ V)
    return np.asfortranarray(np.linalg.solve(L, V.T).T)


def solve(obj, X0, eta_rule="abb", eta0=None, tol=1e-8, maxit=3000, gamma=None,
          clamp=(1e-10, 1e10), eta_min=None, eta_max=None, record=True) -> SolveResult:
    """Run MOptQR from X0 (n-by-p, orthonormal)."""
    X = np.array(X0, dtype=np.float64, order="F", copy=True)
    G = obj.grad(X)
    K0 = fro(kkt_residual(G, X))
    if eta0 is None:
        eta0 = default_eta0(G, X, 0.0)
    # [eta_min, eta_max] when given (the interval the convergence analysis assumes for eta^k),
    # else relative to eta0
    lo = eta_min if eta_min else clamp[0] * eta0
    hi = eta_max if eta_max else clamp[1] * eta0
    hist = []
    X_prev = D_prev = None
    eta = eta0
    converged = diverged = False
    k = 0
    while True:
        if k > 0:
            G = obj.grad(X)
        kkt = fro(kkt_residual(G, X)) / K0 if K0 > 0 else 0.0
        if record:
            hist.append(IterRecord(k, obj.value(X), kkt, feasibility(X), np.nan))
        if not np.isfinite(kkt):
            diverged = True
            break
        if kkt < tol or K0 == 0.0:
            converged = True
            break
        if k >= maxit:
            break
        D = projected_gradient(G, X)
        S = None if X_prev is None else X - X_prev
        Y = None if D_prev is None else D - D_prev
        eta = step_size(eta_rule, k, S, Y, eta, eta0, gamma)
        if not np.isfinite(eta):
            diverged = True
            break
        eta = min(max(eta, lo), hi)
        if record:
            hist[-1].eta = eta
        X_prev, D_prev = X, D
        try:
            X = cholesky_retraction(X - D / eta)
        except np.linalg.LinAlgError:
            diverged = True
            X = X_prev
            break
        k += 1
    res = SolveResult(X=X, X_orth=X, iters=k, converged=converged, diverged=diverged, K0=K0,
                      eta0=eta0, history=hist)
    res.f_stop = res.f_orth = obj.value(X)
    res.kkt_stop = res.kkt_orth = fro(kkt_residual(obj.grad(X), X)) / K0 if K0 > 0 else 0.0
    res.feas_stop = res.feas_orth = feasibility(X)
    return res
