"""PLAM (Algorithm 2) and PCAL (Algorithm 3) of arXiv:1810.03930, FP64, step by step.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Notation (Section 1.3): Psi(A) = (A + A^T)/2, Phi(M) = Diag(diag(M)).
Problem (eq. prob): min f(X) subject to X^T X = I_p.

One iteration at X = X^k (G = grad f(X), B = X^T X):
  multiplier        Lambda = Psi(G^T X)                                  eq. (Lambda1)
  PCAL alternative  Lambda = Psi(G^T X) + Phi(X^T grad_X L_beta(X, Psi(G^T X)))   eq. (lambda2)
  Lagrangian grad   R = G + beta X (B - I - Lambda/beta)
                      = G - X Lambda + beta X (B - I)                   eq. (S1)
  PLAM update       X <- X - R / eta                                     eq. (PLAM-main)
  PCAL update       X_i <- (X_i - R_i/eta) / ||X_i - R_i/eta||_2 for every column i,
                    all columns computed from X^k (closed form after eq. PLLagSph)
  step size         eta rules of Section 5.1: C, D, BB1, BB2 and ABB (default)
  stop              ||G - X Psi(G^T X)||_F / (same at X^0) < tol, or maxit
                    (Section 5.1; the Psi form is the practice of Section 3.3)
  final step        one orthonormalisation of the last iterate (Section 5.3,
                    Table "orth step"): Householder QR with diag(R) > 0.

Readings where the paper is silent or ambiguous (each listed in the design notes):
  * S and Y in the BB rules are the most recent differences,
    S = X^k - X^{k-1}, Y = R^k - R^{k-1}, with R the gradient actually stepped
    with (the PCAL multiplier when PCAL uses eq. lambda2).
  * ABB: k counts from 0; k = 0 uses eta0; odd k uses BB1, even k >= 2 BB2.
  * eta0 (no history at k = 0) defaults to ||G^0||_F / ||X^0||_F + beta.
  * Safeguards: if <S,S> = 0 or <S,Y> = 0 the previous eta is kept; every eta,
    eta0 included, is clamped to [eta_min, eta_max] (the interval of the step-size
    condition of the convergence analysis) when they are given, else to
    [1e-10 eta0, 1e10 eta0].
  * If the initial KKT residual is exactly zero the start is returned as converged.
  * A non-finite KKT value, step size or iterate stops the run as diverged; X
    is then the last finite iterate.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def psi(A: np.ndarray) -> np.ndarray:
    """Psi(A) = (A + A^T)/2 (Section 1.3)."""
    return 0.5 * (A + A.T)


def phi(M: np.ndarray) -> np.ndarray:
    """Phi(M) = Diag(diag(M)) (Section 1.3)."""
    return np.diag(np.diag(M))


def lagrangian_grad(G, X, B, Lam, beta):
    """grad_X L_beta(X, Lambda) = G - X Lambda + beta X (X^T X - I), eq. (S1)."""
    p = X.shape[1]
    return G - X @ Lam + beta * (X @ (B - np.eye(p)))


def multiplier_lambda1(G, X):
    """Lambda = Psi(grad f(X)^T X), eq. (Lambda1)."""
    return psi(G.T @ X)


def multiplier_lambda2(G, X, B, beta):
    """Lambda = Psi(G^T X) + Phi(X^T grad_X L_beta(X, Psi(G^T X))), eq. (lambda2)."""
    L0 = psi(G.T @ X)
    R0 = lagrangian_grad(G, X, B, L0, beta)
    return L0 + phi(X.T @ R0)


def kkt_residual(G, X):
    """G - X Psi(G^T X): the KKT violation of eq. (kkt2) in the Psi form of Section 3.3."""
    return G - X @ psi(G.T @ X)


def feasibility(X):
    """||X^T X - I||_F."""
    p = X.shape[1]
    return float(np.linalg.norm(X.T @ X - np.eye(p)))


def fro(A):
    return float(np.linalg.norm(A))


def orthonormalize(X):
    """Final orthonormalisation: Householder QR (LAPACK geqrf), Q signed so diag(R) > 0."""
    Q, Rf = np.linalg.qr(X)
    s = np.sign(np.diag(Rf))
    s[s == 0] = 1.0
    return np.asfortranarray(Q * s)


def normalize_columns(V):
    """PCAL's closed form (Algorithm 3): every column divided by its 2-norm."""
    return V / np.linalg.norm(V, axis=0)[None, :]


def default_eta0(G0, X0, beta):
    """eta0 = ||G^0||_F / ||X^0||_F + beta (reading: the paper gives no rule for k = 0)."""
    nx = fro(X0)
    return (fro(G0) / nx if nx > 0 else 1.0) + beta


def step_size(rule, k, S, Y, eta_prev, eta0, gamma=None):
    """eta^k by the rules of Section 5.1.  S = X^k - X^{k-1}, Y = R^k - R^{k-1}."""
    if rule == "const":
        return gamma if gamma is not None else eta0
    if k == 0:
        return eta0
    ss = float(np.sum(S * S))
    sy = float(np.sum(S * Y))
    yy = float(np.sum(Y * Y))
    if rule == "diff":                      # eta_D = ||Y||_F / ||S||_F
        return np.sqrt(yy / ss) if ss > 0 and yy > 0 else eta_prev
    if ss == 0.0 or sy == 0.0:
        return eta_prev
    bb1 = abs(sy) / ss                      # eta_BB1 = |<S,Y>| / <S,S>
    bb2 = yy / abs(sy)                      # eta_BB2 = <Y,Y> / |<S,Y>|
    if rule == "bb1":
        return bb1
    if rule == "bb2":
        return bb2
    if rule == "abb":                       # BB1 for odd k, BB2 for even k
        return bb1 if (k % 2 == 1) else bb2
    raise ValueError(rule)


@dataclass
class IterRecord:
    k: int
    f: float
    kkt: float       # relative KKT violation
    feas: float      # ||X^T X - I||_F
    eta: float       # eta^k used for the update of iteration k (nan on the last record)


@dataclass
class SolveResult:
    X: np.ndarray            # last iterate (before orthonormalisation)
    X_orth: np.ndarray       # after the final orthonormalisation
    iters: int               # number of updates performed
    converged: bool
    diverged: bool           # a non-finite KKT value or step size stopped the run
    K0: float                # ||G^0 - X^0 Psi(G0^T X0)||_F
    eta0: float
    history: list = field(default_factory=list)
    f_stop: float = np.nan
    kkt_stop: float = np.nan
    feas_stop: float = np.nan
    f_orth: float = np.nan
    kkt_orth: float = np.nan
    feas_orth: float = np.nan
    Lambda: np.ndarray | None = None   # Psi(G^T X) at the last iterate
    C_last: np.ndarray | None = None   # unsymmetrised X^T G at the last iterate


def solve(obj, X0, variant="pcal", beta=1.0, lambda_rule="lambda2", eta_rule="abb",
          eta0=None, tol=1e-8, maxit=3000, gamma=None, clamp=(1e-10, 1e10), eta_min=None,
          eta_max=None,
          record=True, callback=None) -> SolveResult:
    """Run PLAM (variant='plam') or PCAL (variant='pcal') from X0 (n-by-p, FP64)."""
    if variant not in ("plam", "pcal"):
        raise ValueError(variant)
    X = np.array(X0, dtype=np.float64, order="F", copy=True)
    p = X.shape[1]
    I = np.eye(p)
    G = obj.grad(X)
    K0 = fro(kkt_residual(G, X))
    if eta0 is None:
        eta0 = default_eta0(G, X, beta)
    # [eta_min, eta_max] when given (the interval the convergence analysis assumes for eta^k),
    # else relative to eta0
    lo = eta_min if eta_min else clamp[0] * eta0
    hi = eta_max if eta_max else clamp[1] * eta0
    hist = []
    X_prev = R_prev = None
    Lam_prev = None
    eta = eta0
    converged = diverged = False
    k = 0
    while True:
        if k > 0:
            G = obj.grad(X)
        B = X.T @ X
        C = X.T @ G
        L0 = psi(C)
        kkt = fro(G - X @ L0) / K0 if K0 > 0 else 0.0
        if record:
            hist.append(IterRecord(k, obj.value(X), kkt, fro(B - I), np.nan))
        if not np.isfinite(kkt):
            diverged = True
            break
        if kkt < tol or K0 == 0.0:
            converged = True
            break
        if k >= maxit:
            break
        if lambda_rule == "da":
            # PLAM-DA / PCAL-DA (Section 5.3): Algorithm 1's dual ascent step,
            # Lambda^k = Lambda^{k-1} - beta (X^k^T X^k - I), from Lambda^0 = Psi(G^0^T X^0)
            Lam = L0 if Lam_prev is None else Lam_prev - beta * (B - I)
            Lam_prev = Lam
        elif variant == "pcal" and lambda_rule == "lambda2":
            Lam = multiplier_lambda2(G, X, B, beta)
        else:
            Lam = L0
        R = lagrangian_grad(G, X, B, Lam, beta)
        S = None if X_prev is None else X - X_prev
        Y = None if R_prev is None else R - R_prev
        eta = step_size(eta_rule, k, S, Y, eta, eta0, gamma)
        if not np.isfinite(eta):
            diverged = True
            break
        eta = min(max(eta, lo), hi)
        if record:
            hist[-1].eta = eta
        if callback is not None:
            callback(k, X, G, R, eta)
        X_prev, R_prev = X, R
        V = X - R / eta
        if variant == "plam":
            Xn = V
        else:
            Xn = normalize_columns(V)
        if not np.all(np.isfinite(Xn)):
            diverged = True
            break
        X = np.asfortranarray(Xn)
        k += 1
    if diverged:
        return SolveResult(X=X, X_orth=X, iters=k, converged=False, diverged=True, K0=K0,
                           eta0=eta0, history=hist)
    Xo = orthonormalize(X)
    Go = obj.grad(Xo)
    res = SolveResult(X=X, X_orth=Xo, iters=k, converged=converged, diverged=False, K0=K0,
                      eta0=eta0, history=hist)
    res.f_stop = obj.value(X)
    res.kkt_stop = fro(kkt_residual(G, X)) / K0 if K0 > 0 else 0.0
    res.feas_stop = feasibility(X)
    res.f_orth = obj.value(Xo)
    res.kkt_orth = fro(kkt_residual(Go, Xo)) / K0 if K0 > 0 else 0.0
    res.feas_orth = feasibility(Xo)
    res.Lambda = psi(X.T @ G)
    res.C_last = X.T @ G
    return res
