"""Reference values of the individual steps of one PLAM/PCAL iteration, FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Each function is the plain definition of one step, so that element-wise parity
tests can check a single CUDA kernel in isolation:

  grams(X, G)                       B = X^T X, C = X^T G            (Table "cost": X^T X, grad f^T X)
  multiplier(X, G, beta, ...)       Lambda0 = Psi(C); d = diag(X^T grad_X L_beta(X, Lambda0))
                                    for eq. (lambda2); Lambda; M = Lambda - beta (B - I)
  update(X, G, M, Lambda0)          R = G - X M  (= grad_X L_beta, eq. S1) and
                                    K = G - X Lambda0 (KKT residual, Section 3.3)
  bb_dots(X, R, X_prev, R_prev)     <S,S>, <S,Y>, <Y,Y> with S = X - X_prev, Y = R - R_prev
  primal_update(X, R, eta, variant) the PLAM gradient step or the PCAL column-normalised step
  cholesky_qr_factor(X)             upper-triangular R with X^T X = R^T R, diag(R) > 0
"""
from __future__ import annotations

import numpy as np

from .plam import psi, lagrangian_grad


def grams(X, G):
    """B = X^T X and C = X^T G."""
    return X.T @ X, X.T @ G


def multiplier(X, G, beta, variant="pcal", lambda_rule="lambda2"):
    """(Lambda0, d, Lambda, M) of one iteration from the definitions (eqs. Lambda1, lambda2, S1)."""
    p = X.shape[1]
    B = X.T @ X
    L0 = psi(G.T @ X)
    if variant == "pcal" and lambda_rule == "lambda2":
        R0 = lagrangian_grad(G, X, B, L0, beta)
        d = np.diag(X.T @ R0).copy()
    else:
        d = np.zeros(p)
    Lam = L0 + np.diag(d)
    M = Lam - beta * (B - np.eye(p))
    return L0, d, Lam, M


def update(X, G, M, L0):
    """R = G - X M and K = G - X Lambda0."""
    return G - X @ M, G - X @ L0


def column_dots(X, R):
    """Per-column ||X_i||^2, <X_i, R_i>, ||R_i||^2."""
    return np.sum(X * X, axis=0), np.sum(X * R, axis=0), np.sum(R * R, axis=0)


def bb_dots(X, R, X_prev, R_prev):
    """<S,S>, <S,Y>, <Y,Y> for S = X - X_prev, Y = R - R_prev (Section 5.1)."""
    S = X - X_prev
    Y = R - R_prev
    return float(np.sum(S * S)), float(np.sum(S * Y)), float(np.sum(Y * Y))


def primal_update(X, R, eta, variant="pcal"):
    """PLAM: X - R/eta (eq. PLAM-main).  PCAL: each column of X - R/eta scaled to unit norm."""
    V = X - R / eta
    if variant == "plam":
        return V
    return V / np.linalg.norm(V, axis=0)[None, :]


def cholesky_qr_factor(X):
    """R upper triangular with X^T X = R^T R (definition: R from Householder QR, diag(R) > 0)."""
    _, Rf = np.linalg.qr(X)
    s = np.sign(np.diag(Rf))
    s[s == 0] = 1.0
    return Rf * s[:, None]
