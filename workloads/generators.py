"""Seeded generators for the synthetic PLAM/PCAL workloads.

Every random quantity is drawn from NumPy's PCG64 with a fixed seed

    seed = 1810039300 + 10 * config + stream      (stream 0 = operator, 1 = X0)

so that the oracle and the GPU path receive byte-identical FP64 inputs (the GPU
path casts them to FP32 when it runs a mixed-precision mode).  The shapes and
distributions follow the paper's test problems (Section 5.2: Problems 1 and 3,
the simplified Kohn-Sham energy and Rayleigh-Ritz trace minimisation) at the
sizes of the five benchmark configurations:

  1  dense trace minimisation, A=(B+B^T)/2, B iid N(0,1), n=500, p=20
  2  1D Hartree-type energy, L=tridiag(-1,2,-1) Dirichlet, n=20000, p=50
  3  3D 7-point Laplacian + diagonal potential V iid U[0,1], 64^3, p=256
  4  512 independent dense trace problems of uneven n in [64,2048], p in [4,64]
  5  3D Laplacian + potential, 128^3, p=1024

Nothing here evaluates the objective, the multipliers or any step of the
method; QR is used only to turn a Gaussian matrix into an orthonormal start.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

SEED_BASE = 1810039300

__all__ = [
    "SEED_BASE", "seed_for", "rng_for", "gaussian_symmetric", "orthonormal_start",
    "gaussian_start", "uniform_potential", "paper_p3_operator", "paper_p2_linear", "Workload",
    "workload_dense_trace", "workload_hartree1d", "workload_stencil3d",
    "batched_shapes", "workload_batched_problem", "workload_by_config",
    "workload_ks_exchange", "parameter_study_problems", "multiplier_study_problems",
    "workload_block_hartree", "workload_tridiag_linear", "paper_p4_matrices",
    "separable_potential", "stencil3d_separable_potential",
]


def seed_for(config: int, stream: int) -> int:
    """Seed of random stream `stream` of benchmark configuration `config` (1-based)."""
    return SEED_BASE + 10 * int(config) + int(stream)


def rng_for(config: int, stream: int, sub: Optional[int] = None) -> np.random.Generator:
    """PCG64 generator; `sub` distinguishes the problems of a batched configuration."""
    s = seed_for(config, stream)
    return np.random.Generator(np.random.PCG64(s if sub is None else [s, int(sub)]))


def gaussian_symmetric(n: int, rng: np.random.Generator) -> np.ndarray:
    """A = (B + B^T)/2 with B iid N(0,1) (the paper's `randn(n)` symmetrised)."""
    Bm = rng.standard_normal((n, n))
    return np.asfortranarray(0.5 * (Bm + Bm.T))


def orthonormal_start(n: int, p: int, rng: np.random.Generator) -> np.ndarray:
    """Q factor of an iid N(0,1) n-by-p matrix, columns signed so that diag(R) > 0.

    Column-major (Fortran) FP64, as the C ABI expects.
    """
    Z = rng.standard_normal((n, p))
    Q, Rf = np.linalg.qr(Z)
    s = np.sign(np.diag(Rf))
    s[s == 0] = 1.0
    return np.asfortranarray(Q * s)


def gaussian_start(n: int, p: int, rng: np.random.Generator) -> np.ndarray:
    """iid N(0, 1/n) entries: an infeasible start that is orthonormal to O(sqrt(p/n))."""
    return np.asfortranarray(rng.standard_normal((n, p)) / np.sqrt(n))


def uniform_potential(n: int, rng: np.random.Generator) -> np.ndarray:
    """Diagonal potential V, iid U[0,1]."""
    return rng.random(n)


def separable_potential(nx: int, ny: int, nz: int, rng: np.random.Generator,
                        high: float = 1.0 / 3.0) -> tuple[np.ndarray, np.ndarray, np.ndarray,
                                                          np.ndarray]:
    """A potential that is a sum of one function per grid axis, V[x + nx (y + ny z)] =
    v_x[x] + v_y[y] + v_z[z], each v_k iid U[0, high] (default 1/3, so V lies in [0, 1] with
    mean 1/2 like the iid U[0, 1] potential).  Returns (V, v_x, v_y, v_z)."""
    vx, vy, vz = rng.random(nx) * high, rng.random(ny) * high, rng.random(nz) * high
    V = (vz[:, None, None] + vy[None, :, None] + vx[None, None, :]).ravel()
    return V, vx, vy, vz


def paper_p3_operator(n: int, rng: np.random.Generator, theta: float = 1.01,
                      xi: float = 1.0) -> tuple[np.ndarray, np.ndarray]:
    """A = P diag(lam) P^T with P = qr(rand(n,n)) and lam_i = +-theta^(1-i) (Problem 2/3 generator).

    With xi = 1 every sign is +, so the spectrum is exactly {theta^(1-i)}.
    Returns (A, lam).
    """
    P, _ = np.linalg.qr(rng.random((n, n)))
    signs = np.where(rng.random(n) < xi, 1.0, -1.0)
    lam = signs * theta ** (1.0 - np.arange(1, n + 1))
    A = (P * lam) @ P.T
    return np.asfortranarray(0.5 * (A + A.T)), lam


def paper_p2_linear(n: int, p: int, rng: np.random.Generator, kappa: float = 1.0,
                    zeta: float = 1.01) -> np.ndarray:
    """Linear term of Problem 2: G = kappa Q D, Q_i = Qt_i/||Qt_i||, Qt = rand(n,p), D_jj = zeta^(j-1)."""
    Qt = rng.random((n, p))
    Q = Qt / np.linalg.norm(Qt, axis=0)[None, :]
    return np.asfortranarray(kappa * Q * (zeta ** np.arange(p))[None, :])


def paper_p4_matrices(n: int, p: int, rng: np.random.Generator) -> tuple[np.ndarray, np.ndarray]:
    """Problem 4's data (Section 5.2): A = (A0 + A0^T)/2 with A0 = randn(n), B = (B0 + B0^T)/2 with
    B0 = randn(p)."""
    A0 = rng.standard_normal((n, n))
    B0 = rng.standard_normal((p, p))
    return np.asfortranarray(0.5 * (A0 + A0.T)), 0.5 * (B0 + B0.T)


@dataclass
class Workload:
    """One synthetic problem instance: objective description, sizes and a start X0."""
    name: str
    kind: str                      # "dense" | "hartree1d" | "stencil3d"
    n: int
    p: int
    X0: np.ndarray                 # n-by-p, FP64, column-major
    A: Optional[np.ndarray] = None  # dense operator (kind == "dense")
    V: Optional[np.ndarray] = None  # diagonal potential (kind == "stencil3d")
    m: int = 0                     # grid edge (kind == "stencil3d"), n = m^3
    alpha: float = 1.0             # Hartree coupling (kind == "hartree1d")
    quad_scale: float = 0.25       # coefficient of tr(X^T L X) (kind == "hartree1d")
    xc: float = 0.0                # exchange coefficient gamma (kind == "hartree1d", Problem 6)
    block: int = 0                 # rows per Dirichlet block of L, 0 = one block (kind == "hartree1d")
    lin: Optional[np.ndarray] = None  # linear term G_lin, n-by-p (kind == "hartree1d", Problem 2)
    params: dict = field(default_factory=dict)  # suggested solver parameters


def workload_dense_trace(n: int = 500, p: int = 20, config: int = 1) -> Workload:
    """Configuration 1 shape: dense random symmetric A, orthonormal Gaussian start."""
    A = gaussian_symmetric(n, rng_for(config, 0))
    X0 = orthonormal_start(n, p, rng_for(config, 1))
    return Workload(name=f"dense_trace_n{n}_p{p}", kind="dense", n=n, p=p, X0=X0, A=A,
                    params=dict(variant="plam", beta=1.0, tol=1e-8))


def workload_hartree1d(n: int = 20000, p: int = 50, alpha: float = 1.0,
                       quad_scale: float = 0.25, config: int = 2) -> Workload:
    """Configuration 2 shape: 1D Dirichlet Laplacian + Hartree term, orthonormal start."""
    X0 = orthonormal_start(n, p, rng_for(config, 1))
    # beta = 1e3 sits above the largest Hessian eigenvalue at the solution (the
    # Hartree potential peaks near 3e2 there), the condition of Lemma 1; the
    # paper's PCAL default beta = 1 lets all columns collapse onto one vector.
    return Workload(name=f"hartree1d_n{n}_p{p}", kind="hartree1d", n=n, p=p, X0=X0,
                    alpha=alpha, quad_scale=quad_scale,
                    params=dict(variant="pcal", beta=1000.0, tol=1e-6))


def workload_ks_exchange(n: int = 2000, p: int = 10, config: int = 6) -> Workload:
    """Problem 6 shape (Section 5.2): f = 1/2 tr(X^T L X) + 1/2 rho^T L^{-1} rho
    - (3/4) gamma rho^T rho^{1/3}, gamma = 2 (3/pi)^{1/3}, L = tridiag(-1, 2, -1) Dirichlet
    (q = 1/2, alpha = 2, xc = gamma), orthonormal Gaussian start."""
    X0 = orthonormal_start(n, p, rng_for(config, 1))
    gamma = 2.0 * (3.0 / np.pi) ** (1.0 / 3.0)
    return Workload(name=f"ks_exchange_n{n}_p{p}", kind="hartree1d", n=n, p=p, X0=X0, alpha=2.0,
                    quad_scale=0.5, xc=gamma, params=dict(variant="pcal", beta=100.0, tol=1e-8))


def workload_block_hartree(n: int = 10000, p: int = 1000, block: int = 5,
                           config: int = 17) -> Workload:
    """Section 5.4's Problem 1: f = 1/2 tr(X^T L X) + 1/4 rho^T L^{-1} rho with the block-diagonal
    L = Diag(L_1, ..., L_s), each L_j = tridiag(-1, 2, -1) on `block` rows (q = 1/2, alpha = 1);
    orthonormal Gaussian start."""
    X0 = orthonormal_start(n, p, rng_for(config, 1))
    return Workload(name=f"block_hartree_n{n}_p{p}_b{block}", kind="hartree1d", n=n, p=p, X0=X0,
                    alpha=1.0, quad_scale=0.5, block=block,
                    params=dict(variant="pcal", beta=1.0, tol=1e-6))


def workload_tridiag_linear(n: int = 10000, p: int = 1000, config: int = 18) -> Workload:
    """Section 5.4's Problem 2: f = 1/2 tr(X^T A X) + tr(G_lin^T X) with A = tridiag(-1, 2, -1)
    (q = 1/2, alpha = 0) and G_lin iid U[-1, 1] (a "Random(n, p)" matrix); orthonormal
    Gaussian start."""
    lin = np.asfortranarray(rng_for(config, 0).uniform(-1.0, 1.0, (n, p)))
    X0 = orthonormal_start(n, p, rng_for(config, 1))
    return Workload(name=f"tridiag_linear_n{n}_p{p}", kind="hartree1d", n=n, p=p, X0=X0,
                    alpha=0.0, quad_scale=0.5, lin=lin,
                    params=dict(variant="pcal", beta=1.0, tol=1e-6))


def workload_stencil3d(m: int = 64, p: int = 256, config: int = 3,
                       start: str = "orthonormal") -> Workload:
    """Configurations 3/5 shape: 7-point Dirichlet Laplacian on m^3 + V iid U[0,1]."""
    n = m ** 3
    V = uniform_potential(n, rng_for(config, 0))
    r1 = rng_for(config, 1)
    X0 = orthonormal_start(n, p, r1) if start == "orthonormal" else gaussian_start(n, p, r1)
    return Workload(name=f"stencil3d_m{m}_p{p}", kind="stencil3d", n=n, p=p, X0=X0, V=V, m=m,
                    params=dict(variant="pcal", beta=1.0, tol=1e-6))


def stencil3d_separable_potential(m: int = 128, config: int = 5):
    """The separable potential of the 128^3 workload's companion instance (stream 3 of
    configuration 5), whose optimum is exact: (V, v_x, v_y, v_z)."""
    return separable_potential(m, m, m, rng_for(config, 3))


def batched_shapes(count: int = 512, n_lo: int = 64, n_hi: int = 2048, p_lo: int = 4,
                   p_hi: int = 64, config: int = 4) -> list[tuple[int, int]]:
    """(n_b, p_b) for the batched configuration: n uniform in [n_lo, n_hi], then
    p uniform in [p_lo, min(p_hi, n // 2)] so that 2p <= n."""
    rng = rng_for(config, 2)
    out = []
    for _ in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        p = int(rng.integers(p_lo, min(p_hi, n // 2) + 1))
        out.append((n, p))
    return out


def workload_batched_problem(b: int, n: int, p: int, config: int = 4) -> Workload:
    """Problem b of the batched configuration (its own seeded sub-streams)."""
    A = gaussian_symmetric(n, rng_for(config, 0, sub=b))
    X0 = orthonormal_start(n, p, rng_for(config, 1, sub=b))
    return Workload(name=f"batched_{b}_n{n}_p{p}", kind="dense", n=n, p=p, X0=X0, A=A,
                    params=dict(variant="pcal", beta=1.0, tol=1e-6))


def parameter_study_problems(count: int = 12, n: int = 200, p: int = 8) -> tuple[list, list]:
    """A seeded set of Problem-3-type trace problems for the parameter study of Section 5.1:
    A_i = (B + B^T)/2 with B iid N(0, 1), orthonormal Gaussian starts (config 7, sub-stream i)."""
    As = [gaussian_symmetric(n, rng_for(7, 0, sub=i)) for i in range(count)]
    X0s = [orthonormal_start(n, p, rng_for(7, 1, sub=i)) for i in range(count)]
    return As, X0s


def multiplier_study_problems(count: int = 6, n: int = 200, p: int = 8) -> tuple[list, list]:
    """Seeded Problem 1 and Problem 2 instances for the comparison of the closed-form multiplier
    with dual ascent (Section 5.3, Fig. "PCAL_multiplier"), shaped as Section 5.2 states them.

    Problem 1 (config 15): L = (B + B^T)/2 with B iid N(0, 1); returns (L, X0) pairs.
    Problem 2 (config 16): A = P diag(theta^(1-i)) P^T and G = kappa Q D with the default
    parameters kappa = 1, theta = zeta = 1.01, xi = 1; returns (A, lam, G, X0) tuples.
    Starts are orthonormal Gaussian (stream 1 of each config, sub-stream i)."""
    p1 = [(gaussian_symmetric(n, rng_for(15, 0, sub=i)), orthonormal_start(n, p, rng_for(15, 1, sub=i)))
          for i in range(count)]
    p2 = []
    for i in range(count):
        A, lam = paper_p3_operator(n, rng_for(16, 0, sub=i))
        Gl = paper_p2_linear(n, p, rng_for(16, 2, sub=i))
        p2.append((A, lam, Gl, orthonormal_start(n, p, rng_for(16, 1, sub=i))))
    return p1, p2


def workload_by_config(config: int) -> Workload:
    """Full-size instance of configurations 1, 2, 3 and 5 (4 is a batch: see batched_shapes)."""
    if config == 1:
        return workload_dense_trace(500, 20, config=1)
    if config == 2:
        return workload_hartree1d(20000, 50, config=2)
    if config == 3:
        return workload_stencil3d(64, 256, config=3)
    if config == 5:
        return workload_stencil3d(128, 1024, config=5, start="gaussian")
    raise ValueError(f"no single-instance workload for configuration {config}")
