"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin catches each one.

Each mutation replaces one oracle function with a subtly wrong version (a
dropped term, a flipped sign, a wrong factor, a missing neighbour, a wrong
norm) and runs the pin that should detect it; the pin must fail.
"""
import numpy as np
import pytest

import oracle.objectives as oo
import oracle.plam as op
from tests import test_oracle_pins as pins
from workloads import workload_dense_trace

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _c1_small():
    w = workload_dense_trace(120, 6)
    obj = oo.TraceObjective(w.A)
    ev, U = np.linalg.eigh(w.A)
    return w, obj, ev, U


def _trace_pin():
    w, obj, ev, _ = _c1_small()
    r = op.solve(obj, w.X0, variant="pcal", beta=1.0, tol=1e-8, maxit=600)
    assert r.converged
    fstar = 0.5 * ev[: w.p].sum()
    assert abs(r.f_orth - fstar) <= 1e-10 * abs(fstar)


def test_unmutated_small_trace_pin_passes():
    _trace_pin()


def test_dropped_penalty_term_is_caught(monkeypatch):
    def bad(G, X, B, Lam, beta):
        return G - X @ Lam
    monkeypatch.setattr(op, "lagrangian_grad", bad)
    with pytest.raises(AssertionError):
        pins.test_lemma2_feasibility_bound(0)


def test_flipped_multiplier_sign_is_caught(monkeypatch):
    def bad(G, X, B, Lam, beta):
        p = X.shape[1]
        return G + X @ Lam + beta * (X @ (B - np.eye(p)))
    monkeypatch.setattr(op, "lagrangian_grad", bad)
    with pytest.raises(AssertionError):
        _trace_pin()


def test_wrong_penalty_factor_is_caught(monkeypatch):
    def bad(G, X, B, Lam, beta):
        p = X.shape[1]
        return G - X @ Lam + beta * (X @ (B - np.eye(p))) @ B   # X (B - I) B instead of X (B - I)
    monkeypatch.setattr(op, "lagrangian_grad", bad)
    with pytest.raises(AssertionError):
        pins.test_single_step_matches_definitions()


def test_lambda2_sign_error_is_caught(monkeypatch):
    def bad(G, X, B, beta):
        L0 = op.psi(G.T @ X)
        R0 = op.lagrangian_grad(G, X, B, L0, beta)
        return L0 - op.phi(X.T @ R0)
    monkeypatch.setattr(op, "multiplier_lambda2", bad)
    with pytest.raises(AssertionError):
        pins.test_single_step_matches_definitions()


def test_hartree_missing_factor_two_is_caught(monkeypatch):
    def bad(self, X):
        rho = self.density(X)
        y = self.hartree_potential(rho)
        return self.q * oo.laplacian_1d_apply(X) + self.alpha * (y[:, None] * X)
    monkeypatch.setattr(oo.HartreeObjective, "grad", bad)
    with pytest.raises(AssertionError):
        pins.test_gradient_finite_difference("hartree")


def test_hartree_wrong_operator_is_caught(monkeypatch):
    def bad(self, rho):      # L rho instead of L^{-1} rho
        return oo.laplacian_1d_apply(rho[:, None])[:, 0]
    monkeypatch.setattr(oo.HartreeObjective, "hartree_potential", bad)
    with pytest.raises(AssertionError):
        pins.test_hartree_inverse_laplacian()


def test_stencil_missing_neighbours_is_caught(monkeypatch):
    import scipy.sparse as sp

    def bad(m):
        T = sp.diags([-np.ones(m - 1), 2.0 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1], format="csr")
        Im = sp.identity(m, format="csr")
        # z-direction coupling dropped (diagonal kept at 6)
        return (sp.kron(Im, sp.kron(Im, T)) + sp.kron(Im, sp.kron(T, Im))
                + 2.0 * sp.identity(m ** 3)).tocsr()
    monkeypatch.setattr(oo, "laplacian_3d", bad)
    with pytest.raises(AssertionError):
        pins.test_stencil3d_operator_brute_force()


@pytest.mark.parametrize("wrong", ["row_norms", "max_norm"])
def test_pcal_wrong_normalisation_is_caught(monkeypatch, wrong):
    def bad(V):
        if wrong == "row_norms":     # index mistake: normalise rows instead of columns
            return V / np.linalg.norm(V, axis=1)[:, None]
        return V / np.max(np.abs(V), axis=0)[None, :]
    monkeypatch.setattr(op, "normalize_columns", bad)
    w, obj, _, _ = _c1_small()
    with pytest.raises(AssertionError):
        pins.test_pcal_iterates_have_unit_columns((w, obj, None, None, None))


def test_noop_orthonormalisation_is_caught(monkeypatch):
    monkeypatch.setattr(op, "orthonormalize", lambda X: np.asfortranarray(X.copy()))
    w, obj, ev, U = _c1_small()
    sol = {v: op.solve(obj, w.X0, variant=v, beta=1.0, tol=1e-8, maxit=3000) for v in ("plam", "pcal")}
    with pytest.raises(AssertionError):
        pins.test_final_orthonormalisation((w, obj, ev, U, sol), "plam")


def test_block_coupling_kept_across_block_edges_is_caught(monkeypatch):
    """L with the off-diagonal -1 kept between blocks (one tridiagonal instead of Diag(L_j))."""
    monkeypatch.setattr(oo, "laplacian_1d_coupled", lambda n, block=0: np.ones(max(n - 1, 0), dtype=bool))
    with pytest.raises(AssertionError):
        pins.test_block_laplacian_trace_problem_reaches_ky_fan()


def test_dropped_linear_term_gradient_is_caught(monkeypatch):
    """Problem 2's linear term left out of the gradient (kept in f)."""
    orig = oo.HartreeObjective.grad

    def bad(self, X):
        G = orig(self, X)
        return G - self.lin if self.lin is not None else G
    monkeypatch.setattr(oo.HartreeObjective, "grad", bad)
    with pytest.raises(AssertionError):
        pins.test_gradient_finite_difference("block_hartree_lin_xc")


def test_problem4_gradient_without_b_is_caught(monkeypatch):
    """Problem 4's gradient with the right factor B dropped (A X instead of A X B)."""
    monkeypatch.setattr(oo.QAPObjective, "grad", lambda self, X: self.A @ X)
    with pytest.raises(AssertionError):
        pins.test_gradient_finite_difference("qap")


@pytest.mark.parametrize("wrong", ["unprojected_gradient", "column_normalisation"])
def test_moptqr_mistakes_are_caught(monkeypatch, wrong):
    """MOptQR's projected gradient without the projection X (G^T X), or a retraction that only
    normalises the columns of V (no Cholesky factor): a pin fails for each."""
    from oracle import moptqr as om
    if wrong == "unprojected_gradient":
        monkeypatch.setattr(om, "projected_gradient", lambda G, X: G)
        with pytest.raises(AssertionError):
            pins.test_moptqr_first_step_by_hand()
    else:
        monkeypatch.setattr(om, "cholesky_retraction",
                            lambda V: np.asfortranarray(V / np.linalg.norm(V, axis=0)[None, :]))
        with pytest.raises(AssertionError):
            pins.test_moptqr_retraction_is_the_qr_factor_and_keeps_feasibility()


@pytest.mark.parametrize("wrong", ["update_transposed_m", "update_sign", "update_k_uses_m",
                                   "bb_reversed_s", "bb_s_from_r", "primal_times_eta",
                                   "primal_row_norm", "chol_lower"])
def test_single_step_definition_mistakes_are_caught(monkeypatch, wrong):
    """A mistake in one of the single-step definitions the GPU kernels are checked against
    (oracle.kernels) fails that definition's pin."""
    import oracle.kernels as ok
    if wrong == "update_transposed_m":
        monkeypatch.setattr(ok, "update", lambda X, G, M, L0: (G - X @ M.T, G - X @ L0))
        pin = pins.test_update_residual_lies_outside_the_range_of_x
    elif wrong == "update_sign":
        monkeypatch.setattr(ok, "update", lambda X, G, M, L0: (G + X @ M, G - X @ L0))
        pin = pins.test_update_residual_lies_outside_the_range_of_x
    elif wrong == "update_k_uses_m":
        monkeypatch.setattr(ok, "update", lambda X, G, M, L0: (G - X @ M, G - X @ M))
        pin = pins.test_update_residual_lies_outside_the_range_of_x
    elif wrong == "bb_reversed_s":
        def bad(X, R, Xp, Rp):
            S, Y = Xp - X, R - Rp
            return float(np.sum(S * S)), float(np.sum(S * Y)), float(np.sum(Y * Y))
        monkeypatch.setattr(ok, "bb_dots", bad)
        pin = pins.test_bb_dots_along_one_direction
    elif wrong == "bb_s_from_r":
        def bad(X, R, Xp, Rp):
            S, Y = X - Xp, R - Rp
            return float(np.sum(S * S)), float(np.sum(Y * Y)), float(np.sum(Y * Y))
        monkeypatch.setattr(ok, "bb_dots", bad)
        pin = pins.test_bb_dots_along_one_direction
    elif wrong == "primal_times_eta":
        monkeypatch.setattr(ok, "primal_update", lambda X, R, eta, variant="pcal": X - R * eta)
        pin = pins.test_primal_update_lands_on_a_chosen_target
    elif wrong == "primal_row_norm":
        def bad(X, R, eta, variant="pcal"):
            V = X - R / eta
            return V if variant == "plam" else V / np.linalg.norm(V, axis=1)[:, None]
        monkeypatch.setattr(ok, "primal_update", bad)
        pin = pins.test_primal_update_lands_on_a_chosen_target
    else:
        monkeypatch.setattr(ok, "cholesky_qr_factor", lambda X: np.linalg.cholesky(X.T @ X))
        pin = pins.test_cholesky_qr_factor_recovers_a_planted_triangle
    with pytest.raises(AssertionError):
        pin()
