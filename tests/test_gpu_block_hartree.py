"""GPU parity of the 1D objective with a block-diagonal L and Problem 2's linear term: the
parallel forms of Problems 1 and 2 that Section 5.4 runs (n = 10000, p = 1000).

* the gradient and energy kernels against the oracle, over ragged tiles, ragged column
  groups, a ragged last block, the largest block and every combination of the Hartree,
  exchange and linear terms, in FP64 and FP32;
* PCAL solves at n = 2000 against the oracle's solves from the same start;
* the full-size solves (FP32 storage with tensor-core Grams, and FP64) against the stored
  oracle runs of tests/golden/section54_n10000_p1000.json.
"""
import json
import os

import numpy as np
import pytest

from oracle import objectives as oo
from oracle import plam as op
from tests.gpu_helpers import ITER_FACTOR, assert_entrywise, gpu_solver, to_dev, to_host
from workloads import (orthonormal_start, rng_for, workload_block_hartree,
                       workload_tridiag_linear)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "section54_n10000_p1000.json")

# n, p, block, alpha, xc, linear term
CASES = [
    (1000, 37, 5, 1.0, 0.0, False),    # Problem 1's form: tiles of 255 rows, a ragged last tile
    (1003, 50, 7, 1.3, 0.7, True),     # a ragged last block (1003 = 143 * 7 + 2), all three terms
    (2049, 19, 0, 0.0, 0.0, True),     # Problem 2's form: one block, the linear term only
    (997, 13, 64, 0.5, 0.0, False),    # the largest block
    (3001, 70, 3, 0.0, 0.3, False),    # exchange without Hartree: rho only, 256-row tiles
    (1300, 601, 5, 1.0, 0.0, True),    # three columns per column group, a ragged last group
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "n{}_p{}_b{}_a{}_xc{}_lin{}".format(*c))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_gradient_and_energy_match_oracle(case, precision):
    from paper_1810_03930_gb300 import Solver
    n, p, block, alpha, xc, with_lin = case
    rng = rng_for(20, 0, sub=n + p + block)
    lin = rng.uniform(-1.0, 1.0, (n, p)) if with_lin else None
    X = orthonormal_start(n, p, rng_for(20, 1, sub=n + p)) + 0.01 * rng.standard_normal((n, p))
    if precision == "fp32":
        X = X.astype(np.float32).astype(np.float64)
        lin = None if lin is None else lin.astype(np.float32).astype(np.float64)
    obj = oo.HartreeObjective(n, alpha=alpha, quad_scale=0.5, xc=xc, block=block, lin=lin)
    s = Solver(n, p, "hartree1d", alpha=alpha, quad_scale=0.5, xc=xc, block=block, lin=lin,
               precision=precision)
    Gd = s.new_matrix()
    f = s.energy_grad(to_dev(X, s), Gd)
    tol = 1e-12 if precision == "fp64" else 3e-6
    assert_entrywise(to_host(Gd, n), obj.grad(X), tol, what="chain gradient")
    fr = obj.value(X)
    assert abs(f - fr) <= tol * max(1.0, abs(fr)) * 10
    s.close()


@pytest.mark.parametrize("bad", [dict(block=0, lin=True, alpha=1.0), dict(block=65, alpha=1.0),
                                 dict(block=-1, alpha=0.0)])
def test_unsupported_block_forms_are_rejected(bad):
    """With the Hartree term the blocks must have 1..64 rows (one block of n rows runs on the
    prefix-sum kernels, which take no linear term); a negative block size is invalid."""
    from paper_1810_03930_gb300 import PlamError, Solver
    n, p = 500, 4
    lin = np.ones((n, p)) if bad.get("lin") else None
    with pytest.raises(PlamError):
        Solver(n, p, "hartree1d", alpha=bad["alpha"], quad_scale=0.5, block=bad["block"], lin=lin)


@pytest.mark.parametrize("make", [workload_block_hartree, workload_tridiag_linear],
                         ids=["problem1_blocks", "problem2_tridiag"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_pcal_solve_matches_oracle(make, precision):
    """PCAL (beta = 1, eq. lambda2, ABB) from the seeded start at n = 2000, p = 60: FP64 to
    relative KKT 1e-8 against the oracle's solve (iterations within 25%, f, and for Problem 2,
    whose linear term fixes X, the orthonormalised solution itself); FP32 to 1e-6 (f)."""
    w = make(2000, 60)
    obj = oo.objective_for(w)
    tol = 1e-8 if precision == "fp64" else 1e-6
    ref = op.solve(obj, w.X0, variant="pcal", beta=1.0, tol=tol, maxit=3000, record=False)
    assert ref.converged
    s = gpu_solver(w, precision, variant="pcal", beta=1.0, tol=tol, maxit=3000, final_orth=1,
                   engine="graph")
    Xd = to_dev(w.X0, s)
    Qd = s.new_matrix(dtype=torch.float64)
    st, info = s.solve(Xd, Qd)
    assert st == 0 and info.converged
    assert abs(info.iters - ref.iters) <= max(5, 0.25 * ref.iters)
    assert info.feas_orth <= 1e-12
    ftol = 1e-10 if precision == "fp64" else 2e-6
    assert abs(info.f_orth - ref.f_orth) <= ftol * abs(ref.f_orth)
    Q = to_host(Qd, w.n)
    assert abs(obj.value(Q) - ref.f_orth) <= ftol * abs(ref.f_orth)
    if make is workload_tridiag_linear:
        assert_entrywise(Q, ref.X_orth, ITER_FACTOR * (1e-6 if precision == "fp64" else 2e-3),
                         what="orthonormalised solution")
    s.close()


@pytest.mark.parametrize("make", [workload_block_hartree, workload_tridiag_linear],
                         ids=["problem1_blocks", "problem2_tridiag"])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_full_size_solve_matches_stored_oracle_run(make, precision):
    """Section 5.4's size, n = 10000, p = 1000, PCAL to relative KKT 1e-6 (FP32 storage runs
    its Grams on the tensor cores): the gradient at the start against the oracle's, then the
    solve against the stored oracle run (iterations within 50%, the orthonormalised objective,
    feasibility of the FP64 output), and the objective of the output evaluated by the oracle."""
    with open(GOLDEN) as fh:
        gold = json.load(fh)
    w = make()
    g = gold[w.name]
    assert (g["n"], g["p"]) == (w.n, w.p)
    obj = oo.objective_for(w)
    s = gpu_solver(w, precision, variant="pcal", beta=1.0, tol=1e-6, maxit=3000, final_orth=1)
    Xd = to_dev(w.X0, s)
    Gd = s.new_matrix()
    s.energy_grad(Xd, Gd)
    X0 = w.X0 if precision == "fp64" else w.X0.astype(np.float32).astype(np.float64)
    obj0 = obj
    if precision == "fp32" and w.lin is not None:
        obj0 = oo.HartreeObjective(w.n, w.alpha, w.quad_scale, w.xc, w.block,
                                   w.lin.astype(np.float32).astype(np.float64))
    assert_entrywise(to_host(Gd, w.n), obj0.grad(X0), 1e-12 if precision == "fp64" else 3e-6,
                     what="gradient at the start")
    Qd = s.new_matrix(dtype=torch.float64)
    st, info = s.solve(Xd, Qd)
    ref = g["tol_1e-06"]
    assert st == 0 and info.converged
    assert abs(info.iters - ref["iters"]) <= max(5, 0.5 * ref["iters"])
    assert info.feas_orth <= 1e-12
    ftol = 1e-8 if precision == "fp64" else 1e-5
    fref = g["tol_1e-08"]["f_orth"]
    assert abs(info.f_orth - fref) <= ftol * abs(fref)
    Q = to_host(Qd, w.n)
    assert abs(obj.value(Q) - fref) <= ftol * abs(fref)
    s.close()
