"""Batched persistent solves (configuration 4's shape): many independent dense trace problems of
uneven n, p in one launch, against the FP64 oracle and the paper's closed-form optimum."""
import numpy as np
import pytest

from oracle import objectives as oo
from oracle import plam as op
from tests.gpu_helpers import ITER_FACTOR, assert_entrywise, to_host
from workloads import batched_shapes, workload_batched_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _problems(count, n_hi=640, seed_shift=0):
    shapes = batched_shapes(count=count, n_lo=64, n_hi=n_hi)
    return [workload_batched_problem(b + seed_shift, n, p) for b, (n, p) in enumerate(shapes)]


@pytest.mark.parametrize("variant,tol", [("pcal", 1e-6), ("plam", 1e-5)])
def test_batched_solves_reach_eigenvalue_sums(variant, tol):
    """Every problem of a 40-problem batch (n in [64, 640], p in [4, min(64, n/2)], beta = 1,
    ABB) converges, and the FP64 Cholesky-QR of its last iterate has f = 1/2 sum of the p
    smallest eigenvalues of A (Ky Fan) to 1e-6 and unit feasibility.  PCAL stops at relative KKT
    1e-6; PLAM, whose feasibility comes from the penalty alone, at 1e-5: in FP32 storage one
    problem of the batch (n = 589, p = 64) stalls at 2e-6."""
    from paper_1810_03930_gb300 import BatchSolver
    ws = _problems(40)
    bs = BatchSolver([w.A for w in ws], [w.X0 for w in ws], variant=variant, beta=1.0, tol=tol,
                     maxit=3000)
    infos = bs.solve()
    for w, info, Qd in zip(ws, infos, bs.Q):
        assert info.status == 0 and info.converged, (w.name, info.as_dict())
        assert info.kkt_rel < tol
        Q = to_host(Qd, w.n)
        fstar = 0.5 * np.linalg.eigvalsh(w.A)[: w.p].sum()
        assert abs(oo.TraceObjective(w.A).value(Q) - fstar) <= 1e-6 * abs(fstar), w.name
        assert info.feas_orth <= 1e-12 and op.feasibility(Q) <= 1e-12
    bs.close()


def test_batched_three_iterations_match_oracle():
    """Three PCAL iterations of each problem (edge shapes: p = 1, p = 64, n = 2p, ragged n)
    against the oracle from the same infeasible start: steps and step sizes to FP32 accuracy."""
    from paper_1810_03930_gb300 import BatchSolver
    shapes = [(64, 32), (77, 1), (200, 64), (513, 17), (1000, 40)]
    ws = [workload_batched_problem(100 + b, n, p) for b, (n, p) in enumerate(shapes)]
    rng = np.random.default_rng(3)
    X0s = [w.X0 + 0.02 * rng.standard_normal(w.X0.shape) for w in ws]
    As32 = [w.A.astype(np.float32).astype(np.float64) for w in ws]
    bs = BatchSolver(As32, X0s, beta=1.5, tol=0.0, maxit=3, orthonormalize=False)
    infos = bs.solve()
    for w, A, X0, info, Xd in zip(ws, As32, X0s, infos, bs.X):
        X0f = X0.astype(np.float32).astype(np.float64)
        ref = op.solve(oo.TraceObjective(A), X0f, variant="pcal", beta=1.5, tol=0.0, maxit=3)
        assert info.iters == 3 and info.status == 2          # PLAM_ERR_NOT_CONVERGED at maxit
        X3 = to_host(Xd, w.n)
        assert_entrywise(X3 - X0f, ref.X - X0f, ITER_FACTOR * 1e-4, what=w.name)
        assert abs(info.eta - ref.history[2].eta) <= 1e-4 * ref.history[2].eta
        assert abs(info.kkt_rel - ref.history[3].kkt) <= 1e-4 * ref.history[3].kkt
    bs.close()


def test_batched_agrees_with_the_single_problem_solver():
    from paper_1810_03930_gb300 import BatchSolver
    from tests.gpu_helpers import gpu_solver, to_dev
    ws = _problems(6, n_hi=900, seed_shift=200)
    bs = BatchSolver([w.A for w in ws], [w.X0 for w in ws], tol=1e-6)
    infos = bs.solve()
    for w, info in zip(ws, infos):
        s = gpu_solver(w, "fp32", variant="pcal", beta=1.0, tol=1e-6, maxit=3000, engine="graph")
        st, ref = s.solve(to_dev(w.X0, s))
        # the Barzilai-Borwein sequence is chaotic in rounding: iteration counts of the two
        # kernels' arithmetic differ (e.g. 449 vs 795); the converged objective does not
        assert st == 0 and info.converged
        assert abs(info.f - ref.f) <= 1e-6 * abs(ref.f)
        s.close()
    bs.close()


def test_batched_autotune_and_tiles():
    """The autotuner times each row-block height on the batch, restores the starts and keeps the
    fastest; every tile height gives the same converged objectives."""
    from paper_1810_03930_gb300 import BatchSolver
    ws = _problems(16, seed_shift=300)
    fs = []
    for tile in (64, 128, 256, None):
        bs = BatchSolver([w.A for w in ws], [w.X0 for w in ws], tol=1e-6)
        if tile is None:
            tile, ms = bs.autotune(iters=10)
            assert tile in (64, 128, 256) and ms > 0
        else:
            bs.set_tile(tile)
        infos = bs.solve()
        assert all(i.converged for i in infos)
        fs.append([oo.TraceObjective(w.A).value(to_host(Q, w.n)) for w, Q in zip(ws, bs.Q)])
        bs.close()
    for f in fs[1:]:
        np.testing.assert_allclose(f, fs[0], rtol=1e-6)


def test_batched_rejects_bad_problems():
    from paper_1810_03930_gb300 import BatchSolver, PlamError
    w = workload_batched_problem(0, 200, 64)
    with pytest.raises(PlamError):
        BatchSolver([np.eye(100)], [np.zeros((100, 65))])
    bs = BatchSolver([w.A], [w.X0])
    bs.close()


@pytest.mark.parametrize("variant", ["plam", "pcal"])
def test_batched_parameter_study_reproduces_the_papers_conclusions(variant):
    """The parameter study of Section 5.1 (Figs. 'eta' and 'beta') on the GPU: the 12 seeded trace
    problems of the oracle's parameter-study test (n = 200, p = 8, relative KKT 1e-6) in one
    batched launch per setting.  With beta = s + 0.1 the alternating BB step needs the fewest
    iterations (median, up to 5%) of the rules that converge, the constant step reaches the
    tolerance on none within 3000 iterations, and beta = 10 s + 1 is slower (the smaller steps of
    a large penalty also meet the FP32 noise floor on some problems); the ABB and BB1 medians are
    within 40% of the FP64 oracle's (the BB sequences are chaotic in rounding, and FP32 storage
    moves them).  The rules
    whose quotient carries <Y,Y> feel the FP32 rounding noise of Y = R^k - R^{k-1}: the
    differential rule ||Y||/||S|| still converges but more slowly than in FP64, and pure BB2
    (<Y,Y>/<S,Y>) stalls at relative KKT 1e-6 .. 1e-4 on most problems, while the FP64
    single-problem solve with BB2 converges like the oracle: a property of the storage precision,
    not of the step-size code."""
    from paper_1810_03930_gb300 import BatchSolver, Solver, colmajor_to_device
    from workloads import parameter_study_problems
    As, X0s = parameter_study_problems()
    s = max(float(np.max(np.abs(np.linalg.eigvalsh(A)))) for A in As)

    def batch(beta, rule):
        bs = BatchSolver(As, X0s, variant=variant, beta=beta, eta_rule=rule, tol=1e-6, maxit=3000)
        infos = bs.solve()
        bs.close()
        return infos

    def median(infos):
        return float(np.median([i.iters for i in infos]))

    def oracle(beta, rule, idx=None):
        pairs = list(zip(As, X0s)) if idx is None else [(As[idx], X0s[idx])]
        rs = [op.solve(oo.TraceObjective(A), X0, variant=variant, beta=beta, eta_rule=rule,
                       tol=1e-6, maxit=3000, record=False) for A, X0 in pairs]
        return float(np.median([r.iters for r in rs]))

    runs = {rule: batch(s + 0.1, rule) for rule in ("abb", "bb1", "diff", "bb2", "const")}
    for rule in ("abb", "bb1", "diff"):
        assert all(i.converged for i in runs[rule]), (rule, [i.as_dict() for i in runs[rule]])
        assert median(runs["abb"]) <= 1.05 * median(runs[rule]), {r: median(v) for r, v in runs.items()}
    for rule in ("abb", "bb1"):
        ref = oracle(s + 0.1, rule)
        assert abs(median(runs[rule]) - ref) <= 0.4 * ref, (rule, median(runs[rule]), ref)
    assert not any(i.converged for i in runs["const"])
    stalled = [i for i in runs["bb2"] if not i.converged]
    assert len(stalled) >= len(As) // 2 and all(1e-6 <= i.kkt_rel < 1e-4 for i in stalled), \
        [i.kkt_rel for i in stalled]
    sol = Solver(200, 8, "dense", A=As[0], variant=variant, beta=s + 0.1, eta_rule="bb2", tol=1e-6,
                 maxit=3000, precision="fp64")
    st, info = sol.solve(colmajor_to_device(X0s[0], torch.float64), sol.new_matrix(dtype=torch.float64))
    sol.close()
    ref0 = oracle(s + 0.1, "bb2", idx=0)
    assert st == 0 and info.converged and abs(info.iters - ref0) <= 0.25 * ref0, (info.iters, ref0)
    slow = batch(10 * s + 1, "abb")      # the median counts runs that reach maxit as maxit
    assert median(slow) > 1.3 * median(runs["abb"]), (median(slow), median(runs["abb"]))


def test_full_512_problem_batch_to_kkt_1e6():
    """The batched configuration at full size: 512 problems, n uniform in [64, 2048], p uniform
    in [4, min(64, n/2)], PCAL with beta = 1, ABB, relative KKT 1e-6, maxit 3000, in one launch.
    Every problem either converges or belongs to the expected set the FP32 storage cannot take
    to 1e-6 (R24 of the design notes' readings): those whose spectral gap lambda_{p+1} - lambda_p
    is below 1e-3 |lambda_p| (FP32 rounding of R is then a large part of the Barzilai-Borwein
    differences Y); at most 12 of them, each with its objective within 1e-7 of Ky Fan's optimum.
    The objectives of 32 converged problems spread over the batch (and of the non-converged
    ones) are checked against the eigenvalue sums, and every output is orthonormal."""
    from paper_1810_03930_gb300 import BatchSolver
    shapes = batched_shapes(count=512, n_lo=64, n_hi=2048)
    ws = [workload_batched_problem(b, n, p) for b, (n, p) in enumerate(shapes)]
    bs = BatchSolver([w.A for w in ws], [w.X0 for w in ws], variant="pcal", beta=1.0, tol=1e-6,
                     maxit=3000)
    infos = bs.solve()
    stalled = [b for b, i in enumerate(infos) if not i.converged]
    assert len(stalled) <= 12, stalled
    checked = sorted(set(range(0, 512, 16)) | set(stalled))
    for b in checked:
        w, info = ws[b], infos[b]
        assert info.feas_orth <= 1e-12, (b, info.as_dict())
        ev = np.linalg.eigvalsh(w.A)
        fstar = 0.5 * ev[: w.p].sum()
        f = oo.TraceObjective(w.A).value(to_host(bs.Q[b], w.n))
        if info.converged:
            assert info.kkt_rel < 1e-6
            assert abs(f - fstar) <= 1e-6 * abs(fstar), (b, f, fstar)
        else:
            assert info.status == 2 and info.iters == 3000, (b, info.as_dict())
            assert ev[w.p] - ev[w.p - 1] < 1e-3 * abs(ev[w.p - 1]), (b, ev[w.p - 1], ev[w.p])
            assert abs(f - fstar) <= 1e-7 * abs(fstar), (b, f, fstar)
    print(f"512-problem batch: {512 - len(stalled)} converged, stalled (small gaps): {stalled}")
    bs.close()
