"""The CTA-pair tensor-core Gram (p >= 256: one 256 x 256 tile per pair of CTAs, tcgen05
cta_group::2) against the definition of X^T X and X^T G (Table "cost"), entry by entry, and
against the single-CTA kernel it replaces, on ragged shapes: n not a multiple of the 32-row
stage, p not a multiple of the 256-column tile (the second CTA of the last pair reads columns
past p), and the B-only form (no G).

TF32 products carry up to 2.2 * 2^-10 relative error per product; compensated 3xTF32 about
2^-21; each bound below is that per-product error on |X|^T |Y| plus the FP32 accumulation."""
import numpy as np
import pytest

from tests.gpu_helpers import to_dev
from workloads import orthonormal_start

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _solver(n, p, tc):
    from paper_1810_03930_gb300 import Solver
    return Solver(n, p, "hartree1d", precision="fp32", tensor_cores=tc)


def _bounds(X, Y, n, mode):
    a = np.abs(X).T @ np.abs(Y)
    if mode == "tf32":
        return 2.2 * 2.0 ** -10 * a + 1e-5 * np.sqrt(n)
    return 4 * 2.0 ** -21 * a + 2e-6 * np.sqrt(n)


@pytest.mark.parametrize("n,p", [(8191, 256), (2051, 300), (4133, 520), (12000, 1024)])
@pytest.mark.parametrize("mode", ["tf32", "3xtf32"])
def test_pair_grams_match_definition_and_single_cta(n, p, mode):
    rng = np.random.default_rng(31 * n + p)
    X = rng.standard_normal((n, p)).astype(np.float32).astype(np.float64)
    G = rng.standard_normal((n, p)).astype(np.float32).astype(np.float64)
    ld = (n + 31) // 32 * 32
    s = _solver(n, p, mode)
    s1 = _solver(n, p, mode + "-single")
    Xd, Gd = to_dev(X, s, ld=ld), to_dev(G, s, ld=ld)
    B, Cm = (t.cpu().numpy() for t in s.grams(Xd, Gd))
    B1, C1 = (t.cpu().numpy() for t in s1.grams(Xd, Gd))
    Bref, Cref = X.T @ X, X.T @ G
    tolB, tolC = _bounds(X, X, n, mode), _bounds(X, G, n, mode)
    for got, ref, tol, what in ((B, Bref, tolB, "B pair"), (Cm, Cref, tolC, "C pair"),
                                (B1, Bref, tolB, "B single"), (C1, Cref, tolC, "C single")):
        bad = np.abs(got - ref) > tol
        assert not bad.any(), (what, np.argwhere(bad)[:5])
    # B is symmetric by construction (the lower triangle mirrors the computed upper one)
    assert np.array_equal(B, B.T)
    # the pair kernel's partial sums are its own: different tiles and chunks from the
    # single-CTA kernel, so the results differ in the last bits somewhere
    assert not np.array_equal(Cm, C1)
    # fixed-order reduction: bitwise reproducible
    B2, C2 = (t.cpu().numpy() for t in s.grams(Xd, Gd))
    assert np.array_equal(B, B2) and np.array_equal(Cm, C2)
    s.close()
    s1.close()


@pytest.mark.parametrize("mode", ["tf32", "3xtf32"])
def test_pair_gram_without_g(mode):
    n, p = 6007, 384
    X = orthonormal_start(n, p, np.random.default_rng(2)).astype(np.float32).astype(np.float64)
    s = _solver(n, p, mode)
    B, _ = s.grams(to_dev(X, s, ld=n + 1 + (-(n + 1)) % 4))
    B = B.cpu().numpy()
    assert np.all(np.abs(B - X.T @ X) <= _bounds(X, X, n, mode))
    s.close()


def test_pair_compensated_grams_have_no_accumulation_drift():
    """Compensated mode sums every 32-row segment from zero in TMEM and adds the segments into
    register totals with round-to-nearest FP32: a long same-signed sum (a diagonal of X^T X)
    keeps its relative drift at a few 1e-7."""
    n, p = 131072, 256
    X = np.random.default_rng(9).standard_normal((n, p)).astype(np.float32).astype(np.float64)
    s = _solver(n, p, "3xtf32")
    B, _ = s.grams(to_dev(X, s, ld=n))
    ref = np.sum(X * X, axis=0)
    d = (np.diag(B.cpu().numpy()) - ref) / ref
    assert abs(d.mean()) < 1e-6
    assert np.abs(d).max() < 2e-6
    s.close()


def test_pair_tf32_diagonal_is_unbiased():
    """Plain TF32 mode sums segments of 8 stages (256 rows) before adding them into the
    register totals, so the truncating accumulator does not pull the unit diagonal of an
    orthonormal X low over a long chunk (the single-CTA kernel, one segment per chunk, drifts
    by about -1e-3 at 5e5 rows)."""
    n, p = 262144, 256
    X = orthonormal_start(n, p, np.random.default_rng(5)).astype(np.float32).astype(np.float64)
    s = _solver(n, p, "tf32")
    B, _ = s.grams(to_dev(X, s, ld=n))
    d = np.diag(B.cpu().numpy()) - np.sum(X * X, axis=0)
    assert abs(d.mean()) < 2e-5
    s.close()
