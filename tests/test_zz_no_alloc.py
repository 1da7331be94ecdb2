"""plam_grams_noalloc: the Grams for callers that cannot allocate device memory.

It must give the same B = X^T X and C = X^T G as plam_grams (the handle-based
entry point): bit for bit where its scratch does not cap the row chunks (both
entry points plan the chunks with one rule), within the Gram tolerances of
tests/test_gpu_parity.py where it does, on two calls in a row with different
shapes (the second call reuses the static scratch the first one filled); it
must handle the largest p its scratch admits and reject larger requests, and
every rejection leaves a message.
Collected last on purpose (file name), so a failure here leaves every other
test already run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _handle_grams(precision, X, G):
    from tests.gpu_helpers import gpu_solver, to_dev
    from workloads import Workload
    n, p = X.shape
    w = Workload(name="grams", kind="hartree1d", n=n, p=p, X0=X)
    s = gpu_solver(w, precision, tensor_cores="off")
    B, Cm = s.grams(to_dev(X, s), to_dev(G, s) if G is not None else None)
    s.close()
    return B.cpu().numpy(), (Cm.cpu().numpy() if Cm is not None else None)


def _noalloc_grams(precision, X, G):
    from paper_1810_03930_gb300 import _lib
    from tests.gpu_helpers import to_dev
    n, p = X.shape
    dtype = torch.float64 if precision == "fp64" else torch.float32

    class _S:
        pass
    s = _S()
    s.dtype = dtype
    Xd = to_dev(X, s)
    Gd = to_dev(G, s) if G is not None else None
    B = torch.full((p, p), float("nan"), dtype=torch.float64, device="cuda")
    Cm = torch.full((p, p), float("nan"), dtype=torch.float64, device="cuda") if G is not None else None
    prec = _lib.PLAM_PREC_FP64 if precision == "fp64" else _lib.PLAM_PREC_FP32
    st = _lib.plam_grams_noalloc(n, p, prec, Xd.data_ptr(), Xd.stride(0),
                                 Gd.data_ptr() if Gd is not None else None,
                                 Gd.stride(0) if Gd is not None else 0, B.data_ptr(),
                                 Cm.data_ptr() if Cm is not None else None,
                                 torch.cuda.current_stream().cuda_stream)
    assert st == _lib.PLAM_OK, _lib.load().plam_last_error()
    torch.cuda.synchronize()
    del Xd, Gd
    # column-major p x p outputs held in (p, p) row-major tensors: transpose back
    return B.t().cpu().numpy(), (Cm.t().cpu().numpy() if Cm is not None else None)


def _close(a, b, n, precision):
    tol = 1e-12 if precision == "fp64" else 2e-6
    scale = np.sqrt(n)
    return np.abs(a - b).max() <= tol * scale * max(1.0, np.abs(b).max() / scale)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_grams_match_plam_grams_on_two_calls_in_a_row(precision):
    rng = np.random.default_rng(2024)
    shapes = [(4099, 65, True), (3001, 20, False), (2051, 33, True)]
    for n, p, with_g in shapes:
        X = rng.standard_normal((n, p))
        G = rng.standard_normal((n, p)) if with_g else None
        if precision == "fp32":
            X = X.astype(np.float32).astype(np.float64)
            if G is not None:
                G = G.astype(np.float32).astype(np.float64)
        B_ref, C_ref = _handle_grams(precision, X, G)
        B, Cm = _noalloc_grams(precision, X, G)
        # the scratch does not cap these chunkings: the same reduction order, bit for bit
        assert np.array_equal(B, B_ref), (n, p)
        if with_g:
            assert np.array_equal(Cm, C_ref), (n, p)
            assert _close(Cm, X.T @ G, n, precision)
        # and against the definition
        assert _close(B, X.T @ X, n, precision)


@pytest.mark.parametrize("precision,n,p", [("fp64", 1500, 724), ("fp32", 2100, 1024),
                                           ("fp64", 40000, 300)])
def test_noalloc_grams_at_the_largest_p_and_where_the_scratch_caps_the_chunks(precision, n, p):
    """p = 724 (FP64) and p = 1024 (FP32) fill the 8 MiB scratch with one row chunk; at FP64
    p = 300 the handle's rule asks for 8 chunks and the scratch holds 5, so the cap binds."""
    rng = np.random.default_rng(7 + p)
    X = rng.standard_normal((n, p))
    G = rng.standard_normal((n, p)) if p < 1000 else None
    if precision == "fp32":
        X = X.astype(np.float32).astype(np.float64)
    for _ in range(2):          # two calls in a row on the shared scratch
        B, Cm = _noalloc_grams(precision, X, G)
        assert _close(B, X.T @ X, n, precision), (n, p)
        if G is not None:
            assert _close(Cm, X.T @ G, n, precision), (n, p)
    B_ref, C_ref = _handle_grams(precision, X, G)
    assert _close(B, B_ref, n, precision)
    if G is not None:
        assert _close(Cm, C_ref, n, precision)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1810_03930_gb300 import _lib
    X = torch.zeros((1100, 4000), dtype=torch.float32, device="cuda")   # p = 1100 > 1024 (FP32 limit)
    B = torch.zeros((1100, 1100), dtype=torch.float64, device="cuda")
    st = _lib.plam_grams_noalloc(4000, 1100, _lib.PLAM_PREC_FP32, X.data_ptr(), 4000, None, 0,
                                 B.data_ptr(), None, 0)
    assert st == _lib.PLAM_ERR_INVALID
    assert b"8 MiB" in _lib.load().plam_last_error()
    Xd = torch.zeros((800, 2000), dtype=torch.float64, device="cuda")   # p = 800 > 724 (FP64 limit)
    Bd = torch.zeros((800, 800), dtype=torch.float64, device="cuda")
    st = _lib.plam_grams_noalloc(2000, 800, _lib.PLAM_PREC_FP64, Xd.data_ptr(), 2000, None, 0,
                                 Bd.data_ptr(), None, 0)
    assert st == _lib.PLAM_ERR_INVALID
    st = _lib.plam_grams_noalloc(2000, 725, _lib.PLAM_PREC_FP64, Xd.data_ptr(), 2000, None, 0,
                                 Bd.data_ptr(), None, 0)         # p = 725: one past the FP64 limit
    assert st == _lib.PLAM_ERR_INVALID
    assert b"8 MiB" in _lib.load().plam_last_error()
    # argument errors leave their own message (not a stale one)
    st = _lib.plam_grams_noalloc(2000, 8, _lib.PLAM_PREC_FP64, Xd.data_ptr(), 1999, None, 0,
                                 Bd.data_ptr(), None, 0)
    assert st == _lib.PLAM_ERR_INVALID
    assert b"leading dimension" in _lib.load().plam_last_error()
