"""The row-sharded path's host side on CPU (no GPU): the row plan, the two communicators'
collectives (torch.distributed on gloo ranks, and ranks emulated by threads), and the
decomposition itself — a PCAL solve whose rows are split over two gloo ranks, each rank working
on its own z-slab with halo planes from its neighbours and the Grams and dots summed over the
ranks in rank order, equals the oracle's solve of the whole problem."""
import multiprocessing as mp
import os
import socket
import sys
import threading

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")


def test_shard_rows_plans_whole_units():
    from paper_1810_03930_gb300.dist import shard_rows
    plan = shard_rows(20 * 64, 3, 64)              # 20 z-planes of 64 rows over 3 ranks
    assert plan == [(0, 7 * 64), (7 * 64, 7 * 64), (14 * 64, 6 * 64)]
    plan = shard_rows(10003, 4, 5)                 # blocks of 5, a short last block
    assert sum(n for _, n in plan) == 10003
    assert all(r0 % 5 == 0 for r0, _ in plan) and all(n % 5 == 0 for _, n in plan[:-1])
    assert [r0 + n for r0, n in plan[:-1]] == [r0 for r0, _ in plan[1:]]
    with pytest.raises(ValueError):
        shard_rows(3 * 64, 4, 64)                  # fewer planes than ranks


def _check_collectives(rank, size, member):
    send = torch.arange(4, dtype=torch.float64) + 10.0 * rank
    recv = torch.full((4 * size,), -1.0, dtype=torch.float64)
    member.allgather(send, recv)
    assert torch.equal(recv, torch.cat([torch.arange(4, dtype=torch.float64) + 10.0 * r
                                        for r in range(size)]))
    lo, hi = torch.full((3,), 100.0 * rank + 1), torch.full((3,), 100.0 * rank + 2)
    rlo, rhi = torch.full((3,), -1.0), torch.full((3,), -1.0)
    member.exchange(lo, hi, rlo, rhi)
    # the lower neighbour's last plane and the upper neighbour's first; nothing at the ends
    assert torch.all(rlo == (100.0 * (rank - 1) + 2 if rank > 0 else -1.0))
    assert torch.all(rhi == (100.0 * (rank + 1) + 1 if rank < size - 1 else -1.0))


def test_local_comm_collectives_on_threads():
    from paper_1810_03930_gb300.dist import LocalComm
    size = 3
    comm = LocalComm(size, timeout=30)
    errs = []

    def work(r):
        try:
            _check_collectives(r, size, comm.member(r))
        except Exception as e:      # noqa: BLE001
            errs.append(e)
            comm.barrier.abort()

    ts = [threading.Thread(target=work, args=(r,)) for r in range(size)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errs, errs


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _spawn(target, size, *args):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, size, port, q, *args)) for r in range(size)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


def _init(rank, size, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=size)
    return dist


def _collectives_worker(rank, size, port, q):
    dist = _init(rank, size, port)
    from paper_1810_03930_gb300.dist import TorchDistComm
    try:
        _check_collectives(rank, size, TorchDistComm())
        q.put((rank, "ok"))
    except Exception as e:          # noqa: BLE001
        q.put((rank, repr(e)))
    dist.barrier()
    dist.destroy_process_group()


def test_torch_dist_comm_collectives_on_three_gloo_ranks():
    out = _spawn(_collectives_worker, 3)
    assert [o[1] for o in out] == ["ok"] * 3, out


def _sharded_pcal(member, m, V, X0, beta, tol, maxit):
    """PCAL (eq. lambda2, ABB) on this rank's z-slab of an m^3 stencil problem: the gradient
    from the slab extended by the neighbours' halo planes, every inner product over all rows
    summed over the ranks in rank order.  Returns (eta, kkt, f) per iteration and the rows of
    the orthonormalised result."""
    from oracle import objectives as oo
    from oracle import plam as op
    from paper_1810_03930_gb300.dist import shard_rows
    plane = m * m
    row0, nl = shard_rows(m ** 3, member.size, plane)[member.rank]
    nzl = nl // plane
    p = X0.shape[1]
    Vext = np.zeros(nl + 2 * plane)
    Vext[plane:plane + nl] = V[row0:row0 + nl]
    H = oo.Stencil3DObjective((m, m, nzl + 2), Vext)

    def allsum(a):
        a = np.asarray(a, dtype=np.float64)
        recv = torch.empty(a.size * member.size, dtype=torch.float64)
        member.allgather(torch.as_tensor(a.ravel().copy()), recv)
        parts = recv.numpy().reshape(member.size, -1)
        tot = parts[0].copy()
        for r in range(1, member.size):
            tot += parts[r]
        return tot.reshape(a.shape)

    def grad(X):
        lo = torch.as_tensor(X[:plane].copy())
        hi = torch.as_tensor(X[-plane:].copy())
        rlo, rhi = torch.zeros_like(lo), torch.zeros_like(hi)
        member.exchange(lo, hi, rlo, rhi)
        Xe = np.vstack([rlo.numpy(), X, rhi.numpy()])
        return H.grad(Xe)[plane:plane + nl]

    X = X0[row0:row0 + nl].copy()
    I = np.eye(p)
    hist, Xp, Rp, eta = [], None, None, None
    K0 = None
    for k in range(maxit + 1):
        G = grad(X)
        B = allsum(X.T @ X)
        C = allsum(X.T @ G)
        L0 = op.psi(C)
        kk2 = allsum(np.sum((G - X @ L0) ** 2))
        K0 = np.sqrt(kk2) if K0 is None else K0
        kkt = np.sqrt(kk2) / K0
        f = 0.5 * np.trace(C)
        if kkt < tol:
            hist.append((np.nan, kkt, f))
            break
        d = np.diag(C) - np.sum(B * L0, axis=0) + beta * (np.sum(B * B, axis=0) - np.diag(B))
        R = G - X @ (L0 + np.diag(d)) + beta * X @ (B - I)
        if k == 0:
            eta = np.sqrt(allsum(np.sum(G * G)) / allsum(np.sum(X * X))) + beta
        else:
            S, Y = X - Xp, R - Rp
            ss, sy, yy = allsum(np.array([np.sum(S * S), np.sum(S * Y), np.sum(Y * Y)]))
            eta = abs(sy) / ss if k % 2 else yy / abs(sy)
        hist.append((eta, kkt, f))
        Xp, Rp = X, R
        V1 = X - R / eta
        X = V1 / np.sqrt(allsum(np.sum(V1 * V1, axis=0)))[None, :]
    Rc = np.linalg.cholesky(allsum(X.T @ X)).T
    return np.array(hist), np.linalg.solve(Rc.T, X.T).T, row0


def _decomposition_worker(rank, size, port, q, m, p):
    dist = _init(rank, size, port)
    from oracle import objectives as oo
    from oracle import plam as op
    from paper_1810_03930_gb300.dist import TorchDistComm
    from workloads import orthonormal_start, rng_for
    V = rng_for(31, 0).uniform(0.0, 1.0, m ** 3)
    X0 = orthonormal_start(m ** 3, p, rng_for(31, 1))
    beta = 12.0 + V.max() + 0.1
    hist, Qr, row0 = _sharded_pcal(TorchDistComm(), m, V, X0, beta, 1e-9, 4000)
    ref = op.solve(oo.Stencil3DObjective(m, V), X0, variant="pcal", beta=beta, tol=1e-9,
                   maxit=4000)
    q.put((rank, hist, Qr, row0, [h.eta for h in ref.history], [h.kkt for h in ref.history],
           ref.iters, ref.f_orth))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_pcal_on_two_gloo_ranks_matches_the_oracle():
    """10^3 grid, p = 6 (5 z-planes per rank), FP64 to relative KKT 1e-9."""
    from oracle import objectives as oo
    from workloads import rng_for
    m, p = 10, 6
    out = _spawn(_decomposition_worker, 2, m, p)
    h0, h1 = out[0][1], out[1][1]
    assert np.array_equal(h0, h1, equal_nan=True)    # both ranks took the same steps
    eta_ref, kkt_ref, iters_ref, f_ref = out[0][4], out[0][5], out[0][6], out[0][7]
    k = min(20, len(h0) - 1)
    np.testing.assert_allclose(h0[:k, 0], eta_ref[:k], rtol=1e-9)
    np.testing.assert_allclose(h0[:k, 1], kkt_ref[:k], rtol=1e-8)
    assert abs((len(h0) - 1) - iters_ref) <= max(5, 0.25 * iters_ref)
    Q = np.zeros((m ** 3, p))
    for _, _, Qr, row0, *_ in out:
        Q[row0:row0 + Qr.shape[0]] = Qr
    V = rng_for(31, 0).uniform(0.0, 1.0, m ** 3)
    f = oo.Stencil3DObjective(m, V).value(Q)
    assert abs(f - f_ref) <= 1e-10 * abs(f_ref)
    assert np.abs(Q.T @ Q - np.eye(p)).max() <= 1e-12
