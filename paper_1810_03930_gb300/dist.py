"""Row-sharded PCAL/PLAM solves across ranks (one process per GPU): the Python side of
plam_create_sharded (include/plam.h).

The rows of X, G and R are split into contiguous blocks (Section 5.4's parallel structure:
everything O(np) and O(np^2) stays on a rank's rows); the library calls back, per iteration,
for one all-gather of the reduced Grams [X^T X | X^T G] and one of the column and
Barzilai-Borwein dots, and, for the 3D stencil, one exchange of halo z-planes with the
neighbouring ranks.  This module only plans the row blocks and turns a communicator into those
callbacks; the sums over the ranks (in rank order) and all arithmetic happen in the library.

Communicators:
  TorchDistComm  torch.distributed (NCCL for device tensors across GPUs, gloo for host tensors)
  LocalComm      `size` ranks emulated by host threads of one process, for testing the sharded
                 path on one device: the collectives meet at a host barrier and move data
                 through host memory, so no kernel ever waits for another rank's kernel.
"""
from __future__ import annotations

import ctypes as C
import threading

from . import _lib

__all__ = ["shard_rows", "TorchDistComm", "LocalComm", "comm_struct", "ShardedStencil",
           "sharded_solver"]


def shard_rows(n_global: int, size: int, unit: int = 1) -> list[tuple[int, int]]:
    """(row0, n_local) of each of `size` ranks: contiguous blocks of whole units (z-planes of a
    stencil grid, or blocks of a block-diagonal L; the last unit may be shorter), the first
    (units mod size) ranks taking one unit more."""
    if size < 1 or unit < 1 or n_global < 1:
        raise ValueError("size, unit and n_global must be positive")
    units = (n_global + unit - 1) // unit
    if units < size:
        raise ValueError(f"{units} units of {unit} rows cannot feed {size} ranks")
    base, extra = divmod(units, size)
    out, u0 = [], 0
    for r in range(size):
        cnt = base + (1 if r < extra else 0)
        row0 = u0 * unit
        row1 = min(n_global, (u0 + cnt) * unit)
        out.append((row0, row1 - row0))
        u0 += cnt
    return out


class TorchDistComm:
    """The all-gather and the halo exchange over a torch.distributed process group."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)

    def allgather(self, send, recv):
        """recv (size * count) receives every rank's send (count), in rank order."""
        parts = list(recv.view(self.size, -1).unbind(0))
        self.dist.all_gather(parts, send, group=self.group)

    def exchange(self, send_lo, send_hi, recv_lo, recv_hi):
        """send_lo to rank - 1 and send_hi to rank + 1; recv_lo from rank - 1 (its send_hi) and
        recv_hi from rank + 1 (its send_lo).  Missing neighbours are skipped."""
        dist = self.dist
        ops = []
        if self.rank > 0:
            peer = dist.get_global_rank(self.group, self.rank - 1) if self.group else self.rank - 1
            ops += [dist.P2POp(dist.isend, send_lo, peer, self.group),
                    dist.P2POp(dist.irecv, recv_lo, peer, self.group)]
        if self.rank < self.size - 1:
            peer = dist.get_global_rank(self.group, self.rank + 1) if self.group else self.rank + 1
            ops += [dist.P2POp(dist.isend, send_hi, peer, self.group),
                    dist.P2POp(dist.irecv, recv_hi, peer, self.group)]
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()


class LocalComm:
    """`size` ranks emulated by host threads of one process.  member(r) is rank r's view."""

    def __init__(self, size: int, timeout: float = 120.0):
        self.size = size
        self.barrier = threading.Barrier(size, timeout=timeout)
        self.slots = [None] * size

    def member(self, rank: int) -> "LocalMember":
        return LocalMember(self, rank)


class LocalMember:
    def __init__(self, comm: LocalComm, rank: int):
        self.comm, self.rank, self.size = comm, rank, comm.size

    def _post(self, *tensors):
        import torch
        if tensors[0].is_cuda:
            torch.cuda.current_stream().synchronize()
        self.comm.slots[self.rank] = [t.detach().to("cpu", copy=True) for t in tensors]
        self.comm.barrier.wait()

    def allgather(self, send, recv):
        import torch
        self._post(send)
        out = torch.cat([s[0] for s in self.comm.slots])
        recv.copy_(out.to(recv.device))
        if recv.is_cuda:
            torch.cuda.current_stream().synchronize()
        self.comm.barrier.wait()          # nobody posts again before every rank has read

    def exchange(self, send_lo, send_hi, recv_lo, recv_hi):
        import torch
        self._post(send_lo, send_hi)
        if self.rank > 0:
            recv_lo.copy_(self.comm.slots[self.rank - 1][1].to(recv_lo.device))
        if self.rank < self.size - 1:
            recv_hi.copy_(self.comm.slots[self.rank + 1][0].to(recv_hi.device))
        if recv_lo.is_cuda:
            torch.cuda.current_stream().synchronize()
        self.comm.barrier.wait()


def _device_view(ptr: int, count: int, dtype):
    """count elements of `dtype` at device address ptr as a 1-D torch tensor (zero copy)."""
    import torch
    esz = torch.empty((), dtype=dtype).element_size()
    typestr = {torch.float64: "<f8", torch.float32: "<f4"}[dtype]

    class _Buf:
        pass
    b = _Buf()
    b.__cuda_array_interface__ = {"shape": (count,), "strides": (esz,), "typestr": typestr,
                                  "data": (int(ptr), False), "version": 3}
    return torch.as_tensor(b, device="cuda")


def comm_struct(member, row0: int, n_global: int, dtype):
    """The plam_comm_t of one rank: its callbacks wrap the library's device buffers as tensors
    and call member.allgather / member.exchange with the library's stream current.  Returns
    (struct, keep-alive list); a failing callback returns 1 (the entry point then reports
    PLAM_ERR_CUDA) and leaves the exception in keep[-1]['error']."""
    import torch
    state = {"error": None}

    def on_stream(stream):
        return torch.cuda.stream(torch.cuda.ExternalStream(stream)) if stream else torch.cuda.stream(
            torch.cuda.default_stream())

    def allgather(ctx, send, recv, count, stream):
        try:
            with on_stream(stream):
                member.allgather(_device_view(send, count, torch.float64),
                                 _device_view(recv, count * member.size, torch.float64))
            return 0
        except Exception as e:         # reported through the entry point's status
            state["error"] = e
            return 1

    def exchange(ctx, send_lo, send_hi, recv_lo, recv_hi, count, stream):
        try:
            with on_stream(stream):
                member.exchange(*(_device_view(p, count, dtype)
                                  for p in (send_lo, send_hi, recv_lo, recv_hi)))
            return 0
        except Exception as e:
            state["error"] = e
            return 1

    ag = _lib.plam_allgather_fn(allgather)
    ex = _lib.plam_exchange_fn(exchange)
    s = _lib.plam_comm_t(member.rank, member.size, row0, n_global, ag, ex, None)
    return s, [ag, ex, state]


class ShardedStencil:
    """This rank's z-slab of an nx x ny x nz stencil problem: rows [row0, row0 + n_local) of
    the global index x + nx (y + ny z), planes [z0, z0 + nz_local)."""

    def __init__(self, grid, rank: int, size: int):
        self.nx, self.ny, self.nz = grid
        self.plane = self.nx * self.ny
        self.n_global = self.plane * self.nz
        self.row0, self.n_local = shard_rows(self.n_global, size, self.plane)[rank]
        self.z0, self.nz_local = self.row0 // self.plane, self.n_local // self.plane
        self.rank, self.size = rank, size

    def new_x(self, p: int, dtype):
        """A (p, ld) tensor for this rank's X with a halo plane before and after the local rows
        (ld a multiple of 32 elements); returns (storage, the (p, n_local) view of the local rows,
        whose data pointer and leading dimension are what the library's calls take)."""
        import torch
        ld = (self.n_local + 2 * self.plane + 31) // 32 * 32
        buf = torch.zeros((p, ld), dtype=dtype, device="cuda")
        return buf, buf[:, self.plane:self.plane + self.n_local]


def sharded_solver(member, kind: str, n_local: int, p: int, row0: int, n_global: int, **kw):
    """A Solver on this rank's rows (plam_create_sharded): kind "stencil3d" (grid = this rank's
    slab, V its potential) or "hartree1d" (block >= 1, lin its rows)."""
    import torch
    from . import Solver, storage_dtype
    dtype = storage_dtype(kw.get("precision", "fp64"))
    shard = comm_struct(member, row0, n_global, dtype)
    kw.setdefault("graph_iters", 0)
    kw.setdefault("orth_metrics", False)
    return Solver(n_local, p, kind, shard=shard, **kw)
