"""Row-partitioned walk: ownership, the exchange of S's sends, and its drivers.

T~^dag, P and T~ never change the registers (jc, j, b1) and read only row j of
the QRAM (Sec. IV), so a simulator holding a set of rows advances them alone;
S moves a branch to row (kc, k, b2), which may belong to another partition --
the one exchange of a step.  Ownership is the rule of ``qw_part_owner`` in
``libqwalk.so`` (blocks of ceil(N / P) rows for jc = 0, j < N; a hash of
(jc, j) otherwise).

Drivers (argument marshalling and the exchange only; every walk step runs in
the library's kernels):

* ``walk_in_process(sims, steps)``: P simulators of one process on one device,
  ``qw_part_walk`` -- the exchange by cudaMemcpyAsync inside the library;
* ``walk_partitioned(engine, steps, group)``: one partition per rank of a
  ``torch.distributed`` group.  Per step: ``engine.step()`` returns the
  entries S sent to each other partition, ``exchange`` delivers them (an
  all-to-all), ``engine.inbox`` appends what arrived, and the norms of the
  parts are summed for the renormalisation.  ``SimEngine`` adapts a
  partitioned ``qwalk.Sim``; any object with the same four methods drives the
  same loop.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import qwalk

# one entry of an outbox or inbox (qw_part_entry, 32 bytes)
ENTRY = np.dtype([("rowkey", "<u8"), ("local", "<u8"), ("re", "<f8"), ("im", "<f8")])


def owner(n: int, nparts: int, jc: int, j: int) -> int:
    """Partition owning row (jc, j) of an N-row walk split nparts ways."""
    r = qwalk.load().qw_part_owner(int(n), int(nparts), int(jc), int(j))
    if r < 0:
        raise ValueError("bad row or partition count")
    return r


def owners(n: int, nparts: int, jc: np.ndarray, j: np.ndarray) -> np.ndarray:
    """owner() of many rows."""
    lib = qwalk.load()
    return np.array([lib.qw_part_owner(int(n), int(nparts), int(a), int(b)) for a, b in zip(jc, j)], dtype=np.int64)


def rowkey(jc, j, b1, inst=0):
    """Row key of an entry: inst << 40 | jc << 20 | j << 1 | b1."""
    return (np.uint64(inst) << np.uint64(40)) | (np.asarray(jc, np.uint64) << np.uint64(20)) | \
        (np.asarray(j, np.uint64) << np.uint64(1)) | np.asarray(b1, np.uint64)


def walk_in_process(sims: list, steps: int) -> None:
    """qw_part_walk over partitions 0 .. P-1 of one walk (one device)."""
    arr = (ctypes.c_void_p * len(sims))(*[s._h for s in sims])
    rc = qwalk.load().qw_part_walk(arr, len(sims), int(steps))
    if rc:
        raise qwalk.QwError(rc, qwalk.load().qw_last_error(sims[0]._h).decode())


def exchange(boxes: list, group=None) -> np.ndarray:
    """Deliver boxes[q] (ENTRY arrays) from this rank to rank q; return what
    every rank sent here.  An all-to-all: device tensors over NCCL, host
    objects over other backends."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    if dist.get_backend(group) == "nccl":
        dev = torch.device("cuda", torch.cuda.current_device())
        send_counts = torch.tensor([len(b) for b in boxes], dtype=torch.int64, device=dev)
        recv_counts = torch.empty(world, dtype=torch.int64, device=dev)
        dist.all_to_all_single(recv_counts, send_counts, group=group)
        rc = [int(c) for c in recv_counts.tolist()]
        send = torch.from_numpy(np.concatenate(boxes).view(np.uint8).copy()).to(dev)
        recv = torch.empty(sum(rc) * ENTRY.itemsize, dtype=torch.uint8, device=dev)
        dist.all_to_all_single(recv, send, [c * ENTRY.itemsize for c in rc],
                               [len(b) * ENTRY.itemsize for b in boxes], group=group)
        return recv.cpu().numpy().view(ENTRY)
    gathered = [None] * world
    dist.all_gather_object(gathered, boxes, group=group)
    me = dist.get_rank(group)
    parts = [g[me] for g in gathered if len(g[me])]
    return np.concatenate(parts) if parts else np.zeros(0, ENTRY)


def walk_partitioned(engine, steps: int, group=None) -> None:
    """``steps`` walk steps of a partitioned walk, this rank's part driven by
    ``engine`` (step / inbox / norm / set_norm)."""
    import torch
    import torch.distributed as dist

    for _ in range(int(steps)):
        boxes = engine.step()
        engine.inbox(exchange(boxes, group))
        local = torch.tensor([engine.norm()], dtype=torch.float64,
                             device="cuda" if dist.get_backend(group) == "nccl" else "cpu")
        dist.all_reduce(local, group=group)
        engine.set_norm(float(local.item()))


class SimEngine:
    """A partitioned ``qwalk.Sim`` as the engine of ``walk_partitioned``:
    outboxes are copied out of the library into host arrays, received entries
    are handed back through a device staging buffer."""

    def __init__(self, sim, nparts: int, part: int):
        self.sim, self.nparts, self.part = sim, nparts, part

    def step(self) -> list:
        import torch

        lib = qwalk.load()
        self.sim.enqueue_walk_steps(1)
        self.sim.sync()
        boxes = []
        for q in range(self.nparts):
            if q == self.part:
                boxes.append(np.zeros(0, ENTRY))
                continue
            count = ctypes.c_int64()
            rc = lib.qw_part_outbox(self.sim._h, q, None, 0, ctypes.byref(count))
            self.sim._check(rc)
            buf = torch.empty(max(1, count.value) * ENTRY.itemsize, dtype=torch.uint8, device="cuda")
            self.sim._check(lib.qw_part_outbox(self.sim._h, q, ctypes.c_void_p(buf.data_ptr()), count.value,
                                               ctypes.byref(count)))
            boxes.append(buf[:count.value * ENTRY.itemsize].cpu().numpy().view(ENTRY).copy())
        return boxes

    def inbox(self, entries: np.ndarray) -> None:
        import torch

        if len(entries) == 0:
            return
        dev = torch.from_numpy(np.ascontiguousarray(entries).view(np.uint8)).to("cuda")
        self.sim._check(qwalk.load().qw_part_inbox(self.sim._h, ctypes.c_void_p(dev.data_ptr()), len(entries)))

    def norm(self) -> float:
        v = ctypes.c_double()
        self.sim._check(qwalk.load().qw_part_norm(self.sim._h, ctypes.byref(v)))
        return v.value

    def set_norm(self, global_norm2: float) -> None:
        self.sim._check(qwalk.load().qw_part_set_norm(self.sim._h, float(global_norm2)))
