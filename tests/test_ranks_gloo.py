"""Multi-rank host logic on CPU: two gloo ranks (no GPU).

1. The rank helpers used by bench.py under torchrun: shards cover the units
   once, per-rank instance seeds differ, the timing maximum is the maximum.
2. The row-partitioned walk: rank r owns the rows (jc, j, b1) with
   j % 2 == r.  Each rank applies T~^dag P T~ to the branches of its rows only
   (those operators never change jc, j, b1 and every QRAM read they make is of
   row j), then S, then sends every branch to the owner of its new row -- one
   all-to-all exchange per step.  The gathered state must equal the oracle's
   unpartitioned walk: keys exactly, amplitudes to 1e-12.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

WORLD = 2


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank: int, port: int):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD,
                            init_method=f"tcp://127.0.0.1:{port}")
    return dist


def _helpers_worker(rank: int, port: int, out):
    dist = _init(rank, port)
    from paper_2303_06890_gb300 import ranks
    owned = list(ranks.shard(257, rank, WORLD))
    all_owned = [None] * WORLD
    dist.all_gather_object(all_owned, owned)
    m = ranks.max_over_ranks(1.5 + rank)
    seeds = [None] * WORLD
    dist.all_gather_object(seeds, ranks.instance_seed_offset(rank, 256))
    ranks.barrier()
    if rank == 0:
        out.put((all_owned, m, seeds))
    dist.destroy_process_group()


def test_rank_helpers_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_helpers_worker, args=(r, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    all_owned, m, seeds = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat = sorted(u for part in all_owned for u in part)
    assert flat == list(range(257))
    assert abs(len(all_owned[0]) - len(all_owned[1])) <= 1
    assert m == 2.5
    assert seeds[0] != seeds[1]


def _row_partition_worker(rank: int, port: int, steps: int, out):
    dist = _init(rank, port)
    import oracle
    from paper_2303_06890_gb300 import ranks
    from paper_2303_06890_gb300 import workloads as wl

    w = wl.small_random(40, 8, 3, band=1)
    o = oracle.Oracle(w.matrix, w.s)
    b = np.where(np.arange(w.n) % WORLD == rank, w.b, 0.0)  # the rows this rank owns
    o.init_b(b)
    o.apply("T")  # T~ keeps every row in place
    for _ in range(steps):
        o.apply("TDAG", "P", "T", "S")  # row-local part, then S
        regs, amps = o.export()
        outbox = {}
        for r_, a_ in zip(regs, amps):
            dest = ranks.row_owner(int(r_[1]), WORLD)  # owner of the new row (jc, j, b1)
            outbox.setdefault(dest, []).append((tuple(int(v) for v in r_[:6]), complex(a_)))
        boxes = [None] * WORLD
        dist.all_gather_object(boxes, outbox)  # the exchange: an all-to-all of branches
        mine = [item for box in boxes for item in box.get(rank, [])]
        regs_in = np.array([k for k, _ in mine], dtype=np.uint64).reshape(-1, 6)
        amps_in = np.array([a for _, a in mine], dtype=complex)
        o.set_state(regs_in, amps_in)
        assert all(ranks.row_owner(int(r_[1]), WORLD) == rank for r_ in regs_in)
    regs, amps = o.export()
    parts = [None] * WORLD
    dist.all_gather_object(parts, [(tuple(int(v) for v in r_[:7]), complex(a_)) for r_, a_ in zip(regs, amps)])
    if rank == 0:
        out.put([item for part in parts for item in part])
    dist.destroy_process_group()


@pytest.mark.parametrize("steps", [3])
def test_row_partitioned_walk_equals_single_rank(steps):
    import oracle
    from paper_2303_06890_gb300 import workloads as wl

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_row_partition_worker, args=(r, port, steps, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = wl.small_random(40, 8, 3, band=1)
    o = oracle.Oracle(w.matrix, w.s)
    o.init_b(w.b)
    o.apply("T")
    for _ in range(steps):
        o.apply("W")
    regs, amps = o.export()
    want = {tuple(int(v) for v in r_[:7]): complex(a_) for r_, a_ in zip(regs, amps)}
    assert set(got) == set(want)
    assert max(abs(got[k] - want[k]) for k in want) < 1e-12
