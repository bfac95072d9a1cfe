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


class OracleEngine:
    """The CPU oracle as the engine of the product's partitioned-walk loop
    (paper_2303_06890_gb300.partition.walk_partitioned): this rank's rows of
    the state, T~^dag P T~ and S on them, and the entries S sends away."""

    def __init__(self, w, nparts, part):
        import oracle
        from paper_2303_06890_gb300 import partition
        self.w, self.nparts, self.part, self.P = w, nparts, part, partition
        self.o = oracle.Oracle(w.matrix, w.s)
        own = partition.owners(w.n, nparts, np.zeros(w.n, np.int64), np.arange(w.n)) == part
        self.o.init_b(np.where(own, w.b, 0.0))  # the rows this rank owns
        self.o.apply("T")  # T~ keeps every row in place
        self.kept = None
        self.emitted = 0.0

    def step(self):
        P = self.P
        self.o.apply("TDAG", "P", "T", "S")  # the row-local part, then S
        self.emitted = self.o.norm2()
        regs, amps = self.o.export()
        dest = P.owners(self.w.n, self.nparts, regs[:, 0], regs[:, 1])  # owner of the new row (jc, j)
        mine = dest == self.part
        self.kept = (regs[mine, :6], amps[mine])
        nb = self.o.nb
        boxes = []
        for q in range(self.nparts):
            sel = (dest == q) & ~mine
            e = np.zeros(int(sel.sum()), P.ENTRY)
            r = regs[sel]
            e["rowkey"] = P.rowkey(r[:, 0], r[:, 1], r[:, 2])
            e["local"] = r[:, 5] | (r[:, 4] << np.uint64(1)) | (r[:, 3] << np.uint64(1 + nb))
            e["re"], e["im"] = amps[sel].real, amps[sel].imag
            boxes.append(e)
        return boxes

    def inbox(self, entries):
        nb = self.o.nb
        m = np.uint64((1 << nb) - 1)
        rk, lk = entries["rowkey"], entries["local"]
        regs_in = np.stack([(rk >> np.uint64(20)) & np.uint64(0xfffff), (rk >> np.uint64(1)) & np.uint64(0x7ffff),
                            rk & np.uint64(1), (lk >> np.uint64(1 + nb)) & m, (lk >> np.uint64(1)) & m,
                            lk & np.uint64(1)], axis=1).astype(np.uint64)
        assert all(self.P.owner(self.w.n, self.nparts, int(r[0]), int(r[1])) == self.part for r in regs_in)
        regs = np.concatenate([self.kept[0], regs_in])
        amps = np.concatenate([self.kept[1], entries["re"] + 1j * entries["im"]])
        self.o.set_state(regs, amps)

    def norm(self):
        return self.emitted

    def set_norm(self, global_norm2):
        self.global_norm2 = global_norm2  # the oracle walk is unitary: nothing to rescale


def _row_partition_worker(rank: int, port: int, steps: int, out):
    dist = _init(rank, port)
    from paper_2303_06890_gb300 import partition
    from paper_2303_06890_gb300 import workloads as wl

    w = wl.small_random(40, 8, 3, band=1)
    eng = OracleEngine(w, WORLD, rank)
    partition.walk_partitioned(eng, steps)  # the product's loop: step, exchange, inbox, norms
    regs, amps = eng.o.export()
    parts = [None] * WORLD
    dist.all_gather_object(parts, [(tuple(int(v) for v in r_[:7]), complex(a_)) for r_, a_ in zip(regs, amps)])
    if rank == 0:
        out.put(([item for part in parts for item in part], eng.global_norm2))
    dist.destroy_process_group()


@pytest.mark.parametrize("steps", [3])
def test_row_partitioned_walk_equals_single_rank(steps):
    """Two gloo ranks run the product's partitioned-walk loop (ownership of
    qw_part_owner, the all-to-all exchange, the summed norm) with the oracle
    as each rank's engine; the gathered state equals the unpartitioned walk:
    keys exactly, amplitudes to 1e-12."""
    import oracle
    from paper_2303_06890_gb300 import workloads as wl

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_row_partition_worker, args=(r, port, steps, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    items, gnorm = q.get(timeout=300)
    got = dict(items)
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
    assert abs(gnorm - 1.0) < 1e-12


def test_partition_owner_rule():
    """qw_part_owner: the rows (0, j < N) in contiguous blocks of ceil(N/P),
    every other row somewhere in [0, P)."""
    from paper_2303_06890_gb300 import partition
    n, p = 37, 3
    got = [partition.owner(n, p, 0, j) for j in range(n)]
    assert got == [j // 13 for j in range(n)]
    for jc in range(1, 4):
        for j in range(64):
            assert 0 <= partition.owner(n, p, jc, j) < p
    assert all(0 <= partition.owner(n, p, 0, j) < p for j in range(n, 64))
    with pytest.raises(ValueError):
        partition.owner(n, 0, 0, 1)
