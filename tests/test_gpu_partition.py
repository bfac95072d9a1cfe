"""The row-partitioned walk on one GPU: P simulators of one process, each
owning a block of rows, exchanging S's sends by cudaMemcpyAsync inside the
library (qw_part_walk).  The union of the parts equals the unpartitioned GPU
walk (complex128: bit for bit) and the oracle (keys exactly, 1e-12)."""
import numpy as np
import pytest

import oracle
from paper_2303_06890_gb300 import partition
from paper_2303_06890_gb300 import qwalk
from paper_2303_06890_gb300 import workloads as wl

from parity import compare, compare_union, gpu_state, oracle_state

pytestmark = pytest.mark.gpu


def _parts(w, nparts, **kw):
    sims = [qwalk.Sim(w.matrix, s_pad=w.s, nparts=nparts, part=p, **kw) for p in range(nparts)]
    for s in sims:
        s.state_init(w.b)
    return sims


def _union(sims):
    out = {}
    for s in sims:
        part = gpu_state(s)
        assert not set(part) & set(out)  # rows are owned once
        out.update(part)
    return out


@pytest.mark.parametrize("nparts,variant", [(2, 0), (3, 3), (2, 4), (4, 4)])
def test_partitioned_walk_equals_unpartitioned_and_oracle(nparts, variant):
    w = wl.walk_n1024()
    sims = _parts(w, nparts, walk_variant=variant)
    ref = qwalk.Sim(w.matrix, s_pad=w.s, walk_variant=variant)
    ref.state_init(w.b)
    o = oracle.Oracle(w.matrix, w.s)
    o.init_b(w.b)
    o.apply("T")
    for steps in (1, 4):
        partition.walk_in_process(sims, steps)
        ref.apply_walk_step(steps)
        for _ in range(steps):
            o.apply("W")
        got = _union(sims)
        want = gpu_state(ref)
        assert set(got) == set(want)
        assert all(got[k] == want[k] for k in want)  # same arithmetic per branch: bit for bit
        compare(got, oracle_state(o), 1e-12)
    # every part holds only rows it owns
    for p, s in enumerate(sims):
        regs = s.unpack(s.state_export()[0])
        assert all(partition.owner(w.n, nparts, int(r[0]), int(r[1])) == p for r in regs)
    for s in sims + [ref]:
        s.close()


def test_partitioned_walk_complex64_global_renormalisation():
    """complex64 with renormalisation: the parts rescale by the global norm
    (summed over the parts), matching the unpartitioned complex64 walk."""
    w = wl.walk_n1024()
    sims = _parts(w, 2, precision=qwalk.QW_FP32_AMP, walk_variant=4)
    ref = qwalk.Sim(w.matrix, s_pad=w.s, precision=qwalk.QW_FP32_AMP, walk_variant=4)
    ref.state_init(w.b)
    partition.walk_in_process(sims, 12)
    ref.apply_walk_step(12)
    got, want = _union(sims), gpu_state(ref)
    st = compare_union(got, want, 1e-6, 1e-5)
    print(f"complex64 partitioned vs unpartitioned, 12 steps: {st}")
    total = sum(abs(v) ** 2 for v in got.values())
    assert abs(total - 1.0) < 1e-5
    for s in sims + [ref]:
        s.close()


def test_partitioned_walk_at_the_benchmark_size():
    """N = 16384, s = 16 split in two: three steps, bit for bit equal to the
    unpartitioned complex128 walk."""
    from parity import gpu_arrays
    w = wl.walk_n16384()
    sims = _parts(w, 2, walk_variant=4)
    ref = qwalk.Sim(w.matrix, s_pad=w.s, walk_variant=4)
    ref.state_init(w.b)
    partition.walk_in_process(sims, 3)
    ref.apply_walk_step(3)
    kr, ar = gpu_arrays(ref)
    parts = [gpu_arrays(s) for s in sims]
    k = np.concatenate([p[0] for p in parts])
    a = np.concatenate([p[1] for p in parts])
    order = np.lexsort(tuple(k[:, c] for c in range(6, -1, -1)))
    assert np.array_equal(k[order], kr) and np.array_equal(a[order], ar)
    for s in sims + [ref]:
        s.close()


def test_partition_options_are_checked():
    w = wl.walk_n16()
    with pytest.raises(qwalk.QwError):
        qwalk.Sim(w.matrix, s_pad=w.s, nparts=2, part=2)
    with pytest.raises(qwalk.QwError):
        qwalk.Sim(w.matrix, s_pad=w.s, nparts=2, part=0, fuse_reflection=False)
    s = qwalk.Sim(w.matrix, s_pad=w.s, nparts=2, part=1)
    s.state_init(w.b)
    with pytest.raises(qwalk.QwError):
        s.apply_qls(np.ones(3))
    s.close()
