"""The positional layout (walk_variant 7, k_walk_pos) against the oracle and
against the slot kernel it restates.

Between steps the state is held by position -- no keys, counts or atomics --
and a step writes every position of its output once; the arithmetic per slot
is the slot kernel's, so with renormalisation off the states are bit for bit
those of walk_variant 4."""
import numpy as np
import pytest

import oracle
from oracle import dense
from paper_2303_06890_gb300 import qwalk
from paper_2303_06890_gb300 import workloads as wl

from parity import compare, compare_union, gpu_state, oracle_state

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _sim(w, **kw):
    return qwalk.Sim(w.matrix, s_pad=w.s, **kw)


def _oracle(w):
    o = oracle.Oracle(w.matrix, w.s)
    o.init_b(w.b)
    return o


@pytest.mark.parametrize("n,smax,seed,band,attempts", [(48, 8, 2, 1, None), (100, 8, 3, 0, None),
                                                       (130, 16, 5, 0, None), (300, 16, 8, 1, None),
                                                       (90, 32, 9, 0, 3000), (70, 32, 10, 1, 3000),
                                                       (150, 64, 11, 0, 8000), (200, 64, 12, 1, 12000)])
def test_positional_matches_oracle(n, smax, seed, band, attempts):
    """Step by step against the oracle (each read moves the state back into
    the row buckets, each step into the layout again): keys exactly,
    amplitudes to 1e-12."""
    w = wl.small_random(n, smax, seed, band=band, attempts=attempts)
    assert w.s in (8, 16, 32, 64)
    sim = _sim(w, walk_variant=7)
    sim.state_init(w.b)
    o = _oracle(w)
    o.apply("T")
    for _ in range(6):
        sim.apply_walk_step(1)
        o.apply("W")
        compare(gpu_state(sim), oracle_state(o), TOL64)
    assert o.violations == 0
    sim.close()


@pytest.mark.parametrize("precision", [qwalk.QW_FP64, qwalk.QW_FP32_AMP])
@pytest.mark.parametrize("wname", ["walk_n1024", "walk_n16384"])
def test_positional_bitwise_equals_slot_kernel(wname, precision):
    """No renormalisation: after 1, 3 and 6 steps (graph replays included)
    the state equals walk_variant 4's bit for bit, and so do the branch
    counters of the step."""
    w = getattr(wl, wname)()
    a = _sim(w, walk_variant=7, precision=precision, renorm=0)
    b = _sim(w, walk_variant=4, precision=precision, renorm=0)
    for sim in (a, b):
        sim.state_init(w.b)
    for n in (1, 2, 3):
        a.apply_walk_step(n)
        b.apply_walk_step(n)
        ka, va = a.state_export()
        kb, vb = b.state_export()
        assert np.array_equal(ka, kb), n
        assert np.array_equal(va, vb), n
    sa, sb = a.step_stats(), b.step_stats()
    for k in ("in", "after_rdag", "after_hph", "out", "steps"):
        assert sa[k] == sb[k], k
    a.enqueue_walk_steps(12)  # two 6-step graph replays
    b.enqueue_walk_steps(12)
    ka, va = a.state_export()
    kb, vb = b.state_export()
    assert np.array_equal(ka, kb) and np.array_equal(va, vb)
    a.close()
    b.close()


def test_positional_complex64_bench_config():
    """The benchmarked workload in complex64 (renormalisation on) through the
    positional layout, 20 steps, against the FP64 oracle within the
    reduced-precision bounds."""
    w = wl.walk_n16384()
    sim = _sim(w, precision=qwalk.QW_FP32_AMP, walk_variant=7)
    sim.state_init(w.b)
    sim.apply_walk_step(w.steps)
    o = _oracle(w)
    o.apply("T")
    for _ in range(w.steps):
        o.apply("W")
    compare_union(gpu_state(sim), oracle_state(o), 2e-6, 1e-5)
    sim.close()


def test_positional_runs_states_without_positions_on_the_slot_kernel():
    """An imported state over the whole register space (rows with jc != 0,
    kc != 0, k outside every row's columns) has no positions: the steps run
    on the bucket kernel and equal the oracle; a new |b~> moves into the
    layout again."""
    w = wl.small_random(40, 16, 22)
    rng = np.random.default_rng(22)
    sim = _sim(w, walk_variant=7, row_capacity=128, warp_capacity=256, spill_rows=1024)
    nb = sim.nb
    keys = set()
    while len(keys) < 600:
        keys.add((int(rng.integers(0, 3)) * int(rng.integers(0, 2)), int(rng.integers(0, 1 << nb)),
                  int(rng.integers(0, 2)), int(rng.integers(0, 3)) * int(rng.integers(0, 2)),
                  int(rng.integers(0, 1 << nb)), int(rng.integers(0, 2))))
    regs = np.array(sorted(keys), dtype=np.uint64)
    amps = rng.standard_normal(len(regs)) + 1j * rng.standard_normal(len(regs))
    amps /= np.linalg.norm(amps)
    full = np.zeros((len(regs), 8), dtype=np.uint64)
    full[:, :6] = regs
    sim.state_import(sim.pack(full), amps)
    o = oracle.Oracle(w.matrix, w.s)
    o.set_state(regs, amps)
    for _ in range(3):
        sim.apply_walk_step(1)
        o.apply("W")
        compare(gpu_state(sim), oracle_state(o), TOL64)
    sim.state_init(w.b)
    o2 = _oracle(w)
    o2.apply("T")
    for _ in range(3):
        sim.apply_walk_step(1)
        o2.apply("W")
    compare(gpu_state(sim), oracle_state(o2), TOL64)
    sim.close()


def test_positional_qls_and_measure_equal_slot_kernel():
    """The CKS read-out and p_j through the positional layout (graph-replayed
    terms) equal the slot kernel's; the register marginals after a walk too."""
    w = wl.walk_n1024()
    b_int, j0 = dense.cks_parameters(w.kappa, 1e-3)
    coeffs = dense.cks_coefficients(b_int, j0)[:60]
    out = []
    for v in (7, 4):
        sim = _sim(w, walk_variant=v)
        sim.state_init(w.b)
        y, p = sim.apply_qls(coeffs)
        sim.state_init(w.b)
        sim.apply_walk_step(10)
        m = sim.measure_register("j", w.n)
        mn = sim.measure_register_noalloc("k", w.n)
        out.append((y, p, m, mn, sim.state_size()))
        sim.close()
    (y1, p1, m1, n1, c1), (y2, p2, m2, n2, c2) = out
    assert np.abs(y1 - y2).max() < 1e-12 and np.abs(p1 - p2).max() < 1e-12
    assert np.abs(m1 - m2).max() < 1e-12 and np.abs(n1 - n2).max() < 1e-12 and c1 == c2


def test_autotune_tries_the_positional_layout():
    w = wl.walk_n1024()
    sim = _sim(w, precision=qwalk.QW_FP32_AMP)
    sim.state_init(w.b)
    v, us = sim.autotune(4)
    assert us[7] > 0.0 and v in (0, 1, 2, 3, 4, 7)
    assert us[5] == 0.0 and us[6] == 0.0
    o = _oracle(w)
    o.apply("T")
    steps = sum(1 for u in us if u > 0.0) * 4
    for _ in range(steps):
        o.apply("W")
    compare_union(gpu_state(sim), oracle_state(o), 2e-6, 1e-5)
    sim.close()


def test_positional_batched_instances_match_their_oracles():
    """Several instances of different N in one positional state (rows of all
    instances in order, each with its own column offset): every instance
    equals its own oracle after 5 steps, and a re-initialised instance
    leaves the others' states alone."""
    sizes = [(64, 1), (100, 2), (37, 3), (256, 4), (64, 5), (500, 6)]
    ws = [wl.small_random(n, 8, 40 + seed, band=1) for n, seed in sizes]
    ws = [w for w in ws if w.s == 8]
    assert len(ws) >= 3
    sim = qwalk.Sim([w.matrix for w in ws], s_pad=8, walk_variant=7)
    for i, w in enumerate(ws):
        sim.state_init(w.b, inst=i)
    sim.apply_walk_step(5)
    refs = []
    for w in ws:
        o = _oracle(w)
        o.apply("T")
        for _ in range(5):
            o.apply("W")
        refs.append(o)
    for i in range(len(ws)):
        compare(gpu_state(sim, inst=i), oracle_state(refs[i]), TOL64)
    sim.state_init(ws[1].b, inst=1)  # instance 1 back to T~|b~>, the others at step 5
    sim.apply_walk_step(2)
    o1 = _oracle(ws[1])
    o1.apply("T")
    for _ in range(2):
        o1.apply("W")
    compare(gpu_state(sim, inst=1), oracle_state(o1), TOL64)
    for i in (0, 2):
        for _ in range(2):
            refs[i].apply("W")
        compare(gpu_state(sim, inst=i), oracle_state(refs[i]), TOL64)
    sim.close()


@pytest.mark.parametrize("precision", [qwalk.QW_FP64, qwalk.QW_FP32_AMP])
def test_positional_batched_256_bitwise_equals_slot_kernel(precision):
    """The batched workload (256 walks, N log-uniform in [64, 4096], s = 8):
    without renormalisation the positional layout's states equal the slot
    kernel's bit for bit after 12 steps (graph replays), instance by
    instance on a sample, and the branch counters agree."""
    ws = wl.batched(256)
    sims = []
    for v in (7, 4):
        sim = qwalk.Sim([w.matrix for w in ws], s_pad=8, precision=precision, walk_variant=v, renorm=0)
        for i, w in enumerate(ws):
            sim.state_init(w.b, inst=i)
        sim.enqueue_walk_steps(12)
        sim.sync()
        sims.append(sim)
    a, b = sims
    for i in list(range(0, 256, 37)) + [255]:
        ka, va = a.state_export(inst=i)
        kb, vb = b.state_export(inst=i)
        assert np.array_equal(ka, kb), i
        assert np.array_equal(va, vb), i
    sa, sb = a.step_stats(), b.step_stats()
    for k in ("in", "after_rdag", "after_hph", "out", "steps"):
        assert sa[k] == sb[k], k
    for sim in sims:
        sim.close()


@pytest.mark.parametrize("precision", [qwalk.QW_FP64, qwalk.QW_FP32_AMP])
def test_positional_table1_e_matches_oracle_and_segments(precision):
    """Table 1's matrix E (N = 16384, s = 64: two QRAM slots per lane, 3.1 M
    branches): after 3 steps the positional state equals the segment
    kernel's (variant 2) -- complex128 to 1e-12 with equal keys (the
    zero-type sums add in another order), complex64 within the
    reduced-precision bounds.  (Oracle parity at s = 64 is checked above on
    smaller matrices.)"""
    w = wl.table1("E", steps=3)
    assert w.s == 64
    out = []
    for v in (7, 2):
        sim = _sim(w, walk_variant=v, precision=precision)
        sim.state_init(w.b)
        sim.apply_walk_step(3)
        out.append(gpu_state(sim))
        sim.close()
    if precision == qwalk.QW_FP64:
        compare(out[0], out[1], TOL64)
    else:
        compare_union(out[0], out[1], 2e-6, 1e-5)


@pytest.mark.parametrize("precision", [qwalk.QW_FP64, qwalk.QW_FP32_AMP])
def test_positional_init_and_marginals_in_place(precision):
    """T~|b~> written straight into the positional layout equals the bucket
    path's T~ bit for bit, and the register marginals read in place equal
    the slot kernel's after 7 steps (both measurement entry points)."""
    w = wl.walk_n1024()
    a = _sim(w, walk_variant=7, precision=precision, renorm=0)
    b = _sim(w, walk_variant=4, precision=precision, renorm=0)
    for sim in (a, b):
        sim.state_init(w.b)
    ka, va = a.state_export()
    kb, vb = b.state_export()
    assert np.array_equal(ka, kb) and np.array_equal(va, vb)
    for sim in (a, b):
        sim.state_init(w.b)  # positional again, the steps from the layout
        sim.apply_walk_step(7)
    for reg, length in (("jc", 4), ("j", w.n), ("b1", 2), ("kc", 4), ("k", w.n), ("b2", 2)):
        pa, pb = a.measure_register(reg, length), b.measure_register(reg, length)
        assert np.abs(pa - pb).max() < 1e-12, reg
        na = a.measure_register_noalloc(reg, length)
        assert np.abs(na - pb).max() < 1e-12, reg
    a.close()
    b.close()
