"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Keys (register values) must match exactly; amplitudes within 1e-12 in FP64.
FP32-amplitude results are compared with the FP64 oracle over the union of
keys: max |da| <= 2e-6 and ||da||_2 <= 1e-5 after 100 steps, so a branch
present on one side only must be below 2e-6 (the error is printed)."""
import math

import numpy as np
import pytest

import oracle
from oracle import dense
from paper_2303_06890_gb300 import qwalk
from paper_2303_06890_gb300 import workloads as wl

from parity import compare, compare_union, gpu_state, oracle_state

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TAU32 = 2.0 ** -24


def _sim(w, **kw):
    return qwalk.Sim(w.matrix, s_pad=w.s, **kw)


def _oracle(w):
    o = oracle.Oracle(w.matrix, w.s)
    o.init_b(w.b)
    return o


@pytest.mark.parametrize("apply_T", [False, True])
def test_state_init(apply_T):
    w = wl.walk_n16()
    sim = _sim(w)
    sim.state_init(w.b, apply_T=apply_T)
    o = _oracle(w)
    if apply_T:
        o.apply("T")
    compare(gpu_state(sim), oracle_state(o), TOL64)


@pytest.mark.parametrize("fuse,variant", [(True, 0), (True, 1), (True, 2), (True, 3), (False, 0)])
def test_walk_n16_every_step(fuse, variant):
    w = wl.walk_n16()
    sim = _sim(w, fuse_reflection=fuse, walk_variant=variant)
    sim.state_init(w.b)
    o = _oracle(w)
    o.apply("T")
    for m in range(w.steps):
        sim.apply_walk_step(1)
        o.apply("W")
        compare(gpu_state(sim), oracle_state(o), TOL64)
    assert o.violations == 0


@pytest.mark.parametrize("n,smax,seed,band", [(24, 4, 1, 0), (48, 8, 2, 1), (100, 8, 3, 0),
                                              (33, 4, 4, 1), (130, 16, 5, 0), (77, 2, 6, 0)])
def test_walk_random_cases(n, smax, seed, band):
    w = wl.small_random(n, smax, seed, band=band)
    for fuse in (True, False):
        sim = _sim(w, fuse_reflection=fuse)
        sim.state_init(w.b)
        o = _oracle(w)
        o.apply("T")
        for _ in range(5):
            sim.apply_walk_step(1)
            o.apply("W")
            compare(gpu_state(sim), oracle_state(o), TOL64)


def test_walk_n1024_fp64_100_steps():
    w = wl.walk_n1024()
    sim = _sim(w)
    sim.state_init(w.b)
    o = _oracle(w)
    o.apply("T")
    done = 0
    for target in (1, 2, 10, 50, 100):
        sim.apply_walk_step(target - done)
        for _ in range(target - done):
            o.apply("W")
        done = target
        compare(gpu_state(sim), oracle_state(o), TOL64)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
def test_walk_n16384_fp64_full_size(variant):
    w = wl.walk_n16384()
    sim = _sim(w, walk_variant=variant)
    sim.state_init(w.b)
    o = _oracle(w)
    o.apply("T")
    compare(gpu_state(sim), oracle_state(o), TOL64)
    for _ in range(3):
        sim.apply_walk_step(1)
        o.apply("W")
        compare(gpu_state(sim), oracle_state(o), TOL64)


def test_fp32_amp_n1024_100_steps():
    w = wl.walk_n1024()
    sim = _sim(w, precision=qwalk.QW_FP32_AMP)
    sim.state_init(w.b)
    o = _oracle(w)
    o.apply("T")
    done = 0
    for target in (10, 100):
        sim.apply_walk_step(target - done)
        for _ in range(target - done):
            o.apply("W")
        done = target
        st = compare_union(gpu_state(sim), oracle_state(o), 2e-6, 1e-5)
        print(f"FP32-amp N=1024 step {target}: {st}")


def test_fp32_amp_n16384_bench_config():
    """The benchmarked configuration (N=16384, s=16, complex64 amplitudes), 20
    steps -- 3 of them by each variant the autotuner tries, as bench.py runs
    it -- against the FP64 oracle."""
    w = wl.walk_n16384()
    sim = _sim(w, precision=qwalk.QW_FP32_AMP)
    sim.state_init(w.b)
    choice, us = sim.autotune(3)
    assert choice in range(qwalk.WALK_VARIANTS) and min(us[:4]) > 0 and us[7] > 0
    tried = sum(1 for v in us if v > 0)
    assert 3 * tried <= w.steps
    sim.apply_walk_step(w.steps - 3 * tried)
    o = _oracle(w)
    o.apply("T")
    for _ in range(w.steps):
        o.apply("W")
    st = compare_union(gpu_state(sim), oracle_state(o), 2e-6, 1e-5)
    print(f"FP32-amp N=16384 step 20: {st}")


def test_measure_register_matches_oracle():
    w = wl.small_random(40, 8, 11)
    sim = _sim(w)
    sim.state_init(w.b)
    sim.apply_walk_step(5)
    o = _oracle(w)
    o.apply("T")
    for _ in range(5):
        o.apply("W")
    for reg in ("jc", "j", "b1", "kc", "k", "b2"):
        length = 1 << sim.nb
        got = sim.measure_register(reg, length)
        want = o.marginal(reg, length)
        assert np.abs(got - want).max() < 1e-12, reg
    assert abs(sim.measure_register("j", 1 << sim.nb).sum() - 1.0) < 1e-12


def test_chebyshev_identity_at_full_size_via_readout():
    """Flag-0 blocks read by the QLS path equal T_{2j+1}(A/s) b from the dense
    recurrence, at N = 16384 (a property that holds at any size)."""
    w = wl.walk_n16384()
    a = w.matrix.dense() if w.n <= 4096 else None
    rng = np.random.default_rng(5)
    coeffs = rng.standard_normal(4)
    sim = _sim(w)
    sim.state_init(w.b)
    y, p = sim.apply_qls(coeffs)
    # sparse A/s times vector, from the CSC arrays
    m = w.matrix
    cols = np.repeat(np.arange(m.n), np.diff(m.colptr))
    vals = m.val_q15.astype(np.float64) / 32768.0 / w.s

    def hv(v):
        out = np.zeros(m.n, dtype=complex)
        np.add.at(out, m.rowidx, vals * v[cols])
        return out

    t_prev, t_cur = w.b.astype(complex), hv(w.b.astype(complex))
    cheb = [t_prev, t_cur]
    for _ in range(2, 2 * len(coeffs)):
        t_prev, t_cur = t_cur, 2 * hv(t_cur) - t_prev
        cheb.append(t_cur)
    want = sum(c * cheb[2 * j + 1] for j, c in enumerate(coeffs))
    assert a is None
    assert np.abs(y - want).max() < 1e-12
    acc = np.zeros(m.n, dtype=complex)
    for j, c in enumerate(coeffs):
        acc += c * cheb[2 * j + 1]
        assert abs(p[j] - np.vdot(acc, acc).real) < 1e-10 * max(1.0, p[j])


def test_qls_n16_matches_oracle():
    w = wl.walk_n16()
    b_int, j0 = dense.cks_parameters(w.kappa, 1e-3)
    coeffs = dense.cks_coefficients(b_int, j0)
    sim = _sim(w)
    sim.state_init(w.b)
    y, p = sim.apply_qls(coeffs)
    yo, ys, _ = oracle.qls(w.matrix, w.s, w.b, coeffs)
    assert np.abs(y - yo).max() < 1e-9 * max(1.0, np.abs(yo).max())
    x = dense.qls_reference(w.matrix.dense(), w.b)
    assert dense.fidelity(x, y) > 0.999


@pytest.mark.parametrize("precision", [qwalk.QW_FP64, qwalk.QW_FP32_AMP])
def test_qls_n1024_fidelity(precision):
    """The CKS solve of the cond(A) = 100 N = 1024 system against the dense
    FP64 theory: Y = sum_j a_j T_{2j+1}(A/s) b, p_j = ||Y_j||^2 at every j, and
    the fidelity to the dense solve.  complex128: 1e-9 relative; complex64:
    |dp_j| / p_j <= 1e-4 and |dF| <= 1e-4 (the reduced-precision targets)."""
    w = wl.qls_n1024()
    coeffs, j0, b_int = qwalk.cks_coefficients(w.kappa, 1e-3)
    sim = _sim(w, precision=precision)
    sim.state_init(w.b)
    y, p = sim.apply_qls(coeffs)
    a = w.matrix.dense() / w.s
    t_prev, t_cur = w.b.copy(), a @ w.b
    want = coeffs[0] * t_cur
    want_p = [float(want @ want)]
    for j in range(1, j0 + 1):
        for _ in range(2):
            t_prev, t_cur = t_cur, 2 * (a @ t_cur) - t_prev
        want = want + coeffs[j] * t_cur
        want_p.append(float(want @ want))
    x = dense.qls_reference(w.matrix.dense(), w.b)
    f = dense.fidelity(x, y)
    df = abs(f - dense.fidelity(x, want))
    rel = np.linalg.norm(y - want) / np.linalg.norm(want)
    rel_p = float(np.max(np.abs(p - np.array(want_p)) / np.array(want_p)))
    print(f"QLS N=1024 precision={precision}: j0={j0} F={f:.8f} |dF|={df:.2e} "
          f"rel.err vs dense {rel:.3e} max |dp|/p {rel_p:.2e}")
    if precision == qwalk.QW_FP64:
        assert rel < 1e-9 and rel_p < 1e-9
    else:
        assert rel < 1e-3 and rel_p <= 1e-4 and df <= 1e-4
    assert f > 0.999


def test_batched_instances_match_their_oracles():
    sizes = [(64, 1), (100, 2), (37, 3), (256, 4), (64, 5), (500, 6)]
    ws = [wl.small_random(n, 8, 40 + seed, band=1) for n, seed in sizes]
    ws = [w for w in ws if w.s == 8]
    mats = [w.matrix for w in ws]
    sim = qwalk.Sim(mats, s_pad=8)
    for i, w in enumerate(ws):
        sim.state_init(w.b, inst=i)
    sim.apply_walk_step(5)
    for i, w in enumerate(ws):
        o = oracle.Oracle(w.matrix, 8)
        o.init_b(w.b)
        o.apply("T")
        for _ in range(5):
            o.apply("W")
        compare(gpu_state(sim, inst=i), oracle_state(o), TOL64)


@pytest.mark.parametrize("enqueue", [False, True])
def test_capacity_overflow_keeps_last_clean_state(enqueue):
    """A segment that outgrows the warp's on-chip buffer fails the call with
    QW_ERR_CAPACITY (two rows of up to 8 branches against a buffer of 8, once
    the b1 = 1 rows fill); the steps issued after the failing one do nothing,
    and the state is the output of the last clean step, equal to the oracle's
    after that many steps."""
    w = wl.walk_n16()
    sim = _sim(w, row_capacity=8, warp_capacity=8, walk_variant=2, overflow_fallback=False)
    sim.state_init(w.b)
    o = _oracle(w)
    o.apply("T")
    clean = 0
    with pytest.raises(qwalk.QwError) as e:
        for _ in range(20):
            if enqueue:
                sim.enqueue_walk_steps(3)
                sim.sync()
                clean += 3
            else:
                sim.apply_walk_step(1)
                clean += 1
    assert e.value.code == qwalk.QW_ERR_CAPACITY
    msg = str(e.value)
    kept = int(msg.split("state kept after ")[1].split(" ")[0])
    for _ in range(clean + kept):
        o.apply("W")
    compare(gpu_state(sim), oracle_state(o), TOL64)
    # the simulator stays usable after the error
    sim.state_init(w.b)
    assert sim.state_size() > 0


def test_degenerate_inputs():
    # all-zero b: empty state, steps are no-ops
    w = wl.walk_n16()
    sim = _sim(w)
    sim.state_init(np.zeros(w.n))
    assert sim.state_size() == 0
    sim.apply_walk_step(2)
    assert sim.state_size() == 0
    # a single basis vector and a diagonal matrix (s = 1)
    a = np.diag(np.linspace(0.1, 0.9, 8))
    from test_oracle_pins import dense_to_matrix
    m = dense_to_matrix(a)
    wd = wl.Workload("diag", m, np.eye(8)[3], s=1, steps=3, cond=0, kappa=0)
    for fuse in (True, False):
        sim = _sim(wd, fuse_reflection=fuse)
        sim.state_init(wd.b)
        o = _oracle(wd)
        o.apply("T")
        for _ in range(3):
            sim.apply_walk_step(1)
            o.apply("W")
            compare(gpu_state(sim), oracle_state(o), TOL64)
    # N = 2 with a full row
    m2 = dense_to_matrix(np.array([[0.5, -0.7], [-0.7, 0.2]]))
    w2 = wl.Workload("n2", m2, np.array([0.6, 0.8]), s=2, steps=4, cond=0, kappa=0)
    sim = _sim(w2)
    sim.state_init(w2.b)
    o = _oracle(w2)
    o.apply("T")
    for _ in range(4):
        sim.apply_walk_step(1)
        o.apply("W")
        compare(gpu_state(sim), oracle_state(o), TOL64)


def test_launch_count_and_reinit():
    w = wl.walk_n16()
    sim = _sim(w)
    sim.state_init(w.b)
    c0 = sim.launch_count()
    sim.apply_walk_step(4)
    assert sim.launch_count() - c0 == 4  # one launch per walk step
    sim.state_init(w.b)
    o = _oracle(w)
    o.apply("T")
    compare(gpu_state(sim), oracle_state(o), TOL64)


@pytest.mark.parametrize("precision", [qwalk.QW_FP64, qwalk.QW_FP32_AMP])
def test_graph_replay_equals_direct_launches(precision):
    """Runs issued as replays of the captured 6-step graph give the same state
    as one launch per step, from every (buffer, slot) phase: bit for bit in
    FP64; in FP32 up to the renormalisation factor, whose FP64 norm sums the
    branches in their (atomic, run-dependent) arrival order."""
    w = wl.walk_n1024()
    a = _sim(w, precision=precision, graphs=True)
    b = _sim(w, precision=precision, graphs=False)
    for sim in (a, b):
        sim.state_init(w.b)
    for n in (7, 6, 13, 1, 12):
        a.apply_walk_step(n)
        b.apply_walk_step(n)
        ka, va = a.state_export()
        kb, vb = b.state_export()
        assert np.array_equal(ka, kb), n
        if precision == qwalk.QW_FP64:
            assert np.array_equal(va, vb), n
        else:
            assert np.abs(va - vb).max() <= 1e-6 * np.abs(vb).max(), n
    o = _oracle(w)
    o.apply("T")
    for _ in range(39):
        o.apply("W")
    if precision == qwalk.QW_FP64:
        compare(gpu_state(a), oracle_state(o), TOL64)


@pytest.mark.parametrize("precision", [qwalk.QW_FP64, qwalk.QW_FP32_AMP])
def test_batched_256_instances_full_size(precision):
    """The batched workload at full size: 256 walks (N log-uniform in [64,
    4096], s = 8) advanced together, one launch per step (graph-replayed), 50
    steps.  A sample of instances across the size range equals its own FP64
    oracle: complex128 keys exactly and amplitudes to 1e-12; complex64 over the
    union of keys within the reduced-precision bounds (max |da| <= 2e-6,
    ||da||_2 <= 1e-5).  Every instance keeps unit norm."""
    ws = wl.batched(256)
    sim = qwalk.Sim([w.matrix for w in ws], s_pad=8, precision=precision)
    for i, w in enumerate(ws):
        sim.state_init(w.b, inst=i)
    sim.apply_walk_step(50)
    for i, w in enumerate(ws):
        p = sim.measure_register("b2", 2, inst=i)
        assert abs(p.sum() - 1.0) < (1e-10 if precision == qwalk.QW_FP64 else 1e-5), i
    by_size = sorted(range(len(ws)), key=lambda i: ws[i].n)
    worst = {"max_abs": 0.0, "l2": 0.0}
    for i in by_size[::32] + [by_size[-1]]:
        w = ws[i]
        o = oracle.Oracle(w.matrix, 8)
        o.init_b(w.b)
        o.apply("T")
        for _ in range(50):
            o.apply("W")
        if precision == qwalk.QW_FP64:
            compare(gpu_state(sim, inst=i), oracle_state(o), TOL64)
        else:
            st = compare_union(gpu_state(sim, inst=i), oracle_state(o), 2e-6, 1e-5)
            worst = {k: max(worst[k], st[k]) for k in worst}
    if precision != qwalk.QW_FP64:
        print(f"complex64 batched, 50 steps, worst sampled instance: {worst}")


def test_checkpoint_round_trip():
    """qw_state_export then qw_state_import reproduces the state, and the
    resumed walk equals the uninterrupted one."""
    w = wl.walk_n1024()
    a = _sim(w)
    a.state_init(w.b)
    a.apply_walk_step(5)
    keys, amps = a.state_export()
    b = _sim(w)
    b.state_import(keys, amps)
    k2, a2 = b.state_export()
    assert np.array_equal(keys, k2) and np.array_equal(amps, a2)
    a.apply_walk_step(3)
    b.apply_walk_step(3)
    compare(gpu_state(b), gpu_state(a), 0.0)


@pytest.mark.parametrize("fuse,variant", [(True, 0), (True, 1), (True, 2), (True, 3), (False, 0)])
def test_garbage_subspace_states_match_oracle(fuse, variant):
    """Random states over the whole register space -- rows with jc != 0 (the
    garbage-row table), rows j >= N (N = 12, so the all-zero QRAM list), kc != 0
    and k >= s (QRAM reads outside the row) -- walked by the GPU and by the
    oracle from the same imported state."""
    w = wl.small_random(12, 4, 17)
    rng = np.random.default_rng(99)
    sim = _sim(w, fuse_reflection=fuse, walk_variant=variant, row_capacity=96, warp_capacity=128)
    nb = sim.nb
    keys = set()
    while len(keys) < 400:
        keys.add((int(rng.integers(0, 4)), int(rng.integers(0, 1 << nb)), int(rng.integers(0, 2)),
                  int(rng.integers(0, 4)), int(rng.integers(0, 1 << nb)), int(rng.integers(0, 2))))
    regs = np.array(sorted(keys), dtype=np.uint64)
    amps = rng.standard_normal(len(regs)) + 1j * rng.standard_normal(len(regs))
    amps /= np.linalg.norm(amps)
    assert (regs[:, 0] != 0).sum() > 100 and (regs[:, 1] >= w.n).sum() > 50
    full = np.zeros((len(regs), 8), dtype=np.uint64)
    full[:, :6] = regs
    sim.state_import(sim.pack(full), amps)
    o = oracle.Oracle(w.matrix, w.s)
    o.set_state(regs, amps)
    compare(gpu_state(sim), oracle_state(o), 0.0)
    for _ in range(4):
        sim.apply_walk_step(1)
        o.apply("W")
        compare(gpu_state(sim), oracle_state(o), TOL64)


def test_garbage_row_table_size_is_an_option_and_overflow_is_reported():
    """The rows with jc != 0 live in a hash table of spill_rows slots: a state
    with more such rows than slots is refused with QW_ERR_CAPACITY; one table
    slot per row suffices."""
    w = wl.small_random(12, 4, 17)
    rng = np.random.default_rng(7)
    keys = set()
    while len(keys) < 200:
        keys.add((int(rng.integers(1, 4)), int(rng.integers(0, 16)), int(rng.integers(0, 2)),
                  0, int(rng.integers(0, 16)), int(rng.integers(0, 2))))
    regs = np.array(sorted(keys), dtype=np.uint64)
    rows = len({tuple(r[:3]) for r in regs.tolist()})
    amps = rng.standard_normal(len(regs)) + 0j
    amps /= np.linalg.norm(amps)
    full = np.zeros((len(regs), 8), dtype=np.uint64)
    full[:, :6] = regs
    small = _sim(w, spill_rows=16)
    with pytest.raises(qwalk.QwError) as err:
        small.state_import(small.pack(full), amps)
    assert err.value.code == qwalk.QW_ERR_CAPACITY and "garbage-row table full" in str(err.value)
    small.close()
    fit = _sim(w, spill_rows=int(wl.next_pow2(rows)))
    fit.state_import(fit.pack(full), amps)
    o = oracle.Oracle(w.matrix, w.s)
    o.set_state(regs, amps)
    compare(gpu_state(fit), oracle_state(o), 0.0)
    fit.close()
    with pytest.raises(qwalk.QwError):
        _sim(w, spill_rows=100)  # not a power of two


@pytest.mark.parametrize("n", [20000, 40000])
@pytest.mark.parametrize("variant", [0, 3])
def test_walk_with_64bit_in_kernel_keys_matches_oracle(n, variant):
    """N > 16384 (nb = 15, 16): the step kernel holds its keys in 64 bits
    instead of 32; walked against the oracle element by element."""
    from parity import compare_arrays, gpu_arrays, oracle_arrays
    w = wl.small_random(n, 4, 23, band=1, attempts=n)
    sim = _sim(w, walk_variant=variant)
    assert sim.nb >= 15
    sim.state_init(w.b)
    o = _oracle(w)
    o.apply("T")
    compare_arrays(gpu_arrays(sim), oracle_arrays(o), TOL64)
    for _ in range(3):
        sim.apply_walk_step(1)
        o.apply("W")
    st = compare_arrays(gpu_arrays(sim), oracle_arrays(o), TOL64)
    print(f"N={n} variant {variant}: {st}")
    sim.close()


@pytest.mark.parametrize("fuse", [True, False])
def test_fixed_point_rotation_angle_matches_oracle(fuse):
    """rot_bits = 8: the rotation angle in an 8-bit fixed-point register (the
    square-root and arccos registers of Table 2); the GPU walk equals the
    oracle run with the same register, keys exactly, amplitudes to 1e-12."""
    w = wl.walk_n16()
    sim = _sim(w, rot_bits=8, fuse_reflection=fuse)
    sim.state_init(w.b)
    o = oracle.Oracle(w.matrix, w.s, rot_bits=8)
    o.init_b(w.b)
    o.apply("T")
    compare(gpu_state(sim), oracle_state(o), TOL64)
    for _ in range(5):
        sim.apply_walk_step(1)
        o.apply("W")
        compare(gpu_state(sim), oracle_state(o), TOL64)
    sim.close()
    with pytest.raises(qwalk.QwError):
        _sim(w, rot_bits=53)  # wider than an FP64 mantissa


def test_qls_fidelity_against_the_width_of_the_angle_register():
    """The CKS solve of Table 1's matrix A (kappa 103) with the rotation angle
    held in b bits: the fidelity to the exact solution approaches the
    exact-rotation value as b grows (printed for b = 6 .. 16)."""
    w = wl.table1("A", steps=0)
    coeffs, _, _ = qwalk.cks_coefficients(w.kappa, 1e-3)
    x = dense.qls_reference(w.matrix.dense(), w.b)
    fid = {}
    for bits in (6, 8, 10, 12, 16, 0):
        sim = _sim(w, rot_bits=bits)
        sim.state_init(w.b)
        y, _ = sim.apply_qls(coeffs)
        fid[bits] = dense.fidelity(x, y)
        sim.close()
    print("QLS fidelity by angle-register bits:", {k: round(v, 8) for k, v in fid.items()})
    assert fid[0] > 0.999 and fid[16] > 0.999
    assert fid[6] < fid[16]


def test_complex64_with_64bit_in_kernel_keys_against_fp64_oracle():
    """N = 20000 (64-bit in-kernel keys) in complex64, pipelined segments,
    against the FP64 oracle over the union of keys after 4 steps."""
    from parity import compare_union_arrays, gpu_arrays, oracle_arrays
    w = wl.small_random(20000, 4, 23, band=1, attempts=20000)
    sim = _sim(w, precision=qwalk.QW_FP32_AMP, walk_variant=3)
    sim.state_init(w.b)
    sim.apply_walk_step(4)
    o = _oracle(w)
    o.apply("T")
    for _ in range(4):
        o.apply("W")
    st = compare_union_arrays(gpu_arrays(sim), oracle_arrays(o), 2e-6, 1e-5)
    print(f"complex64 N=20000 step 4: {st}")
    sim.close()


@pytest.mark.parametrize("n,smax,seed,band,attempts", [(48, 8, 2, 1, None), (100, 8, 3, 0, None),
                                                       (130, 16, 5, 0, None), (300, 16, 8, 1, None),
                                                       (90, 32, 9, 0, 3000), (70, 32, 10, 1, 3000)])
def test_slot_kernel_matches_oracle(n, smax, seed, band, attempts):
    """walk_variant 4 (one lane per QRAM slot, s = 8, 16, 32) against the
    oracle, step by step: keys exactly, amplitudes to 1e-12."""
    w = wl.small_random(n, smax, seed, band=band, attempts=attempts)
    assert w.s in (8, 16, 32)
    sim = _sim(w, walk_variant=4)
    sim.state_init(w.b)
    o = _oracle(w)
    o.apply("T")
    for _ in range(6):
        sim.apply_walk_step(1)
        o.apply("W")
        compare(gpu_state(sim), oracle_state(o), TOL64)
    sim.close()


@pytest.mark.parametrize("wname", ["walk_n1024", "walk_n16384"])
def test_slot_kernel_bitwise_equals_row_pipeline(wname):
    """complex128 (no renormalisation): the slot kernel runs the same
    operations in the same order as the row pipeline, so the states after
    each step are bit for bit equal (compared in canonical key order)."""
    w = getattr(wl, wname)()
    a = _sim(w, walk_variant=4, graphs=False)
    b = _sim(w, walk_variant=0, graphs=False)
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
    for k in ("in", "after_rdag", "after_hph", "out"):
        assert sa[k] == sb[k], k
    a.close()
    b.close()


@pytest.mark.parametrize("n,smax,seed", [(12, 8, 21), (40, 16, 22), (24, 8, 23)])
def test_slot_kernel_on_garbage_subspace_states(n, smax, seed):
    """Random states over the whole register space (rows with jc != 0, rows
    j >= N, kc != 0, QRAM reads outside the row, groups with more extras than
    the slot kernel lists): the slot kernel hands them to the row pipeline or
    runs them as extras, and equals the oracle."""
    w = wl.small_random(n, smax, seed)
    assert w.s in (8, 16, 32), w.s
    rng = np.random.default_rng(seed)
    sim = _sim(w, walk_variant=4, row_capacity=128, warp_capacity=256, spill_rows=1024)
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
    sim.close()


def test_slot_kernel_complex64_bench_config():
    """The benchmarked workload in complex64 through the slot kernel, 20
    steps, against the FP64 oracle within the reduced-precision bounds."""
    w = wl.walk_n16384()
    sim = _sim(w, precision=qwalk.QW_FP32_AMP, walk_variant=4)
    sim.state_init(w.b)
    sim.apply_walk_step(w.steps)
    o = _oracle(w)
    o.apply("T")
    for _ in range(w.steps):
        o.apply("W")
    from parity import compare_union_arrays, gpu_arrays, oracle_arrays
    st = compare_union_arrays(gpu_arrays(sim), oracle_arrays(o), 2e-6, 1e-5)
    print(f"slot kernel complex64 N=16384 step 20: {st}")
    sim.close()


def _clustered_matrix():
    """N = 40, s = 8: rows 10..15 form a full block (6 entries each) and pad
    their two free slots onto the same columns 16 and 17 (the padding rule
    takes the first free columns after j), so rows 16 and 17 receive more
    branches than the others; the rest is a tridiagonal band."""
    from test_oracle_pins import dense_to_matrix
    n = 40
    rng = np.random.default_rng(77)
    a = np.zeros((n, n))
    for j in range(n):
        a[j, j] = rng.uniform(0.2, 1.0)
        if j + 1 < n and not (10 <= j < 16 and 10 <= j + 1 < 16):
            a[j, j + 1] = a[j + 1, j] = rng.uniform(-1, 1)
    for i in range(10, 16):
        for j in range(i + 1, 16):
            a[i, j] = a[j, i] = rng.uniform(-1, 1)
    m = dense_to_matrix(a)
    b = rng.standard_normal(n)
    return wl.Workload("clustered_n40", m, b / np.linalg.norm(b), s=8, steps=6, cond=0, kappa=0)


@pytest.mark.parametrize("variant", [0, 3, 4])
def test_overflowing_rows_run_on_the_flat_path(variant):
    """A row capacity below what the clustered rows need: the steps that
    overflow are run again on the flat path (global radix sort by key,
    per-group transform, compaction), the row buckets grow, and every step
    equals the oracle (keys exactly, amplitudes to 1e-12)."""
    w = _clustered_matrix()
    sim = _sim(w, row_capacity=6, walk_variant=variant)
    sim.state_init(w.b)
    o = _oracle(w)
    o.apply("T")
    for _ in range(w.steps):
        sim.apply_walk_step(1)
        o.apply("W")
        compare(gpu_state(sim), oracle_state(o), TOL64)
    # several steps in one call, enqueued and synchronised once
    sim.state_init(w.b)
    sim.enqueue_walk_steps(5)
    sim.sync()
    o = _oracle(w)
    o.apply("T")
    for _ in range(5):
        o.apply("W")
    compare(gpu_state(sim), oracle_state(o), TOL64)
    sim.close()


@pytest.mark.parametrize("precision", [qwalk.QW_FP64, qwalk.QW_FP32_AMP])
@pytest.mark.parametrize("maker", [wl.walk_n16, lambda: wl.small_random(100, 8, 3),
                                   lambda: wl.small_random(130, 16, 5)])
def test_flat_path_matches_oracle(maker, precision):
    """walk_variant 5, the paper's schedule on one globally sorted list:
    complex128 equals the oracle step by step (keys exactly, 1e-12); complex64
    (FP64 arithmetic on the flat path, FP32 storage) within the
    reduced-precision bounds."""
    w = maker()
    sim = _sim(w, walk_variant=5, precision=precision)
    sim.state_init(w.b)
    o = _oracle(w)
    o.apply("T")
    for _ in range(4):
        sim.apply_walk_step(1)
        o.apply("W")
        if precision == qwalk.QW_FP64:
            compare(gpu_state(sim), oracle_state(o), TOL64)
        else:
            compare_union(gpu_state(sim), oracle_state(o), 2e-6, 1e-5)
    st = sim.step_stats()
    assert st["steps"] == 4 and st["after_h1"] > 0
    sim.close()


@pytest.mark.parametrize("variant, n, smax, seed, tries", [(5, 160, 64, 9, 40), (6, 160, 64, 9, 40),
                                                           (5, 300, 128, 11, 80), (6, 300, 128, 11, 80),
                                                           (5, 600, 256, 13, 160)])
def test_flat_path_large_s(variant, n, smax, seed, tries):
    """The flat path's Hadamard stage at s = 64 and 128 (the fast transform
    with 2 and 4 vector entries a lane, the butterflies above bit 5 between a
    lane's registers) and at s = 256 (the direct sums), on the flat path and
    the register-faithful schedule: three complex128 steps equal the
    oracle's."""
    w = wl.small_random(n, smax, seed, attempts=n * tries)
    assert w.s == smax
    # row buckets of s entries (grown by the store where a row needs more), so
    # that the bucket kernels' per-block buffers fit at creation
    sim = _sim(w, walk_variant=variant, row_capacity=smax)
    o = _oracle(w)
    o.apply("T")
    if smax <= 128:
        sim.state_init(w.b)
    else:  # T~|b~> (rows of 2 s branches) imported: beyond the initialisation kernel's row buffers
        regs, amps = o.export()
        full = np.zeros((len(regs), 8), dtype=np.uint64)
        full[:, :7] = regs
        sim.state_import(sim.pack(full), amps)
    for _ in range(3):
        sim.apply_walk_step(1)
        o.apply("W")
        compare(gpu_state(sim), oracle_state(o), TOL64)
    sim.close()


def test_flat_path_on_garbage_states_and_qls():
    """The flat path on a random state over the whole register space, and the
    CKS read-out through it (the flag-0 block after T~^dag's H)."""
    w = wl.small_random(12, 4, 17)
    rng = np.random.default_rng(5)
    sim = _sim(w, walk_variant=5, spill_rows=1024)
    nb = sim.nb
    keys = set()
    while len(keys) < 300:
        keys.add((int(rng.integers(0, 4)), int(rng.integers(0, 1 << nb)), int(rng.integers(0, 2)),
                  int(rng.integers(0, 4)), int(rng.integers(0, 1 << nb)), int(rng.integers(0, 2))))
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
    sim.close()
    w = wl.walk_n16()
    b_int, j0 = dense.cks_parameters(w.kappa, 1e-3)
    coeffs = dense.cks_coefficients(b_int, j0)[:40]
    flat = _sim(w, walk_variant=5)
    flat.state_init(w.b)
    y, p = flat.apply_qls(coeffs)
    ref = _sim(w)
    ref.state_init(w.b)
    y2, p2 = ref.apply_qls(coeffs)
    assert np.abs(y - y2).max() < 1e-12 and np.abs(p - p2).max() < 1e-12


@pytest.mark.parametrize("variant", [5, 6])
def test_flat_sort_spans_two_key_chunks(variant):
    """A random state whose branches differ in 66 register bits (nb = 16:
    jc, j, kc, k over their whole ranges, b1, b2; 5000 branches, several
    2048-entry tiles of the sort's passes with a ragged last one): the flat
    path's radix sort takes the varying bits in two 64-bit chunks (the second
    formed in the order the first left); three steps on the flat path and on
    the register-faithful schedule equal the oracle's."""
    w = wl.small_random(40000, 4, 29)
    rng = np.random.default_rng(7)
    sim = _sim(w, walk_variant=variant, spill_rows=1 << 15)  # rows with jc != 0
    nb = sim.nb
    assert 4 * nb + 2 > 64
    keys = set()
    while len(keys) < 5000:
        keys.add((int(rng.integers(0, 1 << nb)), int(rng.integers(0, 1 << nb)), int(rng.integers(0, 2)),
                  int(rng.integers(0, 1 << nb)), int(rng.integers(0, 1 << nb)), int(rng.integers(0, 2))))
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
    sim.close()


def test_import_grows_row_capacity():
    """qw_state_import of a state whose rows exceed row_capacity grows the
    buckets (overflow_fallback) and the walk continues equal to the oracle."""
    w = wl.small_random(24, 8, 23)
    rng = np.random.default_rng(3)
    sim = _sim(w, row_capacity=8)
    nb = sim.nb
    keys = set()
    while len(keys) < 60:  # 60 branches in one row (jc = 0, j = 5, b1 = 0)
        keys.add((0, 5, 0, 0, int(rng.integers(0, 1 << nb)), int(rng.integers(0, 2))))
    regs = np.array(sorted(keys), dtype=np.uint64)
    amps = rng.standard_normal(len(regs)) + 0j
    amps /= np.linalg.norm(amps)
    full = np.zeros((len(regs), 8), dtype=np.uint64)
    full[:, :6] = regs
    sim.state_import(sim.pack(full), amps)
    o = oracle.Oracle(w.matrix, w.s)
    o.set_state(regs, amps)
    compare(gpu_state(sim), oracle_state(o), 0.0)
    for _ in range(2):
        sim.apply_walk_step(1)
        o.apply("W")
        compare(gpu_state(sim), oracle_state(o), TOL64)
    sim.close()
