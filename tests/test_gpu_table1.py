"""Matrices shaped like the paper's Table 1 (Sec. V-B): positive symmetric band
matrices A..E with s = 8, 16, 32, 32, 64, through the C ABI.

* walk steps against the oracle, element by element, at full size (E: N =
  16384, s = 64, 2.1 M branches), every step-kernel variant;
* the complex64 path on C and E against the FP64 oracle;
* the CKS solver on A and B (kappa 103 and 665, as Table 1 prints 1.0e2 and
  6.6e2): the success rate p_j at every j against the dense Chebyshev theory
  (the 'theory' curves of Fig. 9) and the final fidelity against a dense solve;
* QLS terms replayed as CUDA graphs give the same bits as direct launches.
"""
import functools

import numpy as np
import pytest

import oracle
from oracle import dense
from paper_2303_06890_gb300 import qwalk
from paper_2303_06890_gb300 import workloads as wl

from parity import compare_arrays, compare_union_arrays, gpu_arrays, oracle_arrays

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
# walk steps after T~ at which the states are compared
CHECKS = {"A": (0, 1, 2, 10, 50), "B": (0, 1, 5, 20), "C": (0, 1, 4), "D": (0, 2), "E": (0, 2)}


@functools.lru_cache(maxsize=None)
def _oracle_states(name):
    w = wl.table1(name)
    o = oracle.Oracle(w.matrix, w.s)
    o.init_b(w.b)
    o.apply("T")
    states, done = {}, 0
    for c in CHECKS[name]:
        for _ in range(c - done):
            o.apply("W")
        done = c
        states[c] = oracle_arrays(o)
    assert o.violations == 0
    return w, states


@pytest.mark.parametrize("name", "ABCDE")
@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_table1_walk_fp64_matches_oracle(name, variant):
    w, states = _oracle_states(name)
    sim = qwalk.Sim(w.matrix, s_pad=w.s, walk_variant=variant)
    sim.state_init(w.b)
    done = 0
    for c in CHECKS[name]:
        sim.apply_walk_step(c - done)
        done = c
        st = compare_arrays(gpu_arrays(sim), states[c], TOL64)
    print(f"{w.name} variant {variant} step {done}: {st}")
    sim.close()


def test_table1_a_literal_schedule_matches_oracle():
    w, states = _oracle_states("A")
    sim = qwalk.Sim(w.matrix, s_pad=w.s, fuse_reflection=False)
    sim.state_init(w.b)
    done = 0
    for c in CHECKS["A"]:
        sim.apply_walk_step(c - done)
        done = c
        compare_arrays(gpu_arrays(sim), states[c], TOL64)
    sim.close()


@pytest.mark.parametrize("name", ["C", "E"])
def test_table1_complex64_against_fp64_oracle(name):
    w, states = _oracle_states(name)
    sim = qwalk.Sim(w.matrix, s_pad=w.s, precision=qwalk.QW_FP32_AMP)
    sim.state_init(w.b)
    choice, _ = sim.autotune(1)  # one step per variant
    assert choice in range(qwalk.WALK_VARIANTS)
    last = CHECKS[name][-1]
    sim.close()
    # the same number of steps from a fresh state, with the chosen variant
    sim = qwalk.Sim(w.matrix, s_pad=w.s, precision=qwalk.QW_FP32_AMP, walk_variant=choice)
    sim.state_init(w.b)
    sim.apply_walk_step(last)
    st = compare_union_arrays(gpu_arrays(sim), states[last], 2e-6, 1e-5)
    print(f"{w.name} complex64 step {last}: {st}")
    sim.close()


def _dense_success_rates(w, coeffs):
    """p_j = || sum_{k<=j} a_k T_{2k+1}(A/s) b ||^2 and the final sum, by the
    dense three-term recurrence."""
    a = w.matrix.dense() / w.s
    t_prev, t_cur = w.b.copy(), a @ w.b
    acc = coeffs[0] * t_cur
    p = [float(acc @ acc)]
    for j in range(1, len(coeffs)):
        for _ in range(2):
            t_prev, t_cur = t_cur, 2.0 * (a @ t_cur) - t_prev
        acc = acc + coeffs[j] * t_cur
        p.append(float(acc @ acc))
    return np.array(p), acc


@pytest.mark.parametrize("name", ["A", "B"])
def test_table1_qls_success_rate_and_fidelity_follow_the_dense_theory(name):
    w = wl.table1(name, steps=0)
    coeffs, j0, _ = qwalk.cks_coefficients(w.kappa, 1e-3)
    sim = qwalk.Sim(w.matrix, s_pad=w.s)
    sim.state_init(w.b)
    y, p = sim.apply_qls(coeffs)
    want_p, want_y = _dense_success_rates(w, coeffs)
    rel_p = np.abs(p - want_p) / np.maximum(want_p, 1e-30)
    rel_y = np.linalg.norm(y - want_y) / np.linalg.norm(want_y)
    x = dense.qls_reference(w.matrix.dense(), w.b)
    f = dense.fidelity(x, y)
    norm = np.abs(coeffs).sum() ** 2
    print(f"{w.name}: kappa {w.kappa:.1f} j0 {j0} F {f:.6f} p_succ {p[-1] / norm:.4e} "
          f"max rel dp {rel_p.max():.2e} rel dy {rel_y:.2e}")
    assert len(p) == j0 + 1
    assert rel_p.max() < 1e-9
    assert rel_y < 1e-9
    assert f > 0.999
    sim.close()


def test_qls_graph_replay_equals_direct_terms():
    w = wl.table1("B", steps=0)
    coeffs, _, _ = qwalk.cks_coefficients(w.kappa, 1e-3)
    coeffs = coeffs[:301]  # 301 terms: 100 graph replays of 3 terms + 1 direct term
    out = []
    for graphs in (False, True):
        sim = qwalk.Sim(w.matrix, s_pad=w.s, graphs=graphs)
        sim.state_init(w.b)
        c0 = sim.launch_count()
        y, p = sim.apply_qls(coeffs)
        assert sim.launch_count() - c0 == 3 * len(coeffs)
        out.append((y, p))
        sim.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
