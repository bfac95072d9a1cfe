"""Register-faithful mode (the qw_faithful_* calls and walk_variant 6) against
the oracle's sub-operations.

After every sub-operation of W = S T~ P T~^dag the GPU's registers -- the base
ones, A, the QRAM address and Alg. 1's left, right, mid, midval, flag and
comparison bits with every stack frame -- equal the oracle's bit for bit, and
the amplitudes agree within 1e-12 (FP64)."""
import numpy as np
import pytest

import oracle
from oracle import dense
from paper_2303_06890_gb300 import qwalk
from paper_2303_06890_gb300 import workloads as wl

from parity import compare, compare_union, gpu_state, oracle_state

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
NCOL = len(qwalk.FQ_COLUMNS) - 1  # every column but the instance


def _sim(w, **kw):
    return qwalk.Sim(w.matrix, s_pad=w.s, **kw)


def _oracle(w):
    o = oracle.Oracle(w.matrix, w.s)
    o.init_b(w.b)
    return o


def gpu_faithful(sim) -> dict:
    regs, amps = sim.faithful_export()
    assert np.all(regs[:, 0] == 0)
    return {tuple(int(v) for v in r[1:]): complex(a) for r, a in zip(regs, amps)}


def oracle_faithful(o) -> dict:
    regs, amps = o.export_faithful()
    assert regs.shape[1] == NCOL
    return {tuple(int(v) for v in r): complex(a) for r, a in zip(regs, amps)}


MAKERS = [wl.walk_n16, lambda: wl.small_random(48, 8, 2), lambda: wl.small_random(130, 16, 5)]


@pytest.mark.parametrize("maker", MAKERS)
def test_every_sub_operation_matches_oracle(maker):
    """Two walk steps, compared after each of their 116 sub-operations, then
    the list stored back as the state and compared with the oracle's."""
    w = maker()
    sim = _sim(w)
    sim.state_init(w.b)
    o = _oracle(w)
    o.apply("T")
    info = sim.faithful_info()
    assert info["fits"] and info["addr_bits"] == o.faithful_addr_bits
    sim.faithful_begin()
    compare(gpu_faithful(sim), oracle_faithful(o), TOL64)
    for _ in range(2):
        for op in qwalk.FQ_STEP:
            sim.faithful_apply(op)
            o.apply_faithful(op)
            compare(gpu_faithful(sim), oracle_faithful(o), TOL64)
    sim.faithful_end()
    compare(gpu_state(sim), oracle_state(o), TOL64)
    assert o.violations == 0
    st = sim.step_stats()
    assert st["steps"] == 1 and st["after_hph"] > 0
    sim.close()


def test_search_registers_mid_search():
    """Alg. 1 stopped after its forward loop: left, right, flag and the L + 1
    frames of (mid, midval, cl, ce) are held in the state and equal the
    oracle's on every branch; undoing it clears them."""
    w = wl.small_random(100, 8, 3)
    sim = _sim(w)
    sim.state_init(w.b)
    o = _oracle(w)
    o.apply("T")
    sim.faithful_begin()
    ops = ("SWAP", "QBS_FWD")
    sim.faithful_apply(*ops)
    o.apply_faithful(*ops)
    g, r = gpu_faithful(sim), oracle_faithful(o)
    compare(g, r, TOL64)
    cols = qwalk.FQ_COLUMNS[1:]
    flag, right = cols.index("flag"), cols.index("right")
    assert all(k[right] != 0 for k in g)  # the search interval is live on every branch
    assert any(k[cols.index("ce0")] or k[flag] for k in g)
    sim.faithful_apply("QBS_BWD", "SWAP")
    o.apply_faithful("QBS_BWD", "SWAP")
    g = gpu_faithful(sim)
    compare(g, oracle_faithful(o), TOL64)
    assert all(all(v == 0 for v in k[7:]) for k in g)
    sim.faithful_end(keep=False)
    sim.close()


@pytest.mark.parametrize("precision", [qwalk.QW_FP64, qwalk.QW_FP32_AMP])
@pytest.mark.parametrize("maker", MAKERS[:2])
def test_walk_variant_6_matches_oracle(maker, precision):
    """walk_variant 6 runs each walk step as the 58 sub-operations; the state
    after every step equals the oracle's walk (complex64 storage within the
    reduced-precision bounds)."""
    w = maker()
    sim = _sim(w, walk_variant=6, precision=precision)
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
    assert sim.step_stats()["steps"] == 4
    sim.close()


def test_walk_variant_6_qls_equals_fused_kernel():
    """The CKS read-out on the register-faithful schedule (after its first
    H) gives the fused step kernel's y and p_j."""
    w = wl.walk_n16()
    b_int, j0 = dense.cks_parameters(w.kappa, 1e-3)
    coeffs = dense.cks_coefficients(b_int, j0)[:24]
    fa = _sim(w, walk_variant=6)
    fa.state_init(w.b)
    y, p = fa.apply_qls(coeffs)
    ref = _sim(w)
    ref.state_init(w.b)
    y2, p2 = ref.apply_qls(coeffs)
    assert np.abs(y - y2).max() < 1e-12 and np.abs(p - p2).max() < 1e-12


def test_session_rules():
    """Calls refused while a session is open; end(keep=False) leaves the
    state as it was; end with a working register not 0 is refused and the
    session stays open."""
    w = wl.walk_n16()
    sim = _sim(w)
    sim.state_init(w.b)
    before = gpu_state(sim)
    with pytest.raises(qwalk.QwError) as e:
        sim.faithful_apply("SWAP")
    assert e.value.code == qwalk.QW_ERR_STATE
    sim.faithful_begin()
    for call in (lambda: sim.apply_walk_step(1), lambda: sim.faithful_begin(), lambda: sim.state_init(w.b)):
        with pytest.raises(qwalk.QwError) as e:
            call()
        assert e.value.code == qwalk.QW_ERR_STATE
    sim.faithful_apply("H", "P", "H")
    sim.faithful_end(keep=False)
    compare(gpu_state(sim), before, 0.0)
    sim.faithful_begin()
    sim.faithful_apply("ADDR_COL", "QRAM_COL")
    with pytest.raises(qwalk.QwError) as e:
        sim.faithful_end()
    assert e.value.code == qwalk.QW_ERR_DEVICE_STATUS
    with pytest.raises(qwalk.QwError) as e:
        sim.faithful_apply("H")  # the address register is live
    assert e.value.code == qwalk.QW_ERR_DEVICE_STATUS
    sim.faithful_end(keep=False)
    sim.apply_walk_step(1)
    o = _oracle(w)
    o.apply("T")
    o.apply("W")
    compare(gpu_state(sim), oracle_state(o), TOL64)
    sim.close()
