"""qw_measure_register_noalloc against qw_measure_register, through the C ABI.

The no-allocation entry point serves callers that cannot call cudaMalloc when
they measure: a runtime whose device memory belongs to another allocator with
no headroom left, or a loop that must not enter the allocator for latency.  It
accumulates into a fixed scratch array of the library instead of the
simulator's own histogram (which qw_measure_register may allocate).  It must give the same marginals as the allocating
call, also on consecutive calls (the shared scratch is re-zeroed each time),
and reject lengths above its fixed limit.  This file is collected last so a
failure here stops a -x run only after every other test has run.
"""
import ctypes

import numpy as np
import pytest

from paper_2303_06890_gb300 import qwalk
from paper_2303_06890_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _measure(lib, h, fn, reg, length):
    out = np.zeros(length)
    rc = getattr(lib, fn)(h, 0, qwalk.REGS[reg], out.ctypes.data_as(ctypes.c_void_p), length)
    assert rc == qwalk.QW_OK, (fn, rc, lib.qw_last_error(h).decode())
    return out


@pytest.mark.parametrize("precision", [qwalk.QW_FP64, qwalk.QW_FP32_AMP])
def test_noalloc_measure_matches_allocating_measure_on_consecutive_calls(precision):
    lib = qwalk.load()
    w = wl.walk_n1024()
    sim = qwalk.Sim(w.matrix, s_pad=w.s, precision=precision)
    sim.state_init(w.b)
    sim.apply_walk_step(3)
    h = sim._h
    length = 1 << sim.nb
    # two calls in a row on the same state: a wide register, then a narrow one
    for reg, ln in (("j", length), ("b1", 2)):
        got = _measure(lib, h, "qw_measure_register_noalloc", reg, ln)
        want = _measure(lib, h, "qw_measure_register", reg, ln)
        assert np.abs(got - want).max() <= TOL, reg
    # and again after the state changed
    sim.apply_walk_step(1)
    for reg, ln in (("k", length), ("k", length)):
        got = _measure(lib, h, "qw_measure_register_noalloc", reg, ln)
        want = _measure(lib, h, "qw_measure_register", reg, ln)
        assert np.abs(got - want).max() <= TOL, reg
    assert abs(got.sum() - 1.0) < 1e-6
    sim.close()


def test_noalloc_measure_rejects_length_above_its_scratch():
    lib = qwalk.load()
    w = wl.walk_n16()
    sim = qwalk.Sim(w.matrix, s_pad=w.s)
    sim.state_init(w.b)
    too_long = qwalk.MEASURE_NOALLOC_MAX_LEN + 1
    out = np.zeros(too_long)
    rc = lib.qw_measure_register_noalloc(sim._h, 0, qwalk.REGS["j"],
                                         out.ctypes.data_as(ctypes.c_void_p), too_long)
    assert rc == qwalk.QW_ERR_ARG
    assert "exceeds" in lib.qw_last_error(sim._h).decode()
    # the limit itself is accepted
    ok = np.zeros(qwalk.MEASURE_NOALLOC_MAX_LEN)
    rc = lib.qw_measure_register_noalloc(sim._h, 0, qwalk.REGS["j"],
                                         ok.ctypes.data_as(ctypes.c_void_p), ok.size)
    assert rc == qwalk.QW_OK
    assert abs(ok.sum() - 1.0) < 1e-12
    sim.close()
