"""CPU-side checks of the C-ABI library: it loads, exports every function that
include/qwalk.h declares, validates its inputs before touching a GPU, and its
host-only CKS coefficients agree with the oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2303_06890_gb300 import qwalk
from paper_2303_06890_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "qwalk.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qw_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = qwalk.load()
    names = declared_functions()
    assert len(names) >= 13
    for name in names:
        assert hasattr(lib, name), name
    assert set(qwalk.EXPORTED) == set(names)


def _csc(matrix, **kw):
    cp = np.ascontiguousarray(kw.get("colptr", matrix.colptr), dtype=np.int32)
    ri = np.ascontiguousarray(kw.get("rowidx", matrix.rowidx), dtype=np.int32)
    va = np.ascontiguousarray(kw.get("val", matrix.val_q15), dtype=np.int16)
    c = qwalk.CSC(kw.get("n", matrix.n), ri.size, cp.ctypes.data, ri.ctypes.data, va.ctypes.data,
                  kw.get("s_pad", 0))
    return c, (cp, ri, va)


def _create(csc):
    lib = qwalk.load()
    h = ctypes.c_void_p()
    rc = lib.qw_sim_create(ctypes.byref(csc), 1, None, ctypes.byref(h))
    return rc, lib.qw_last_error(None).decode()


@pytest.mark.parametrize("case", ["unsorted", "duplicate", "range", "asym", "negdiag", "spad", "colptr", "n"])
def test_create_rejects_bad_matrices_before_any_device_work(case):
    m = wl.walk_n16().matrix
    ri = m.rowidx.copy()
    va = m.val_q15.copy()
    cp = m.colptr.copy()
    kw = {}
    lo, hi = cp[0], cp[1]
    if case == "unsorted":
        ri[lo:hi] = ri[lo:hi][::-1]
        kw = dict(rowidx=ri)
    elif case == "duplicate":
        ri[lo + 1] = ri[lo]
        kw = dict(rowidx=ri)
    elif case == "range":
        ri[-1] = m.n
        kw = dict(rowidx=ri)
    elif case == "asym":
        off = next(t for t in range(m.nnz) if ri[t] != np.searchsorted(cp, t, side="right") - 1)
        va[off] = va[off] // 2 + 1
        kw = dict(val=va)
    elif case == "negdiag":
        d = next(t for t in range(cp[0], cp[1]) if ri[t] == 0)
        va[d] = -100
        kw = dict(val=va)
    elif case == "spad":
        kw = dict(s_pad=3)
    elif case == "colptr":
        cp[-1] += 1
        kw = dict(colptr=cp)
    elif case == "n":
        kw = dict(n=1)
    csc, keep = _csc(m, **kw)
    rc, msg = _create(csc)
    want = qwalk.QW_ERR_ARG if case == "n" else qwalk.QW_ERR_CSC
    assert rc == want, (rc, msg)
    assert msg


def test_cks_coefficients_match_oracle():
    from oracle import dense
    for kappa in (2.0, 10.0, 100.0, 403.9):
        c, j0, b = qwalk.cks_coefficients(kappa, 1e-3)
        assert (b, j0) == dense.cks_parameters(kappa, 1e-3)
        ref = dense.cks_coefficients(b, j0)
        assert np.abs(c - ref).max() <= 1e-11 * np.abs(ref).max()


def test_cks_rejects_bad_arguments():
    lib = qwalk.load()
    assert lib.qw_cks_coefficients(0.5, 1e-3, None, 0, None, None) == qwalk.QW_ERR_ARG
    assert lib.qw_cks_coefficients(10.0, 0.0, None, 0, None, None) == qwalk.QW_ERR_ARG
    assert lib.qw_cks_coefficients(10.0, 1e-3, None, 5, None, None) == qwalk.QW_ERR_ARG


def test_null_and_destroy_are_safe():
    lib = qwalk.load()
    assert lib.qw_sim_destroy(None) == 0
    assert lib.qw_state_size(None, 0, None) == qwalk.QW_ERR_ARG
    assert lib.qw_apply_walk_step(None, 1) == qwalk.QW_ERR_ARG
    assert lib.qw_launch_count(None) == 0


@pytest.mark.parametrize("nb", [4, 14, 16])
@pytest.mark.parametrize("key_words", [2, 10])
def test_key_pack_unpack_follow_the_header_layout(nb, key_words):
    """pack_keys / unpack_keys against the layout written out as one big
    integer: b2 | k | kc | b1 | j | jc | A(16) | inst(16) from bit 0."""
    rng = np.random.default_rng(nb)
    widths = {"jc": nb, "j": nb, "b1": 1, "kc": nb, "k": nb, "b2": 1, "A": 16, "inst": 16}
    names = ["jc", "j", "b1", "kc", "k", "b2", "A", "inst"]
    regs = np.stack([rng.integers(0, 1 << widths[f], 500, dtype=np.uint64) for f in names], axis=1)
    keys = qwalk.pack_keys(regs, nb, key_words)
    for row, key in zip(regs, keys):
        v, pos = 0, 0
        for f in ["b2", "k", "kc", "b1", "j", "jc", "A", "inst"]:
            v |= int(row[names.index(f)]) << pos
            pos += widths[f]
        assert [int(x) for x in key] == [(v >> (64 * t)) & ((1 << 64) - 1) for t in range(key_words)]
    assert np.array_equal(qwalk.unpack_keys(keys, nb), regs)


def _header_defines():
    text = open(os.path.join(ROOT, "include", "qwalk.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = text.replace("\\\n", " ")
    return dict(re.findall(r"^#define\s+(QW_\w+)\s+(.*?)\s*$", text, flags=re.M))


def test_faithful_codes_and_step_follow_the_header():
    """The binding's register-faithful codes, table columns and W sequence
    are the header's, and the oracle's codes and sequence agree with them."""
    import oracle

    d = _header_defines()
    for name, code in qwalk.FQ.items():
        assert int(d["QW_FQ_" + name]) == code
    assert oracle.FQ == qwalk.FQ
    assert int(d["QW_FQ_COLS"].replace("(", "").split("+")[0]) + 4 * int(d["QW_FQ_FRAMES"]) == \
        len(qwalk.FQ_COLUMNS)
    assert int(d["QW_WALK_VARIANTS"]) == qwalk.WALK_VARIANTS

    def expand(body):
        out = []
        for tok in re.findall(r"QW_FQ_\w+", body):
            if tok.endswith("_SEQ"):
                out += expand(d[tok])
            else:
                out.append(tok[len("QW_FQ_"):])
        return out

    step = expand(d["QW_FQ_STEP"])
    assert tuple(step) == qwalk.FQ_STEP == tuple(oracle.FQ_STEP)
    assert len(step) == int(d["QW_FQ_STEP_LEN"])


@pytest.mark.parametrize("variant,words", [(7, "walk_variant 7 (positional layout) needs"), (4, "walk_variant 4 (one lane"),
                                           (8, "walk_variant must be 0..7"), (-1, "walk_variant must be 0..7")])
def test_create_rejects_unsupported_walk_variants_before_device_work(variant, words):
    """The slot kernel needs s = 8, 16 or 32, the positional layout s = 8 to
    64 (the N = 16 walk has s = 4); variants outside 0..QW_WALK_VARIANTS - 1 are
    refused.  Both before any device call."""
    lib = qwalk.load()
    csc, keep = _csc(wl.walk_n16().matrix)
    opts = qwalk.Opts()
    lib.qw_sim_opts_default(ctypes.byref(opts))
    opts.walk_variant = variant
    h = ctypes.c_void_p()
    rc = lib.qw_sim_create(ctypes.byref(csc), 1, ctypes.byref(opts), ctypes.byref(h))
    assert rc == qwalk.QW_ERR_ARG
    assert words in lib.qw_last_error(None).decode()
