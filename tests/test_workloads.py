"""The seeded generators of the Table 1 matrices (Sec. V-B): shape, band,
value grid, and the condition numbers Table 1 prints for A, B, C."""
import os

import numpy as np
import pytest

from paper_2303_06890_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("name", "ABCDE")
def test_table1_matrix_is_a_full_positive_band_with_the_printed_s(name):
    n, word, s = wl.TABLE1[name]
    w = wl.table1(name)
    m = w.matrix
    bw = s // 2 - 1
    assert m.n == n and w.s == s
    # footnote b: s = 2^ceil(log2(2 bandwidth + 1)), with the widest such band
    assert wl.next_pow2(2 * bw + 1) == s and wl.next_pow2(2 * bw + 3) > s
    assert m.nnz == n * (2 * bw + 1) - bw * (bw + 1)
    cols = np.repeat(np.arange(n), np.diff(m.colptr))
    assert np.all(np.abs(cols - m.rowidx) <= bw)
    assert np.all(m.val_q15 > 0)
    if word <= 15:  # w-bit fixed point, exact in Q1.15
        assert np.all(m.val_q15.astype(np.int64) % (1 << (15 - word)) == 0)
    # symmetric: the (row, col, value) triples are closed under transposition
    fwd = set(zip(m.rowidx.tolist(), cols.tolist(), m.val_q15.tolist()))
    assert fwd == set(zip(cols.tolist(), m.rowidx.tolist(), m.val_q15.tolist()))
    assert abs(np.linalg.norm(w.b) - 1.0) < 1e-12 and np.all(w.b >= 0)


def test_table1_kappa_within_5_percent_of_the_printed_values():
    rows = [x.split() for x in open(os.path.join(GOLDEN, "table1_j0.txt"))
            if x.strip() and not x.startswith("#")]
    for name, kappa, _ in rows:
        w = wl.table1(name)
        # kappa = 1 / min |lambda(A / s)| (Table 1, footnote a)
        lam = np.linalg.eigvalsh(w.matrix.dense() / w.s)
        k = 1.0 / np.min(np.abs(lam))
        assert abs(k - w.kappa) < 1e-9 * k
        assert abs(k / float(kappa) - 1.0) < 0.05, (name, k, kappa)
