"""Seeded synthetic workloads for the sparse quantum-walk simulator.

This module only *generates inputs*: a real symmetric sparse matrix in CSC
form with 16-bit fixed-point values, a normalised right-hand side |b>, and the
condition numbers of the quantised matrix.  It holds none of the walk's
arithmetic; both the CUDA path and the CPU oracle consume its output.

The paper (Sec. V-B) draws random symmetric band matrices with fixed-point
entries and preprocesses them: rescale to max-norm <= 1, convert to CSC, pad
rows to a power-of-two sparsity s, and take kappa = 1 / min|lambda(A/s)|.
The recipes below follow that shape with these choices:

* values are Q1.15 two's complement, q = round_half_even(u * 32767), a = q/32768;
* the diagonal is always present and drawn from [0, 1] (a negative diagonal
  element cannot be block-encoded by the walk's isometry, Eq. psi_j), the
  off-diagonal values from [-1, 1];
* off-diagonal symmetric pairs (i < j) are drawn uniformly at random and kept
  while both columns hold fewer than ``smax`` entries;
* |b> is a normal(0, 1) vector normalised to 1 (real).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

Q15_SCALE = 32768.0


@dataclasses.dataclass
class Matrix:
    """A real symmetric sparse matrix in CSC (= CSR, by symmetry) form."""

    n: int
    colptr: np.ndarray  # int32 [n+1]
    rowidx: np.ndarray  # int32 [nnz], sorted within each column
    val_q15: np.ndarray  # int16 [nnz], Q1.15 two's complement

    @property
    def nnz(self) -> int:
        return int(self.colptr[-1])

    @property
    def max_col_nnz(self) -> int:
        return int(np.max(np.diff(self.colptr)))

    def dense(self) -> np.ndarray:
        """Dense float64 copy of the quantised matrix (value q / 32768)."""
        a = np.zeros((self.n, self.n))
        for c in range(self.n):
            lo, hi = self.colptr[c], self.colptr[c + 1]
            a[self.rowidx[lo:hi], c] = self.val_q15[lo:hi].astype(np.float64) / Q15_SCALE
        return a


@dataclasses.dataclass
class Workload:
    name: str
    matrix: Matrix
    b: np.ndarray  # float64 [n], unit norm
    s: int  # padded sparsity (power of two >= max column nnz)
    steps: int
    cond: float  # max|lambda| / min|lambda| of the quantised A
    kappa: float  # 1 / min|lambda(A / s)|, the walk's condition number

    @property
    def n(self) -> int:
        return self.matrix.n


def quantise_q15(u: np.ndarray) -> np.ndarray:
    """Q1.15 code of values in [-1, 1]: round half to even of u * 32767."""
    q = np.rint(np.asarray(u, dtype=np.float64) * 32767.0)
    return np.clip(q, -32767, 32767).astype(np.int16)


def next_pow2(x: int) -> int:
    p = 1
    while p < x:
        p *= 2
    return p


def _symmetric_pattern(n: int, smax: int, band: int, attempts: int,
                       rng: np.random.Generator) -> list[tuple[int, int]]:
    """Upper-triangle off-diagonal positions (i < j) of a symmetric pattern.

    ``band`` = 1 adds the tridiagonal band first; then ``attempts`` uniformly
    random pairs are tried and kept while both columns have < smax entries
    (the diagonal counts as one entry per column).
    """
    count = np.ones(n, dtype=np.int64)  # the diagonal
    present: set[tuple[int, int]] = set()
    pairs: list[tuple[int, int]] = []

    def add(i: int, j: int) -> None:
        if i == j:
            return
        if i > j:
            i, j = j, i
        if (i, j) in present or count[i] >= smax or count[j] >= smax:
            return
        present.add((i, j))
        pairs.append((i, j))
        count[i] += 1
        count[j] += 1

    for d in range(1, band + 1):
        for i in range(n - d):
            add(i, i + d)
    draws = rng.integers(0, n, size=(attempts, 2))
    for i, j in draws:
        add(int(i), int(j))
    return pairs


def _assemble(n: int, diag_q: np.ndarray, pairs: list[tuple[int, int]],
              off_q: np.ndarray) -> Matrix:
    rows = [np.arange(n)]
    cols = [np.arange(n)]
    vals = [diag_q]
    if pairs:
        p = np.asarray(pairs, dtype=np.int64)
        rows += [p[:, 0], p[:, 1]]
        cols += [p[:, 1], p[:, 0]]
        vals += [off_q, off_q]
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals).astype(np.int16)
    order = np.lexsort((r, c))
    r, c, v = r[order], c[order], v[order]
    colptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(colptr, c + 1, 1)
    colptr = np.cumsum(colptr).astype(np.int32)
    return Matrix(n=n, colptr=colptr, rowidx=r.astype(np.int32), val_q15=v)


def _spectrum_stats(m: Matrix, s: int) -> tuple[float, float]:
    if m.n > 4096:
        return float("nan"), float("nan")
    lam = np.linalg.eigvalsh(m.dense())
    amin = float(np.min(np.abs(lam)))
    amax = float(np.max(np.abs(lam)))
    cond = amax / amin if amin > 0 else float("inf")
    kappa = s / amin if amin > 0 else float("inf")
    return cond, kappa


def random_b(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    b = rng.standard_normal(n)
    return b / np.linalg.norm(b)


def random_symmetric(n: int, smax: int, band: int, attempts: int, seed: int) -> Matrix:
    """Diagonal U[0,1], off-diagonal U[-1,1] on a random symmetric pattern."""
    rng = np.random.default_rng(seed)
    pairs = _symmetric_pattern(n, smax, band, attempts, rng)
    diag_q = quantise_q15(rng.uniform(0.0, 1.0, n))
    off_q = quantise_q15(rng.uniform(-1.0, 1.0, len(pairs)))
    return _assemble(n, diag_q, pairs, off_q)


def conditioned_symmetric(n: int, smax: int, attempts: int, cond: float, seed: int) -> Matrix:
    """Tridiagonal-plus-random symmetric matrix with cond(A) close to ``cond``.

    A = c I + alpha O with O the off-diagonal U[-1,1] part, c = 1 and
    alpha = (cond - 1) / (mu_max + cond |mu_min|) from O's extreme eigenvalues,
    so that (c + alpha mu_max) / (c + alpha mu_min) = cond.  Quantisation then
    perturbs the spectrum by ~1e-5; the recorded cond/kappa are recomputed
    from the quantised matrix.
    """
    rng = np.random.default_rng(seed)
    pairs = _symmetric_pattern(n, smax, 1, attempts, rng)
    off = rng.uniform(-1.0, 1.0, len(pairs))
    o = np.zeros((n, n))
    p = np.asarray(pairs)
    o[p[:, 0], p[:, 1]] = off
    o[p[:, 1], p[:, 0]] = off
    mu = np.linalg.eigvalsh(o)
    alpha = (cond - 1.0) / (mu[-1] + cond * abs(mu[0]))
    diag_q = quantise_q15(np.full(n, 1.0))
    off_q = quantise_q15(alpha * off)
    return _assemble(n, diag_q, pairs, off_q)


def _workload(name: str, m: Matrix, b: np.ndarray, steps: int, s: int | None = None,
              spectrum: bool = True) -> Workload:
    s = next_pow2(m.max_col_nnz) if s is None else s
    cond, kappa = _spectrum_stats(m, s) if spectrum else (float("nan"), float("nan"))
    return Workload(name=name, matrix=m, b=b, s=s, steps=steps, cond=cond, kappa=kappa)


# --- the five workloads -------------------------------------------------------

def walk_n16() -> Workload:
    """N=16, <=4 nnz/column at random symmetric positions, 10 walk steps, c128."""
    m = random_symmetric(16, 4, 0, 32, seed=101)
    return _workload("walk_n16_s4", m, random_b(16, 102), steps=10)


def walk_n1024() -> Workload:
    """N=1024, <=8 nnz/column (tridiagonal + random off-band), 100 steps."""
    m = random_symmetric(1024, 8, 1, 1536, seed=201)
    return _workload("walk_n1024_s8", m, random_b(1024, 202), steps=100)


def walk_n16384() -> Workload:
    """N=16384, <=16 nnz/column at random symmetric positions, 20 steps."""
    m = random_symmetric(16384, 16, 0, 6 * 16384, seed=301)
    return _workload("walk_n16384_s16", m, random_b(16384, 302), steps=20)


def qls_n1024() -> Workload:
    """N=1024 tridiagonal + random symmetric, cond(A) ~ 100, QLS."""
    m = conditioned_symmetric(1024, 8, 1536, 100.0, seed=401)
    return _workload("qls_n1024_s8", m, random_b(1024, 402), steps=0)


def batched_sizes(count: int = 256, seed: int = 500) -> list[int]:
    rng = np.random.default_rng(seed)
    return [int(round(2.0 ** x)) for x in rng.uniform(6.0, 12.0, count)]


def batched(count: int = 256, first: int = 0) -> list[Workload]:
    """``count`` walks, N log-uniform in [64, 4096], <=8 nnz/column, 50 steps.

    Instance ``first + i`` uses matrix seed 500 + first + i and |b> seed
    1000 + first + i (``first`` > 0 gives another rank its own instances).
    """
    out = []
    sizes = batched_sizes(count, seed=500 + first)
    for i, n in enumerate(sizes):
        m = random_symmetric(n, 8, 1, (3 * n) // 2, seed=500 + first + i)
        out.append(_workload(f"batched_{first + i}_n{n}", m, random_b(n, 1000 + first + i), steps=50,
                             s=8, spectrum=False))
    return out


def small_random(n: int, smax: int, seed: int, band: int = 0, attempts: int | None = None,
                 steps: int = 4) -> Workload:
    """Small random case for parity sweeps (several tiles and a ragged tail)."""
    attempts = 2 * n if attempts is None else attempts
    m = random_symmetric(n, smax, band, attempts, seed=seed)
    return _workload(f"random_n{n}_s{smax}_seed{seed}", m, random_b(n, seed + 7), steps=steps)


# --- matrices shaped like the paper's Table 1 (Sec. V-B) ----------------------

TABLE1 = {  # name: (N, word length w, s) as printed in Table 1
    "A": (16, 8, 8),
    "B": (128, 8, 16),
    "C": (1024, 8, 32),
    "D": (8192, 16, 32),
    "E": (16384, 32, 64),
}


def band_positive(n: int, bandwidth: int, word: int, seed: int) -> Matrix:
    """Positive symmetric band matrix of Sec. V-B: every entry with
    |i - j| <= bandwidth is a w-bit fixed-point number in (0, 1).

    Entries are drawn as uniform integers m in [1, 2^w - 1], value m / 2^w (0
    is excluded so the band is full).  For w <= 15 the value is exact in
    Q1.15; for w > 15 it is rounded half to even to 15 fractional bits and
    kept in [2^-15, 1 - 2^-15] (positive, like the w-bit value).
    """
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for dist in range(bandwidth + 1):
        m = rng.integers(1, 1 << word, n - dist, dtype=np.int64)
        if word <= 15:
            q = m << (15 - word)
        else:
            q = np.rint(m.astype(np.float64) / float(1 << (word - 15))).astype(np.int64)
        q = np.clip(q, 1, 32767)
        i = np.arange(n - dist)
        rows.append(i)
        cols.append(i + dist)
        vals.append(q)
        if dist:
            rows.append(i + dist)
            cols.append(i)
            vals.append(q)
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals).astype(np.int16)
    order = np.lexsort((r, c))
    r, c, v = r[order], c[order], v[order]
    colptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(colptr, c + 1, 1)
    return Matrix(n=n, colptr=np.cumsum(colptr).astype(np.int32), rowidx=r.astype(np.int32), val_q15=v)


# Matrix seeds: for A, B, C (whose kappa Table 1 prints: 1.0e2, 6.6e2, 5.0e3)
# the first seed from 600 on whose kappa = s / min|lambda(A)| is within 5 % of
# the printed value (103.0, 665.3, 4906.6); D and E print none.
TABLE1_SEEDS = {"A": 631, "B": 612, "C": 733, "D": 603, "E": 604}


def table1(name: str, steps: int = 50, seed: int | None = None) -> Workload:
    """Matrix ``name`` of Table 1 (A..E): N and w as printed, the widest band
    whose row count 2 bandwidth + 1 rounds up to the printed s (footnote b),
    |b> uniform random in [0, 1) normalised (Sec. V-B), seed 700 + i for
    i = 0..4 (A..E)."""
    n, word, s = TABLE1[name]
    i = "ABCDE".index(name)
    bw = s // 2 - 1
    m = band_positive(n, bw, word, seed=TABLE1_SEEDS[name] if seed is None else seed)
    rng = np.random.default_rng(700 + i)
    b = rng.uniform(0.0, 1.0, n)
    b /= np.linalg.norm(b)
    return _workload(f"table1_{name}_n{n}_w{word}_s{s}", m, b, steps=steps, s=s, spectrum=n <= 4096)


CONFIGS = {
    "walk_n16": walk_n16,
    "walk_n1024": walk_n1024,
    "walk_n16384": walk_n16384,
    "qls_n1024": qls_n1024,
}


def ceil_log2(x: int) -> int:
    return max(0, math.ceil(math.log2(x))) if x > 1 else 0
