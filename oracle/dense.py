"""Dense FP64 closed forms that pin the register-level oracle.

TEST INFRASTRUCTURE (see the package docstring).

* ``chebyshev``: T_m(A/s) b by the three-term recurrence; by the block
  encoding of the walk (Sec. IV, Eq. (impl) and the CKS identity, Eq. before
  (fx)), the flag-0 block of T~^dag W^m T~ |b~> equals it.
* ``cks_parameters`` / ``cks_coefficients``: Eq. (fx) -- b = kappa^2 ln(kappa/eps),
  j0 = sqrt(b ln(4b/eps)) and a_j = 4 (-1)^j P[X >= b+j+1] with X ~ Bin(2b, 1/2),
  which is the bracketed tail sum sum_{i=j+1}^{b} C(2b, b+i) / 2^{2b}.
* ``f_closed`` / ``f_chebyshev``: both sides of Eq. (fx).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import stats


def chebyshev(a_over_s: np.ndarray, b: np.ndarray, m_max: int) -> list[np.ndarray]:
    """[T_0(H) b, T_1(H) b, ..., T_{m_max}(H) b] for the dense matrix H."""
    b = np.asarray(b, dtype=np.complex128)
    out = [b.copy()]
    if m_max >= 1:
        out.append(a_over_s @ b)
    for _ in range(2, m_max + 1):
        out.append(2.0 * (a_over_s @ out[-1]) - out[-2])
    return out


def cks_parameters(kappa: float, eps: float = 1e-3) -> tuple[int, int]:
    """(b, j0) of Eq. (fx): natural logarithm, b and j0 rounded up to integers."""
    b = math.ceil(kappa * kappa * math.log(kappa / eps))
    j0 = math.ceil(math.sqrt(b * math.log(4.0 * b / eps)))
    return b, j0


def j0_real(kappa: float, eps: float = 1e-3) -> float:
    """j0 = sqrt(b log(4b/eps)) with b = kappa^2 log(kappa/eps), unrounded."""
    b = kappa * kappa * math.log(kappa / eps)
    return math.sqrt(b * math.log(4.0 * b / eps))


def cks_coefficients(b: int, j0: int) -> np.ndarray:
    """a_j, j = 0..j0, of Eq. (fx); the binomial tail is a library routine."""
    j = np.arange(j0 + 1)
    tail = stats.binom.sf(b + j, 2 * b, 0.5)  # P[X > b + j] = P[X >= b + j + 1]
    return 4.0 * np.where(j % 2 == 0, 1.0, -1.0) * tail


def f_closed(x: np.ndarray, b: int) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    return (1.0 - (1.0 - x * x) ** b) / x


def f_chebyshev(x: np.ndarray, coeffs: np.ndarray) -> np.ndarray:
    """sum_j a_j T_{2j+1}(x) for x in [-1, 1]."""
    x = np.asarray(x, dtype=np.float64)
    theta = np.arccos(np.clip(x, -1.0, 1.0))
    j = np.arange(len(coeffs))
    return np.cos(np.outer(theta, 2 * j + 1)) @ coeffs


def qls_reference(a_dense: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x = A^{-1} b / ||A^{-1} b|| by a dense FP64 solve."""
    x = np.linalg.solve(a_dense, b)
    return x / np.linalg.norm(x)


def fidelity(x: np.ndarray, y: np.ndarray) -> float:
    """|<x|y>|^2 / ||y||^2 for unit x."""
    ny = np.linalg.norm(y)
    return float(abs(np.vdot(x, y)) ** 2 / (ny * ny)) if ny > 0 else 0.0


def intuitive_os(cols, l: int) -> int:
    """App. B's intuitive sparsity oracle on one row: k(j, l) for 0 <= l < N.
    cols are the row's s column indices, sorted.  l < s: the l-th column of
    the row ("sparsity mapping"); l >= s: the (l - s)-th column that is not in
    the row ("bijection filler"), found by walking the sorted columns upward
    from l - s and stepping over each one that is not above the running
    index (Alg. "Find k from input l >= s", with the comparison strict: the
    reading that reproduces the example of Sec. III-B)."""
    s = len(cols)
    if l < s:
        return int(cols[l])
    k = l - s
    for c in cols:
        if c > k:
            return k
        k += 1
    return k
