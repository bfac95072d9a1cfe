"""CPU oracle for the sparse-state quantum walk (arXiv 2303.06890).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA path.  ``qw_oracle.c`` is the register-level simulator (plain C,
FP64, single thread); ``dense.py`` holds the dense closed forms used to pin
it (Chebyshev recurrence, CKS coefficients, dense solve).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qw_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libqw_oracle.so")

OP = {"T": 0, "TDAG": 1, "W": 2, "P": 3, "S": 4, "H": 5, "R": 6, "RDAG": 7,
      "OA": 8, "OS": 9, "OSDAG": 10, "ALLOC_A": 11, "FREE_A": 12}
REGS = ("jc", "j", "b1", "kc", "k", "b2", "A")
TAU64 = 1e-13

# register-faithful sub-operations (qw_oracle.c): the working registers of
# O_s', O_A' and Alg. 1 kept per branch between them
FQ = {"ADDR_COL": 1, "QRAM_COL": 2, "QBS_FWD": 3, "QBS_BWD": 4, "SWAP": 5, "ADDR_VAL": 6, "QRAM_VAL": 7,
      "R": 8, "RDAG": 9, "H": 10, "P": 11, "S": 12, "ALLOC_A": 13, "FREE_A": 14}
G_REGS = ("addr", "left", "right", "mid", "midval", "flag", "cl", "ce")  # then 8 frames of (mid, midval, cl, ce)
FQ_OS = ("ADDR_COL", "QRAM_COL", "ADDR_COL", "QBS_FWD", "QBS_BWD", "SWAP")
FQ_OSDAG = ("SWAP", "QBS_FWD", "QBS_BWD", "ADDR_COL", "QRAM_COL", "ADDR_COL")
FQ_OA = ("ADDR_VAL", "QRAM_VAL", "ADDR_VAL")
# W = S T~ P T~^dag as sub-operations (Alg. T~, Alg. "Quantum walk operator")
FQ_STEP = (("ALLOC_A",) + FQ_OSDAG + FQ_OA + FQ_OS + ("RDAG",) + FQ_OSDAG + FQ_OA + ("H", "FREE_A", "P", "ALLOC_A", "H")
           + FQ_OA + FQ_OS + ("R",) + FQ_OSDAG + FQ_OA + FQ_OS + ("FREE_A", "S"))

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no -march flags: x86 and Arm alike)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    i64, i32, u64, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
    lib.or_create.restype = P
    lib.or_create.argtypes = [i32, P, P, P, i32, dbl]
    lib.or_destroy.argtypes = [P]
    for name in ("or_nb", "or_size", "or_violations", "or_max_live_bits"):
        getattr(lib, name).restype = i64
        getattr(lib, name).argtypes = [P]
    lib.or_set_tau.argtypes = [P, dbl]
    lib.or_set_rot_bits.argtypes = [P, ctypes.c_int]
    lib.or_image.argtypes = [P, i64, i64, P, P]
    lib.or_init_b.argtypes = [P, P, P]
    lib.or_import.argtypes = [P, P, P, i64]
    lib.or_export.restype = i64
    lib.or_export.argtypes = [P, P, P, i64]
    lib.or_apply.argtypes = [P, ctypes.c_int]
    lib.or_flag0.argtypes = [P, P]
    lib.or_marginal.argtypes = [P, ctypes.c_int, P, i64]
    lib.or_norm2.restype = dbl
    lib.or_norm2.argtypes = [P]
    lib.or_qbs.restype = u64
    lib.or_qbs.argtypes = [P, u64, u64]
    lib.or_os_single.argtypes = [P, u64, u64, u64, ctypes.c_int, P, P]
    lib.or_apply_faithful.argtypes = [P, ctypes.c_int]
    lib.or_export_faithful.restype = i64
    lib.or_export_faithful.argtypes = [P, P, P, i64]
    lib.or_faithful_ng.restype = ctypes.c_int
    lib.or_faithful_ng.argtypes = []
    lib.or_faithful_addr_bits.restype = ctypes.c_int
    lib.or_faithful_addr_bits.argtypes = [P]
    lib.or_faithful_live_bits.restype = i64
    lib.or_faithful_live_bits.argtypes = [P]
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Oracle:
    """One register-level sparse state over the QRAM image of one matrix."""

    def __init__(self, matrix, s: int, tau: float = TAU64, rot_bits: int = 0):
        lib = _load()
        self._colptr = np.ascontiguousarray(matrix.colptr, dtype=np.int32)
        self._rowidx = np.ascontiguousarray(matrix.rowidx, dtype=np.int32)
        self._val = np.ascontiguousarray(matrix.val_q15, dtype=np.int16)
        self.n = int(matrix.n)
        self.s = int(s)
        self._h = lib.or_create(self.n, _ptr(self._colptr), _ptr(self._rowidx), _ptr(self._val),
                                self.s, float(tau))
        if not self._h:
            raise ValueError("oracle: invalid matrix or sparsity")
        self.nb = int(lib.or_nb(self._h))
        if rot_bits:
            lib.or_set_rot_bits(self._h, int(rot_bits))

    def __del__(self):
        if getattr(self, "_h", None):
            _load().or_destroy(self._h)
            self._h = None

    # --- state -----------------------------------------------------------
    def init_b(self, b: np.ndarray) -> None:
        b = np.asarray(b)
        re = np.ascontiguousarray(b.real, dtype=np.float64)
        im = np.ascontiguousarray(b.imag if np.iscomplexobj(b) else np.zeros(self.n), dtype=np.float64)
        if _load().or_init_b(self._h, _ptr(re), _ptr(im)):
            raise MemoryError

    def set_state(self, regs: np.ndarray, amps: np.ndarray) -> None:
        regs = np.ascontiguousarray(regs, dtype=np.uint64).reshape(-1, 6)
        a = np.ascontiguousarray(np.stack([np.real(amps), np.imag(amps)], axis=1), dtype=np.float64)
        if _load().or_import(self._h, _ptr(regs), _ptr(a), regs.shape[0]):
            raise MemoryError

    def apply(self, *ops: str) -> None:
        for op in ops:
            if _load().or_apply(self._h, OP[op]):
                raise RuntimeError(f"oracle op {op} failed")

    def size(self) -> int:
        return int(_load().or_size(self._h))

    def export(self) -> tuple[np.ndarray, np.ndarray]:
        """(regs [M,7] uint64 in REGS order, amps [M] complex128), oracle order."""
        m = self.size()
        regs = np.zeros((m, 7), dtype=np.uint64)
        a = np.zeros((m, 2), dtype=np.float64)
        _load().or_export(self._h, _ptr(regs), _ptr(a), m)
        return regs, a[:, 0] + 1j * a[:, 1]

    def flag0(self) -> np.ndarray:
        y = np.zeros(2 * self.n)
        _load().or_flag0(self._h, _ptr(y))
        return y[0::2] + 1j * y[1::2]

    def marginal(self, reg: str, length: int) -> np.ndarray:
        p = np.zeros(length)
        if _load().or_marginal(self._h, REGS.index(reg), _ptr(p), length):
            raise ValueError(reg)
        return p

    def apply_faithful(self, *ops: str) -> None:
        """Register-faithful sub-operations (FQ), in order."""
        for op in ops:
            if _load().or_apply_faithful(self._h, FQ[op]):
                raise RuntimeError(f"oracle sub-operation {op} failed")

    def export_faithful(self) -> tuple[np.ndarray, np.ndarray]:
        """(regs [M, 7 + NG] uint64: jc, j, b1, kc, k, b2, A, then the working
        registers G_REGS and the stack frames; amps [M]), oracle order."""
        ng = _load().or_faithful_ng()
        m = self.size()
        regs = np.zeros((m, 7 + ng), dtype=np.uint64)
        a = np.zeros((m, 2), dtype=np.float64)
        _load().or_export_faithful(self._h, _ptr(regs), _ptr(a), m)
        return regs, a[:, 0] + 1j * a[:, 1]

    @property
    def faithful_addr_bits(self) -> int:
        return int(_load().or_faithful_addr_bits(self._h))

    @property
    def faithful_live_bits(self) -> int:
        return int(_load().or_faithful_live_bits(self._h))

    def norm2(self) -> float:
        return float(_load().or_norm2(self._h))

    @property
    def violations(self) -> int:
        return int(_load().or_violations(self._h))

    @property
    def max_live_bits(self) -> int:
        return int(_load().or_max_live_bits(self._h))

    # --- single-branch probes ----------------------------------------------
    def qbs(self, j: int, target: int) -> int:
        return int(_load().or_qbs(self._h, j, target))

    def os_single(self, j: int, k: int, kc: int, dagger: bool = False) -> tuple[int, int]:
        ko = ctypes.c_uint64()
        kco = ctypes.c_uint64()
        _load().or_os_single(self._h, j, k, kc, int(dagger), ctypes.byref(ko), ctypes.byref(kco))
        return int(ko.value), int(kco.value)

    def image(self, j: int, l: int) -> tuple[int, int]:
        v = ctypes.c_uint32()
        c = ctypes.c_uint32()
        _load().or_image(self._h, j, l, ctypes.byref(v), ctypes.byref(c))
        return int(v.value), int(c.value)


def walk(matrix, s: int, b: np.ndarray, steps: int, tau: float = TAU64) -> Oracle:
    """|phi_m> = W^m T~ |b~> (the walk workload)."""
    o = Oracle(matrix, s, tau)
    o.init_b(b)
    o.apply("T")
    for _ in range(steps):
        o.apply("W")
    return o


def qls(matrix, s: int, b: np.ndarray, coeffs: np.ndarray, tau: float = TAU64,
        iterations: int | None = None):
    """CKS linear solver by the paper's iteration (Sec. V-B).

    tau_0 = T~^dag W T~ |b~>, tau_j = T~^dag W^2 T~ tau_{j-1}; the flag-0
    block of tau_j is T_{2j+1}(A/s) b.  Returns (Y, ys) with ys[j] the flag-0
    block of tau_j and Y = sum_j coeffs[j] ys[j].
    """
    o = Oracle(matrix, s, tau)
    o.init_b(b)
    count = len(coeffs) if iterations is None else iterations
    ys = []
    Y = np.zeros(o.n, dtype=np.complex128)
    for j in range(count):
        o.apply("T", "W") if j == 0 else o.apply("T", "W", "W")
        o.apply("TDAG")
        y = o.flag0()
        ys.append(y)
        Y = Y + coeffs[j] * y
    return Y, ys, o
