"""Thin ctypes binding of the C ABI in include/qwalk.h (argument marshalling only).

Every step of the walk runs in libqwalk.so's CUDA kernels; this module only
converts numpy arrays to pointers and error codes to exceptions.  PyTorch, when
present, supplies the CUDA stream.  Loading fails loudly when the library is
missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

QW_OK = 0
QW_ERR_ARG = -1
QW_ERR_CSC = -2
QW_ERR_CAPACITY = -3
QW_ERR_CUDA = -4
QW_ERR_DEVICE_STATUS = -5
QW_ERR_STATE = -6
QW_FP64 = 0
QW_FP32_AMP = 1
REGS = {"jc": 0, "j": 1, "b1": 2, "kc": 3, "k": 4, "b2": 5}

EXPORTED = ("qw_sim_opts_default", "qw_sim_create", "qw_state_init", "qw_apply_walk_step",
            "qw_enqueue_walk_steps", "qw_sync",
            "qw_cks_coefficients", "qw_apply_qls", "qw_measure_register", "qw_state_size",
            "qw_state_export", "qw_sim_info", "qw_step_stats", "qw_launch_count", "qw_sim_destroy",
            "qw_last_error", "qw_measure_register_noalloc", "qw_autotune", "qw_state_import",
            "qw_part_owner", "qw_part_outbox", "qw_part_inbox", "qw_part_norm", "qw_part_set_norm",
            "qw_part_walk", "qw_faithful_info", "qw_faithful_begin", "qw_faithful_apply",
            "qw_faithful_export", "qw_faithful_end")
MEASURE_NOALLOC_MAX_LEN = 65536
WALK_VARIANTS = 8  # QW_WALK_VARIANTS

# register-faithful sub-operations (QW_FQ_* of qwalk.h)
FQ = {"ADDR_COL": 1, "QRAM_COL": 2, "QBS_FWD": 3, "QBS_BWD": 4, "SWAP": 5, "ADDR_VAL": 6, "QRAM_VAL": 7,
      "R": 8, "RDAG": 9, "H": 10, "P": 11, "S": 12, "ALLOC_A": 13, "FREE_A": 14}
FQ_FRAMES = 8
FQ_COLUMNS = (("inst", "jc", "j", "b1", "kc", "k", "b2", "A", "addr", "left", "right", "mid", "midval", "flag",
               "cl", "ce") + tuple(f"{n}{f}" for f in range(FQ_FRAMES) for n in ("mid", "midval", "cl", "ce")))
FQ_OS = ("ADDR_COL", "QRAM_COL", "ADDR_COL", "QBS_FWD", "QBS_BWD", "SWAP")
# Alg. 1 forward then backward is k ^= index, its own inverse: O_s'^dag keeps that pair's order
FQ_OSDAG = ("SWAP", "QBS_FWD", "QBS_BWD", "ADDR_COL", "QRAM_COL", "ADDR_COL")
FQ_OA = ("ADDR_VAL", "QRAM_VAL", "ADDR_VAL")
# W = S T~ P T~^dag (QW_FQ_STEP)
FQ_STEP = (("ALLOC_A",) + FQ_OSDAG + FQ_OA + FQ_OS + ("RDAG",) + FQ_OSDAG + FQ_OA + ("H", "FREE_A", "P", "ALLOC_A", "H")
           + FQ_OA + FQ_OS + ("R",) + FQ_OSDAG + FQ_OA + FQ_OS + ("FREE_A", "S"))


class QwError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"qwalk error {code}: {msg}")
        self.code = code


class CSC(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int32), ("colptr", ctypes.c_void_p),
                ("rowidx", ctypes.c_void_p), ("val_q15", ctypes.c_void_p), ("s_pad", ctypes.c_int32)]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("fuse_reflection", ctypes.c_int32),
                ("prune_tau", ctypes.c_double), ("row_capacity", ctypes.c_int32),
                ("warp_capacity", ctypes.c_int32), ("renorm", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("walk_variant", ctypes.c_int32),
                ("graphs", ctypes.c_int32), ("spill_rows", ctypes.c_int32), ("rot_bits", ctypes.c_int32),
                ("overflow_fallback", ctypes.c_int32), ("nparts", ctypes.c_int32), ("part", ctypes.c_int32),
                ("outbox_capacity", ctypes.c_int64)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libqwalk.so (building it first if asked); raise if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError(f"libqwalk.so not built: {path}")
        _build.build()
    lib = ctypes.CDLL(path)
    P, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.qw_sim_opts_default.argtypes = [P]
    lib.qw_sim_opts_default.restype = None
    lib.qw_sim_create.argtypes = [P, i32, P, P]
    lib.qw_state_init.argtypes = [P, i32, P, P, i32, i32]
    lib.qw_apply_walk_step.argtypes = [P, i64]
    lib.qw_enqueue_walk_steps.argtypes = [P, i64]
    lib.qw_sync.argtypes = [P]
    lib.qw_cks_coefficients.argtypes = [dbl, dbl, P, i64, P, P]
    lib.qw_apply_qls.argtypes = [P, i32, P, i64, P, P]
    lib.qw_measure_register.argtypes = [P, i32, i32, P, i64]
    lib.qw_measure_register_noalloc.argtypes = [P, i32, i32, P, i64]
    lib.qw_state_size.argtypes = [P, i32, P]
    lib.qw_state_export.argtypes = [P, i32, i32, P, P, i64, P]
    lib.qw_sim_info.argtypes = [P, P, P, P, P]
    lib.qw_step_stats.argtypes = [P, P, i32, i32]
    lib.qw_autotune.argtypes = [P, i32, P, P]
    lib.qw_state_import.argtypes = [P, i32, P, P, i64]
    lib.qw_part_owner.argtypes = [i32, i32, i32, i32]
    lib.qw_part_outbox.argtypes = [P, i32, P, i64, P]
    lib.qw_part_inbox.argtypes = [P, P, i64]
    lib.qw_part_norm.argtypes = [P, P]
    lib.qw_part_set_norm.argtypes = [P, dbl]
    lib.qw_part_walk.argtypes = [P, i32, i64]
    lib.qw_faithful_info.argtypes = [P, P, P, P]
    lib.qw_faithful_begin.argtypes = [P]
    lib.qw_faithful_apply.argtypes = [P, P, i32]
    lib.qw_faithful_export.argtypes = [P, P, P, i64, P]
    lib.qw_faithful_end.argtypes = [P, i32]
    for name in ("qw_part_owner", "qw_part_outbox", "qw_part_inbox", "qw_part_norm", "qw_part_set_norm",
                 "qw_part_walk"):
        getattr(lib, name).restype = ctypes.c_int
    lib.qw_launch_count.argtypes = [P]
    lib.qw_launch_count.restype = i64
    lib.qw_sim_destroy.argtypes = [P]
    lib.qw_last_error.argtypes = [P]
    lib.qw_last_error.restype = ctypes.c_char_p
    for name in ("qw_sim_create", "qw_state_init", "qw_apply_walk_step", "qw_enqueue_walk_steps",
                 "qw_sync", "qw_cks_coefficients",
                 "qw_apply_qls", "qw_measure_register", "qw_measure_register_noalloc",
                 "qw_state_size", "qw_state_export",
                 "qw_sim_info", "qw_step_stats", "qw_autotune", "qw_state_import", "qw_sim_destroy",
                 "qw_faithful_info", "qw_faithful_begin", "qw_faithful_apply", "qw_faithful_export",
                 "qw_faithful_end"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def current_stream() -> int | None:
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


def cks_coefficients(kappa: float, eps: float = 1e-3) -> tuple[np.ndarray, int, int]:
    """qw_cks_coefficients: (a_0..a_j0, j0, b) of Eq. (fx)."""
    lib = load()
    j0 = ctypes.c_int64()
    b = ctypes.c_int64()
    rc = lib.qw_cks_coefficients(float(kappa), float(eps), None, 0, ctypes.byref(j0), ctypes.byref(b))
    if rc:
        raise QwError(rc, "qw_cks_coefficients: bad kappa or eps")
    out = np.zeros(j0.value + 1)
    rc = lib.qw_cks_coefficients(float(kappa), float(eps), _p(out), out.size, None, None)
    if rc:
        raise QwError(rc, "qw_cks_coefficients")
    return out, int(j0.value), int(b.value)


_FIELD_ORDER = {"jc": 0, "j": 1, "b1": 2, "kc": 3, "k": 4, "b2": 5, "A": 6, "inst": 7}


def _fields(nb: int) -> list[tuple[str, int]]:
    """Packed key layout of qw_state_export, from bit 0 up."""
    return [("b2", 1), ("k", nb), ("kc", nb), ("b1", 1), ("j", nb), ("jc", nb), ("A", 16), ("inst", 16)]


def pack_keys(regs: np.ndarray, nb: int, key_words: int = 2) -> np.ndarray:
    """[M, 8] (jc, j, b1, kc, k, b2, A, inst) -> packed keys [M, key_words]."""
    regs = np.asarray(regs, dtype=np.uint64).reshape(len(regs), -1)
    out = np.zeros((len(regs), key_words), dtype=np.uint64)
    pos = 0
    for name, w in _fields(nb):
        v = regs[:, _FIELD_ORDER[name]] & np.uint64((1 << w) - 1)
        word, off = divmod(pos, 64)
        if word < key_words:
            out[:, word] |= v << np.uint64(off)
        if off + w > 64 and word + 1 < key_words:  # the field continues in the next word
            out[:, word + 1] |= v >> np.uint64(64 - off)
        pos += w
    return out


def unpack_keys(keys: np.ndarray, nb: int) -> np.ndarray:
    """Packed keys [M, key_words] -> [M, 8] (jc, j, b1, kc, k, b2, A, inst)."""
    keys = np.asarray(keys, dtype=np.uint64).reshape(len(keys), -1)
    out = np.zeros((len(keys), 8), dtype=np.uint64)
    pos = 0
    for name, w in _fields(nb):
        word, off = divmod(pos, 64)
        if word < keys.shape[1]:
            v = keys[:, word] >> np.uint64(off)
            if off + w > 64 and word + 1 < keys.shape[1]:
                v = v | (keys[:, word + 1] << np.uint64(64 - off))
            out[:, _FIELD_ORDER[name]] = v & np.uint64((1 << w) - 1)
        pos += w
    return out


class Sim:
    """qw_sim_create ... qw_sim_destroy for one or several matrices."""

    def __init__(self, matrices, s_pad: int = 0, precision: int = QW_FP64, fuse_reflection: bool = True,
                 prune_tau: float = 0.0, row_capacity: int = 0, warp_capacity: int = 0,
                 renorm: int = -1, stream: int | None = None, walk_variant: int = 0,
                 graphs: bool = True, spill_rows: int = 0, rot_bits: int = 0, overflow_fallback: bool = True,
                 nparts: int = 1, part: int = 0, outbox_capacity: int = 0):
        lib = load()
        if not isinstance(matrices, (list, tuple)):
            matrices = [matrices]
        self._keep = []
        arr = (CSC * len(matrices))()
        for i, m in enumerate(matrices):
            cp = np.ascontiguousarray(m.colptr, dtype=np.int32)
            ri = np.ascontiguousarray(m.rowidx, dtype=np.int32)
            va = np.ascontiguousarray(m.val_q15, dtype=np.int16)
            self._keep += [cp, ri, va]
            arr[i] = CSC(int(m.n), int(ri.size), cp.ctypes.data, ri.ctypes.data, va.ctypes.data, int(s_pad))
        opts = Opts()
        lib.qw_sim_opts_default(ctypes.byref(opts))
        opts.precision = precision
        opts.fuse_reflection = int(bool(fuse_reflection))
        opts.prune_tau = prune_tau
        opts.row_capacity = row_capacity
        opts.warp_capacity = warp_capacity
        opts.renorm = renorm
        opts.stream = current_stream() if stream is None else stream
        opts.walk_variant = walk_variant
        opts.graphs = int(bool(graphs))
        opts.spill_rows = int(spill_rows)
        opts.rot_bits = int(rot_bits)
        opts.overflow_fallback = int(bool(overflow_fallback))
        opts.nparts = int(nparts)
        opts.part = int(part)
        opts.outbox_capacity = int(outbox_capacity)
        h = ctypes.c_void_p()
        rc = lib.qw_sim_create(arr, len(matrices), ctypes.byref(opts), ctypes.byref(h))
        if rc:
            raise QwError(rc, lib.qw_last_error(None).decode())
        self._h = h
        self.ns = [int(m.n) for m in matrices]
        nb, s, ni, by = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        lib.qw_sim_info(h, ctypes.byref(nb), ctypes.byref(s), ctypes.byref(ni), ctypes.byref(by))
        self.nb, self.s, self.num_instances, self.device_bytes = nb.value, s.value, ni.value, by.value

    def _check(self, rc: int) -> None:
        if rc:
            raise QwError(rc, load().qw_last_error(self._h).decode())

    def close(self) -> None:
        if getattr(self, "_h", None):
            load().qw_sim_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # --- the ABI calls ------------------------------------------------------
    def state_init(self, b, inst: int = 0, apply_T: bool = True) -> None:
        b = np.asarray(b)
        re = np.ascontiguousarray(b.real, dtype=np.float64)
        im = np.ascontiguousarray(b.imag, dtype=np.float64) if np.iscomplexobj(b) else None
        self._check(load().qw_state_init(self._h, inst, _p(re), None if im is None else _p(im),
                                         re.size, int(bool(apply_T))))

    def apply_walk_step(self, nsteps: int = 1) -> None:
        self._check(load().qw_apply_walk_step(self._h, int(nsteps)))

    def autotune(self, steps_per_candidate: int = 8) -> tuple[int, list[float]]:
        """qw_autotune: (chosen variant, [us/step of variants 0..WALK_VARIANTS-1])."""
        choice = ctypes.c_int32()
        us = np.zeros(WALK_VARIANTS)
        self._check(load().qw_autotune(self._h, int(steps_per_candidate), ctypes.byref(choice), _p(us)))
        return int(choice.value), [float(v) for v in us]

    def enqueue_walk_steps(self, nsteps: int = 1) -> None:
        self._check(load().qw_enqueue_walk_steps(self._h, int(nsteps)))

    def sync(self) -> None:
        self._check(load().qw_sync(self._h))

    def apply_qls(self, coeffs: np.ndarray, inst: int = 0) -> tuple[np.ndarray, np.ndarray]:
        coeffs = np.ascontiguousarray(coeffs, dtype=np.float64)
        j0 = coeffs.size - 1
        y = np.zeros(2 * self.ns[inst])
        p = np.zeros(j0 + 1)
        self._check(load().qw_apply_qls(self._h, inst, _p(coeffs), j0, _p(y), _p(p)))
        return y[0::2] + 1j * y[1::2], p

    def measure_register(self, reg: str, length: int, inst: int = 0, out: np.ndarray | None = None) -> np.ndarray:
        """qw_measure_register into ``out`` (float64, contiguous; e.g. a view of
        pinned host memory) or a new array."""
        if out is None:
            out = np.zeros(int(length))
        if out.dtype != np.float64 or not out.flags.c_contiguous or out.size != int(length):
            raise ValueError("out must be a contiguous float64 array of the given length")
        self._check(load().qw_measure_register(self._h, inst, REGS[reg], _p(out), out.size))
        return out

    def measure_register_noalloc(self, reg: str, length: int, inst: int = 0) -> np.ndarray:
        """qw_measure_register_noalloc: the same marginal without any device
        allocation (fixed scratch in the library; length <= 65536)."""
        out = np.zeros(int(length))
        self._check(load().qw_measure_register_noalloc(self._h, inst, REGS[reg], _p(out), out.size))
        return out

    def state_size(self, inst: int = -1) -> int:
        c = ctypes.c_int64()
        self._check(load().qw_state_size(self._h, inst, ctypes.byref(c)))
        return int(c.value)

    def state_export(self, inst: int = -1, key_words: int = 2) -> tuple[np.ndarray, np.ndarray]:
        """(keys [M, key_words] uint64, amps [M] complex128), keys ascending."""
        n = self.state_size(inst)
        keys = np.zeros((max(n, 1), key_words), dtype=np.uint64)
        amps = np.zeros((max(n, 1), 2))
        c = ctypes.c_int64()
        self._check(load().qw_state_export(self._h, inst, key_words, _p(keys), _p(amps), n,
                                           ctypes.byref(c)))
        m = min(n, int(c.value))
        return keys[:m], amps[:m, 0] + 1j * amps[:m, 1]

    STAT_NAMES = ("rows", "in", "after_rdag", "after_h1", "after_hph", "out", "steps")

    def step_stats(self, reset: bool = False) -> dict:
        """qw_step_stats: per-op branch counters summed over the steps run."""
        out = np.zeros(8, dtype=np.int64)
        self._check(load().qw_step_stats(self._h, _p(out), 8, int(bool(reset))))
        return dict(zip(self.STAT_NAMES, (int(v) for v in out[:7])))

    def state_import(self, keys: np.ndarray, amps: np.ndarray) -> None:
        """qw_state_import: replace the state by packed keys [M, W] and amplitudes."""
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        a = np.ascontiguousarray(np.stack([np.real(amps), np.imag(amps)], axis=1), dtype=np.float64)
        self._check(load().qw_state_import(self._h, keys.shape[1], _p(keys), _p(a), keys.shape[0]))

    def pack(self, regs: np.ndarray, key_words: int = 2) -> np.ndarray:
        """[M, 8] (jc, j, b1, kc, k, b2, A, inst) -> packed keys [M, key_words]."""
        return pack_keys(regs, self.nb, key_words)

    def launch_count(self) -> int:
        return int(load().qw_launch_count(self._h))

    def faithful_info(self) -> dict:
        """qw_faithful_info: address width, key bits, live bits at the widest
        point, and whether the register-faithful layout fits."""
        aw, kb, live = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        rc = load().qw_faithful_info(self._h, ctypes.byref(aw), ctypes.byref(kb), ctypes.byref(live))
        return {"addr_bits": aw.value, "key_bits": kb.value, "live_bits": live.value, "fits": rc == QW_OK}

    def faithful_begin(self) -> None:
        """qw_faithful_begin: open a register-faithful session on the state."""
        self._check(load().qw_faithful_begin(self._h))

    def faithful_apply(self, *ops: str) -> None:
        """qw_faithful_apply: sub-operations by name (keys of FQ), in order."""
        codes = np.array([FQ[o] for o in ops], dtype=np.int32)
        self._check(load().qw_faithful_apply(self._h, _p(codes) if len(codes) else None, len(codes)))

    def faithful_export(self) -> tuple[np.ndarray, np.ndarray]:
        """qw_faithful_export: (regs [M, len(FQ_COLUMNS)] uint64, rows ascending;
        amps [M] complex128)."""
        c = ctypes.c_int64()
        self._check(load().qw_faithful_export(self._h, None, None, 0, ctypes.byref(c)))
        n = int(c.value)
        regs = np.zeros((max(n, 1), len(FQ_COLUMNS)), dtype=np.uint64)
        a = np.zeros((max(n, 1), 2))
        self._check(load().qw_faithful_export(self._h, _p(regs), _p(a), n, ctypes.byref(c)))
        return regs[:n], a[:n, 0] + 1j * a[:n, 1]

    def faithful_end(self, keep: bool = True) -> None:
        """qw_faithful_end: store the list as one walk step's output (keep) or
        drop it."""
        self._check(load().qw_faithful_end(self._h, int(bool(keep))))

    def unpack(self, keys: np.ndarray) -> np.ndarray:
        """Packed keys -> [M, 8] (jc, j, b1, kc, k, b2, A, inst) per the header's layout."""
        return unpack_keys(keys, self.nb)
