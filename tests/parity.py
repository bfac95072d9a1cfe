"""Helpers that compare the CUDA path's state with the oracle's (test-only)."""
from __future__ import annotations

import numpy as np

KEY_FIELDS = ("jc", "j", "b1", "kc", "k", "b2", "A")


def gpu_state(sim, inst: int = 0) -> dict:
    keys, amps = sim.state_export(inst=inst, key_words=2 if 4 * sim.nb + 34 <= 128 else 10)
    regs = sim.unpack(keys)
    assert np.all(regs[:, 7] == inst)
    return {tuple(int(v) for v in r[:7]): complex(a) for r, a in zip(regs, amps)}


def oracle_state(o) -> dict:
    regs, amps = o.export()
    return {tuple(int(v) for v in r[:7]): complex(a) for r, a in zip(regs, amps)}


def compare(gpu: dict, ref: dict, tol: float, drop_below: float = 0.0) -> dict:
    """Key sets equal (after dropping |a_ref| <= drop_below on both sides) and
    max |delta a| <= tol.  Returns error statistics."""
    if drop_below > 0:
        small = {k for k, v in ref.items() if abs(v) <= drop_below}
        ref = {k: v for k, v in ref.items() if k not in small}
        gpu = {k: v for k, v in gpu.items() if k not in small and abs(v) > drop_below}
    missing = set(ref) - set(gpu)
    extra = set(gpu) - set(ref)
    assert not missing and not extra, (
        f"key sets differ: {len(missing)} missing (e.g. {sorted(missing)[:3]}), "
        f"{len(extra)} extra (e.g. {sorted(extra)[:3]})")
    if not ref:
        return {"max_abs": 0.0, "l2": 0.0, "count": 0}
    d = np.array([gpu[k] - ref[k] for k in ref])
    stats = {"max_abs": float(np.abs(d).max()), "l2": float(np.linalg.norm(d)), "count": len(ref)}
    assert stats["max_abs"] <= tol, stats
    return stats


def compare_union(gpu: dict, ref: dict, max_tol: float, l2_tol: float) -> dict:
    """Reduced-precision comparison: the difference over the union of keys
    (a key missing on one side counts as amplitude 0) must satisfy both
    bounds; so a branch kept on one side only is allowed exactly when its
    amplitude is below max_tol."""
    keys = set(gpu) | set(ref)
    d = np.array([gpu.get(k, 0j) - ref.get(k, 0j) for k in keys]) if keys else np.zeros(1)
    only = [abs(gpu.get(k, 0j)) + abs(ref.get(k, 0j)) for k in set(gpu) ^ set(ref)]
    stats = {"max_abs": float(np.abs(d).max()), "l2": float(np.linalg.norm(d)),
             "count": len(keys), "one_sided": len(only),
             "one_sided_max": float(max(only)) if only else 0.0}
    assert stats["max_abs"] <= max_tol and stats["l2"] <= l2_tol, stats
    return stats


# --- array forms for states with millions of branches ------------------------

def _canonical(regs: np.ndarray, amps: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    regs = np.ascontiguousarray(regs[:, :7], dtype=np.uint64)
    order = np.lexsort(tuple(regs[:, c] for c in range(6, -1, -1)))
    return regs[order], np.asarray(amps)[order]


def gpu_arrays(sim, inst: int = 0) -> tuple[np.ndarray, np.ndarray]:
    keys, amps = sim.state_export(inst=inst, key_words=2 if 4 * sim.nb + 34 <= 128 else 10)
    regs = sim.unpack(keys)
    assert np.all(regs[:, 7] == inst)
    return _canonical(regs, amps)


def oracle_arrays(o) -> tuple[np.ndarray, np.ndarray]:
    return _canonical(*o.export())


def compare_arrays(gpu, ref, tol: float) -> dict:
    """compare() for canonical arrays: identical key lists, max |delta a| <= tol."""
    (kg, ag), (kr, ar) = gpu, ref
    assert kg.shape == kr.shape, f"branch counts differ: {len(kg)} vs {len(kr)}"
    bad = np.flatnonzero(np.any(kg != kr, axis=1))
    assert bad.size == 0, f"{bad.size} keys differ, first at {bad[0]}: {kg[bad[0]]} vs {kr[bad[0]]}"
    d = ag - ar
    stats = {"max_abs": float(np.abs(d).max()) if d.size else 0.0,
             "l2": float(np.linalg.norm(d)), "count": int(len(kr))}
    assert stats["max_abs"] <= tol, stats
    return stats


def compare_union_arrays(gpu, ref, max_tol: float, l2_tol: float) -> dict:
    """compare_union() for canonical arrays (a key on one side only counts as 0)."""
    (kg, ag), (kr, ar) = gpu, ref
    both = np.concatenate([kg, kr])
    _, inv = np.unique(both.view(np.dtype((np.void, 56))).ravel(), return_inverse=True)
    inv = inv.ravel()
    m = int(inv.max()) + 1 if inv.size else 0
    vg = np.zeros(m, dtype=complex)
    vr = np.zeros(m, dtype=complex)
    hg = np.zeros(m, dtype=bool)
    hr = np.zeros(m, dtype=bool)
    vg[inv[:len(kg)]] = ag
    hg[inv[:len(kg)]] = True
    vr[inv[len(kg):]] = ar
    hr[inv[len(kg):]] = True
    d = vg - vr
    one = hg ^ hr
    stats = {"max_abs": float(np.abs(d).max()) if m else 0.0, "l2": float(np.linalg.norm(d)),
             "count": m, "one_sided": int(one.sum()),
             "one_sided_max": float((np.abs(vg) + np.abs(vr))[one].max()) if one.any() else 0.0}
    assert stats["max_abs"] <= max_tol and stats["l2"] <= l2_tol, stats
    return stats
