"""Host logic of the flat path's radix sort (`qw_sort_chunks.h`): which key
bits its passes sort by.  The header is compiled here with the host C++
compiler (no CUDA) and checked against a restatement of its definition: the
varying bits in order of significance, 64 to a chunk, each chunk 8 bits a
pass; and sorting by the chunks' compacted keys, chunk 0 first (stable LSD
order), orders keys as the full multi-word key does."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2303_06890_gb300", "csrc")

SHIM = r"""
#include "qw_sort_chunks.h"
extern "C" int plan(const uint64_t *var, int nw, uint8_t *word, uint8_t *shift, uint8_t *len, int *nruns, int *npass)
{
    CkRuns c[16];
    const int nc = qw_sort_chunks(var, nw, c);
    for (int i = 0; i < nc; ++i) {
        for (int r = 0; r < c[i].n; ++r) {
            word[i * CK_MAXRUNS + r] = c[i].word[r];
            shift[i * CK_MAXRUNS + r] = c[i].shift[r];
            len[i * CK_MAXRUNS + r] = c[i].len[r];
        }
        nruns[i] = c[i].n;
        npass[i] = c[i].npass;
    }
    return nc;
}
"""


@pytest.fixture(scope="module")
def planner(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("sortplan")
    src = d / "shim.cpp"
    src.write_text(SHIM)
    so = d / "libplan.so"
    subprocess.run([cxx, "-std=c++17", "-O1", "-shared", "-fPIC", "-I", CSRC, str(src), "-o", str(so)], check=True)
    lib = ctypes.CDLL(str(so))
    lib.plan.restype = ctypes.c_int

    def run(var):
        var = np.ascontiguousarray(var, dtype=np.uint64)
        nw = len(var)
        word = np.zeros(16 * 64, np.uint8)
        shift = np.zeros(16 * 64, np.uint8)
        ln = np.zeros(16 * 64, np.uint8)
        nruns = np.zeros(16, np.int32)
        npass = np.zeros(16, np.int32)
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        nc = lib.plan(p(var), nw, p(word), p(shift), p(ln), p(nruns), p(npass))
        return [([(int(word[64 * c + r]), int(shift[64 * c + r]), int(ln[64 * c + r])) for r in range(nruns[c])],
                 int(npass[c])) for c in range(nc)]

    return run


def varying_positions(var):
    """Definition: the varying bits, as global positions 64 w + b, ascending."""
    return [64 * w + b for w, v in enumerate(var) for b in range(64) if (int(v) >> b) & 1]


def random_masks(rng, nw):
    out = []
    for w in range(nw):
        kind = rng.integers(0, 5)
        if kind == 0:
            out.append(0)
        elif kind == 1:
            out.append((1 << 64) - 1)
        elif kind == 2:  # one contiguous field
            lo = int(rng.integers(0, 64))
            hi = int(rng.integers(lo + 1, 65))
            out.append(((1 << hi) - 1) ^ ((1 << lo) - 1))
        else:  # scattered bits
            out.append(int(rng.integers(0, 1 << 63)) * 2 + int(rng.integers(0, 2)))
    return np.array(out, dtype=np.uint64)


@pytest.mark.parametrize("nw", [1, 2, 10])
def test_chunks_cover_the_varying_bits_in_order(planner, nw):
    rng = np.random.default_rng(nw)
    for _ in range(300):
        var = random_masks(rng, nw)
        chunks = planner(var)
        pos = varying_positions(var)
        assert len(chunks) == (len(pos) + 63) // 64
        got = []
        for c, (runs, npass) in enumerate(chunks):
            bits = []
            for w, s, n in runs:
                assert n >= 1 and s + n <= 64 and w < nw
                bits += [64 * w + s + t for t in range(n)]
            assert bits == pos[64 * c: 64 * c + 64]  # chunk c: the (64 c ..)-th varying bits
            assert npass == (len(bits) + 7) // 8
            got += bits
        assert got == pos


def test_no_varying_bit_gives_no_chunk(planner):
    assert planner(np.zeros(2, np.uint64)) == []
    assert planner(np.zeros(10, np.uint64)) == []


@pytest.mark.parametrize("nw", [2, 10])
def test_lsd_passes_over_the_chunks_sort_by_the_full_key(planner, nw):
    """Keys equal outside a random mask; stable 8-bit passes over the
    compacted keys, chunk after chunk, give the order of the full key (word
    nw - 1 most significant), ties by position."""
    rng = np.random.default_rng(100 + nw)
    for _ in range(20):
        mask = random_masks(rng, nw)
        base = [int(rng.integers(0, 1 << 63)) for _ in range(nw)]
        m = int(rng.integers(2, 400))
        keys = [[(base[w] & ~int(mask[w])) | (int(rng.integers(0, 1 << 63)) * 2 + int(rng.integers(0, 2))) & int(mask[w])
                 for w in range(nw)] for _ in range(m)]
        keys += keys[: m // 4]  # equal keys: the sort must keep their order
        orv = [0] * nw
        andv = [(1 << 64) - 1] * nw
        for k in keys:
            for w in range(nw):
                orv[w] |= k[w]
                andv[w] &= k[w]
        var = np.array([o ^ a for o, a in zip(orv, andv)], dtype=np.uint64)
        perm = list(range(len(keys)))
        for runs, npass in planner(var):
            ck = []
            for i in perm:
                c, dst = 0, 0
                for w, s, n in runs:
                    c |= ((keys[i][w] >> s) & ((1 << n) - 1)) << dst
                    dst += n
                ck.append(c)
            for p in range(npass):
                order = sorted(range(len(perm)), key=lambda q: (ck[q] >> (8 * p)) & 255)
                perm = [perm[q] for q in order]
                ck = [ck[q] for q in order]
        want = sorted(range(len(keys)), key=lambda i: tuple(reversed(keys[i])))
        assert perm == want
