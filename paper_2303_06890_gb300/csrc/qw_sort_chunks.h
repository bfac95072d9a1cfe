/*
 * qw_sort_chunks.h -- host-side plan of the flat path's radix sort: which key
 * bits the passes sort by.  Plain C++ (no CUDA), shared by qw_flat.cu and
 * the host-logic test.
 *
 * The sort runs on a compacted key: the bits that vary between the keys of
 * the list (OR ^ AND over all keys, word by word), taken in order of
 * significance of the permuted key, 64 at a time (a "chunk").  Chunk c's bit
 * b is the (64 c + b)-th varying bit; a chunk is held as runs of adjacent
 * varying bits (key word, first bit, length), lowest first, and sorted by
 * ceil(bits / 8) passes of 8-bit digits.
 */
#pragma once
#include <stdint.h>

constexpr int CK_MAXRUNS = 64, CK_MAXPASS = 8;

struct CkRuns {
    uint8_t word[CK_MAXRUNS], shift[CK_MAXRUNS], len[CK_MAXRUNS];
    int n, npass;
};

/* The chunks of the varying bits var[0 .. nw - 1] (word 0 least
 * significant) into out[0 ..]; returns their number (0 when no bit varies:
 * the keys are all equal).  out must hold nw chunks. */
inline int qw_sort_chunks(const uint64_t *var, int nw, CkRuns *out)
{
    int nc = 0, cbits = 0;
    CkRuns cur{};
    for (int wi = 0; wi < nw; ++wi) {
        const uint64_t v = var[wi];
        int b = 0;
        while (b < 64) {
            if (!((v >> b) & 1ull)) {
                ++b;
                continue;
            }
            int e = b;
            while (e < 64 && ((v >> e) & 1ull) && cbits + (e - b) < 64) ++e;
            cur.word[cur.n] = (uint8_t)wi;
            cur.shift[cur.n] = (uint8_t)b;
            cur.len[cur.n] = (uint8_t)(e - b);
            ++cur.n;
            cbits += e - b;
            if (cbits == 64) { /* the chunk is full */
                cur.npass = CK_MAXPASS;
                out[nc++] = cur;
                cur = CkRuns{};
                cbits = 0;
            }
            b = e;
        }
    }
    if (cbits > 0) {
        cur.npass = (cbits + 7) / 8;
        out[nc++] = cur;
    }
    return nc;
}
