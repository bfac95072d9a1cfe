/*
 * qw_internal.h -- device data layout shared by the kernels (qw_kernels.cu)
 * and the host side of the C ABI (qw_api.cpp).
 *
 * Layout in HBM.  The state is bucketed by row: one bucket per (inst, jc, j, b1)
 * value, i.e. per value of the registers that T~, P and T~^dag never change
 * and that every QRAM access of those operators indexes (row j).  A bucket
 * holds up to cap_row branches as
 *   key[b * cap_row + i]  uint64, the "local" registers (k, kc, A, b2) packed
 *                         in the R layout below,
 *   amp[b * cap_row + i]  double2 or float2,
 *   count[b]              int32 branches present.
 * Rows with jc = 0 have dense buckets: inst_bkt[inst] + (j << 1 | b1).  Rows
 * with jc != 0 (garbage subspace) go to spill buckets dense_buckets + slot,
 * slot found by open addressing on the packed row key in spill[].
 * Three such buffers rotate: a step reads X_t, writes X_{t+1} and clears
 * X_{t+2}; X_t stays intact until the step after next.
 *
 * Local-key layouts (bit 0 first):
 *   R layout: b2 | k (nb) | kc (nb) | A (16)            -- b2-pairs adjacent
 *   H layout: k_low (L) | b2 | k_high (nb-L) | kc | A   -- Hadamard groups adjacent
 * Both keep kc and A at bits 1+nb and above.
 */
#ifndef QW_INTERNAL_H
#define QW_INTERNAL_H

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/qwalk.h"

#define QW_SPILL_EMPTY (~0ull)

/* device status word bits */
#define QW_ST_ROW_OVERFLOW 1   /* a bucket received more than cap_row branches */
#define QW_ST_WARP_OVERFLOW 2  /* a row outgrew the on-chip row buffer */
#define QW_ST_SPILL_FULL 4     /* no free spill slot for a jc != 0 row */
#define QW_ST_ANCILLA 8        /* register A not zero where it must be */
#define QW_ST_NOT_BTILDE 16    /* T~ at initialisation met a row that was not |b~> */
#define QW_ST_OUTBOX_FULL 32   /* a partition's outbox toward another overflowed */
#define QW_ST_POS_UNREP 64     /* a branch the positional layout has no position for */
#define QW_ST_SORT_WAIT 128    /* the flat path's radix sort gave up waiting for a tile's count */

/* A branch sent by S to a row another partition owns: its row key
   (qw_rowkey), its local registers (R layout) and its amplitude in FP64. */
struct QwPartEntry {
    uint64_t rowkey, local;
    double re, im;
};

/* per-step branch counters (index into QwStepArgs.stats) */
#define QW_STAT_ROWS 0      /* rows processed */
#define QW_STAT_IN 1        /* branches entering the step (input of R^dag) */
#define QW_STAT_RDAG 2      /* after R^dag (input of the H P H stage) */
#define QW_STAT_H1 3        /* after the first H (literal mode only) */
#define QW_STAT_HPH 4       /* after H P H (input of R) */
#define QW_STAT_OUT 5       /* after R (branches written) */
#define QW_STAT_STEPS 6     /* clean steps counted */
#define QW_NSTAT 8

/* step kernel modes */
#define QW_MODE_WALK_FUSED 0   /* T~^dag, (H P H as one reflection), T~, S */
#define QW_MODE_WALK_LITERAL 1 /* T~^dag, H, P, H, T~, S */
#define QW_MODE_T 2            /* T~ only, in place on a bucket range */
#define QW_MODE_WALK_FUSED_PF 3 /* fused step, row loop software-pipelined */
#define QW_MODE_WALK_SEG 4      /* fused step, both rows of a j as one segment */
#define QW_MODE_WALK_SEG_PF 5   /* segments, software-pipelined */
#define QW_MODE_WALK_SLOT 6     /* fused step, one lane per QRAM slot (s = 8, 16, 32) */
#define QW_MODE_WALK_FLAT 7     /* the literal step on one globally sorted branch list (qw_flat.cu) */
#define QW_MODE_WALK_FAITHFUL 8 /* the flat step with every working register in a 10-word key */
#define QW_MODE_WALK_POS 9      /* the state held by position, one lane per QRAM slot (s = 8, 16, 32) */

struct QwSimDev {
    int nb, s, L, ninst;
    int n_single;  /* N of the instance when ninst == 1 (tables not read then) */
    int cap_row;   /* branches per bucket */
    int warp_cap;  /* on-chip branches per warp */
    int spill_slots;          /* power of two */
    int64_t dense_buckets;    /* sum over instances */
    int64_t total_buckets;    /* dense + spill */
    double tau2;              /* prune threshold squared */
    uint64_t tau_hi_bits;     /* bits of tau (1 + 2^-30): |x| above it => kept */
    uint64_t tau_lo_bits;     /* bits of tau sqrt(1/2) (1 - 2^-30): |x|,|y| at most it => pruned */
    float tau2f;              /* tau^2 as float (complex64 path) */
    int rot_calc;             /* rot_bits == 0: the FP32 rotation pairs follow from the code alone */
    double inv_sqrt_s;        /* 1 / sqrt(s) */
    double two_over_s;        /* 2 / s */
    const uint32_t *img;      /* QRAM words: column << 16 | Q1.15 value */
    const double2 *fg;        /* per Q1.15 code: (sqrt|a|, sqrt(1-|a|)) */
    const float4 *fg32;       /* the same as float pairs: (hi, lo) of each, hi + lo ~ 48 bits */
    const void *slot_rot;     /* per QRAM slot: its code's entry of fg (FP64) or fg32 (FP32) */
    const int32_t *inst_n;    /* N per instance */
    const int64_t *inst_img;  /* image offset per instance */
    const int64_t *inst_bkt;  /* first dense bucket per instance, ninst + 1 entries */
    const uint16_t *unit_inst; /* instance of dense bucket pair u (buckets 2u, 2u + 1); ninst > 1 */
    /* row-partitioned walk (single instance): rows (jc = 0, j < N) in blocks of
       part_rows per partition, the others by a hash of (jc, j); S sends a
       branch whose new row another partition owns to that partition's
       outbox segment (outbox_cap entries each) */
    int nparts, part;
    int64_t part_rows;
    QwPartEntry *outbox;
    unsigned long long *outbox_count;
    int64_t outbox_cap;
    /* positional layout: the rows j < N of all instances in order, row g
       (instance i, g = inst_img[i] / s + j) of pos_rows; row (g, b1) is
       pos_R = 2 s + 2 pos_E amplitudes at (2 g + b1) pos_R.  pos_tp[g s + l]:
       the position of the branch k = j in row col(j, l) of the instance;
       pos_xin[g pos_E + e] = x << 8 | l for the e-th row x (global) < pos_xcnt[g]
       whose slot l holds column j while row j holds no column x;
       pos_rowbase[g] / pos_rowinst[g]: the first row and the instance of
       row g's instance (null with one instance) */
    int pos_R, pos_E;
    int64_t pos_rows;
    const uint16_t *pos_tp;
    const uint32_t *pos_xin;
    const uint16_t *pos_xcnt;
    const uint32_t *pos_rowbase;
    const uint16_t *pos_rowinst;
};

struct QwBufDev {
    uint64_t *key;
    void *amp;
    int32_t *count;
    uint64_t *spill;
};

struct QwStepArgs {
    int mode;
    int renorm;
    int64_t bucket_lo, bucket_hi; /* bucket range processed (MODE_T) */
    const double *scale_in;  /* amplitude scale of the input (renormalisation), nullable */
    double *partials;        /* per-block norm partial sums */
    unsigned int *done_ctr;  /* blocks finished (last block reduces partials) */
    double *norm_out;        /* ||output||^2 */
    double *scale_out;       /* sqrt(target / norm_out) when renorm, else 1 */
    const double *renorm_target; /* sum of the instances' initial ||b||^2 */
    int64_t *steps_done;     /* incremented by each step that completes cleanly */
    int32_t *status;
    unsigned long long *stats; /* QW_STAT_* counters, accumulated (nullable) */
    double2 *qls_y;          /* flag-0 accumulator (nullable) */
    const double *qls_coefs; /* Y += qls_coefs[*qls_j] * Pi_0 tau at this step's midpoint */
    const int64_t *qls_j;    /* index of the current QLS term (advanced by k_qls_norm) */
    int qls_readout;
    int32_t *deferred;          /* slot kernel: units left to the row pipeline (dense unit u,
                                   or 0x80000000 | garbage-row slot), run by the last block */
    unsigned int *deferred_ctr; /* entries in deferred (reset by the last block) */
    unsigned int *work_ctr;     /* slot kernel: groups claimed beyond each warp's first
                                   (reset by the last block) */
};

/* launchers (qw_kernels.cu); all return cudaGetLastError() of the launch */
int qw_sm_count(void);
cudaError_t qw_launch_step(const QwSimDev &d, const QwBufDev &in, const QwBufDev &out,
                           const QwBufDev &clear, const QwStepArgs &a, int fp32, int grid,
                           cudaStream_t st);
/* whether the slot kernel (QW_MODE_WALK_SLOT) covers this sparsity */
int qw_slot_supported(const QwSimDev &d);
/* whether the positional layout (QW_MODE_WALK_POS) covers this s (8 .. 64) */
int qw_pos_supported(const QwSimDev &d);
/* dynamic shared memory per block of the step kernel of `mode` */
size_t qw_step_smem_bytes(const QwSimDev &d, int fp32, int mode);
/* positional layout: one walk step pin -> pout (both pos_R-strided row
   arrays), the grid of its launch, and the conversions from and to the row
   buckets (pack: pout zeroed by the caller; a branch without a position sets
   QW_ST_POS_UNREP; unpack: the buckets cleared by the caller) */
cudaError_t qw_launch_walk_pos(const QwSimDev &d, const void *pin, void *pout, const QwStepArgs &a, int fp32,
                               int grid, cudaStream_t st);
int qw_pos_grid(const QwSimDev &d, int fp32);
cudaError_t qw_launch_pos_pack(const QwSimDev &d, const QwBufDev &buf, void *pbuf, int fp32, int32_t *status,
                               cudaStream_t st);
cudaError_t qw_launch_pos_unpack(const QwSimDev &d, const void *pbuf, const QwBufDev &buf, int fp32,
                                 int32_t *status, cudaStream_t st);
/* T~|b~> written straight into rows g0 .. g0 + n of the positional layout
   (the rest of those rows zeroed); a register marginal read straight from
   those rows (probs zeroed by the caller, accumulated by atomics) */
cudaError_t qw_launch_tinit_pos(const QwSimDev &d, void *pbuf, int64_t g0, int64_t n, const double *b_re,
                                const double *b_im, const double *scale, int fp32, cudaStream_t st);
cudaError_t qw_launch_measure_pos(const QwSimDev &d, const void *pbuf, int64_t g0, int64_t n, int fp32,
                                  const double *scale, int reg, double *probs, int64_t len, cudaStream_t st);
int qw_step_grid(const QwSimDev &d, int fp32, int mode);
cudaError_t qw_launch_clear(const QwSimDev &d, const QwBufDev &buf, int64_t lo, int64_t hi,
                            int clear_spill, cudaStream_t st);
cudaError_t qw_launch_init_b(const QwSimDev &d, const QwBufDev &buf, int inst, const double *b_re,
                             const double *b_im, int n, int fp32, const double *scale, cudaStream_t st);
cudaError_t qw_launch_tinit(const QwSimDev &d, const QwBufDev &buf, int64_t lo, int64_t hi, int fp32,
                            int32_t *status, cudaStream_t st);
cudaError_t qw_launch_import(const QwSimDev &d, const QwBufDev &buf, const uint64_t *rowkey,
                             const uint64_t *local, const double2 *amp, int64_t count, int fp32,
                             int32_t *status, cudaStream_t st);
cudaError_t qw_launch_export(const QwSimDev &d, const QwBufDev &buf, int inst, int fp32,
                             const double *scale, uint64_t *rowkey, uint64_t *local, double2 *amp,
                             unsigned long long *counter, int64_t cap, cudaStream_t st);
cudaError_t qw_launch_measure(const QwSimDev &d, const QwBufDev &buf, int inst, int fp32,
                              const double *scale, int reg, double *probs, int64_t len,
                              cudaStream_t st);
/* pbuf (nullable): read rows g0 .. g0 + pn of the positional layout instead of buf */
cudaError_t qw_launch_measure_noalloc(const QwSimDev &d, const QwBufDev &buf, int inst, int fp32,
                                      const double *scale, int reg, double *host_probs,
                                      int64_t len, int device, cudaStream_t st, const void *pbuf = nullptr,
                                      int64_t g0 = 0, int64_t pn = 0);
cudaError_t qw_launch_count(const QwSimDev &d, const QwBufDev &buf, int inst,
                            unsigned long long *counter, cudaStream_t st);
cudaError_t qw_launch_qls_norm(const double2 *y, int n, double *p, int64_t *jctr, cudaStream_t st);
/* copy buffer `from` (row capacity cap_old) into new key/amp arrays laid out
   with d.cap_row entries per bucket */
cudaError_t qw_launch_regrow(const QwSimDev &d, const QwBufDev &from, int cap_old, uint64_t *key_new, void *amp_new,
                             int fp32, cudaStream_t st);

/* flat, globally sorted step (qw_flat.cu): keys are packed register keys of
   kw 64-bit words (2: the qw_state_export layout; 10: the register-faithful
   layout with the working registers above bit 128), amplitudes complex FP64;
   see qw_flat.cu for each stage */
#define QW_FLAT_OSDAG 1u
#define QW_FLAT_OA 2u
#define QW_FLAT_OS 3u
#define QW_FLAT_S 4u
#define QW_FLAT_A0 5u /* check A = 0 */
#define QW_FAITH_WORDS 10
cudaError_t qw_flat_gather(const QwSimDev &d, const QwBufDev &buf, int fp32, const double *scale, void *keys,
                           double2 *amps, unsigned long long *counter, int64_t cap, cudaStream_t st, int kw);
cudaError_t qw_flat_map(const QwSimDev &d, void *keys, int64_t M, uint32_t ops, int32_t *status, cudaStream_t st,
                        int kw);
cudaError_t qw_flat_phase(const QwSimDev &d, const void *keys, double2 *amps, int64_t M, cudaStream_t st, int kw);
size_t qw_flat_scan_words(int64_t n);
cudaError_t qw_flat_scan(const uint32_t *in, int64_t n, uint32_t *sums, uint32_t *out, cudaStream_t st);
/* stable sort by the permuted key (order 0: R, 1: H); work holds
   qw_flat_sort_bytes(M); the result is left in tmpk / tmpa when *in_tmp */
size_t qw_flat_sort_bytes(int64_t M);
cudaError_t qw_flat_sort(const QwSimDev &d, void *keys, double2 *amps, void *tmpk, double2 *tmpa, int64_t M,
                         int order, void *work, int32_t *status, cudaStream_t st, int kw, int *in_tmp);
/* the Hadamard stage's groups: head flags of the sorted list, and the first
   member of each of its G groups (starts[G] = M) from their exclusive scan */
cudaError_t qw_flat_heads(const QwSimDev &d, const void *keys, int64_t M, uint32_t *flags, cudaStream_t st, int kw);
cudaError_t qw_flat_starts(const uint32_t *heads, const uint32_t *gidx, int64_t M, int64_t G, int64_t *starts,
                           cudaStream_t st);
/* op 0 (R^dag) and 1 (R): 2 M outputs with their keep flags */
cudaError_t qw_flat_group(const QwSimDev &d, int op, const void *keys, const double2 *amps, int64_t M, void *okeys,
                          double2 *oamps, uint32_t *flags, cudaStream_t st, int kw);
/* H on the G groups (starts): gpos == nullptr -- the kept outputs of each
   group into cnt; otherwise the kept outputs written from gpos[g] on */
cudaError_t qw_flat_hgroups(const QwSimDev &d, const void *keys, const double2 *amps, const int64_t *starts, int64_t G,
                            uint32_t *cnt, const uint32_t *gpos, void *okeys, double2 *oamps, cudaStream_t st, int kw);
cudaError_t qw_flat_compact(const void *keys, const double2 *amps, const uint32_t *flags, const uint32_t *pos,
                            int64_t n, void *okeys, double2 *oamps, cudaStream_t st, int kw);
cudaError_t qw_flat_readout(const QwSimDev &d, const void *keys, const double2 *amps, int64_t M, const QwStepArgs &a,
                            cudaStream_t st, int kw);
cudaError_t qw_flat_scatter(const QwSimDev &d, const QwBufDev &out, int fp32, const void *keys, const double2 *amps,
                            int64_t M, int32_t *status, unsigned int *maxrow, double *norm, cudaStream_t st, int kw);
cudaError_t qw_flat_finish(const QwStepArgs &a, const double *norm, const int64_t *counts, cudaStream_t st);
/* register-faithful sub-operations on 10-word keys (op codes QW_FQ_* of qwalk.h) */
int qw_faithful_layout(const QwSimDev &d, int *addr_bits, int *layout_bits);
cudaError_t qw_faithful_op(const QwSimDev &d, void *keys, int64_t M, int op, int32_t *status, cudaStream_t st);
cudaError_t qw_faithful_check_idle(const QwSimDev &d, const void *keys, int64_t M, int32_t *status, cudaStream_t st);
cudaError_t qw_faithful_export(const QwSimDev &d, const void *keys, int64_t M, uint64_t *table, cudaStream_t st);
/* the other partitions' outbox segments toward this one (entries and device
   counts, cap entries each) and the norm slots of all parts' last step */
struct QwPartSources {
    const QwPartEntry *e[64];
    const unsigned long long *count[64];
    int n;
    int64_t cap;
};
struct QwPartNorms {
    const double *norm[64];
    int n;
};
cudaError_t qw_launch_part_gather(const QwSimDev &d, const QwBufDev &buf, const QwPartSources &src, int fp32,
                                  int32_t *status, cudaStream_t st);
cudaError_t qw_launch_part_scale(const QwPartNorms &nm, const double *target, double *scale_out, int renorm,
                                 cudaStream_t st);
cudaError_t qw_launch_part_inbox(const QwSimDev &d, const QwBufDev &buf, const QwPartEntry *e, int64_t count, int fp32,
                                 int32_t *status, cudaStream_t st);

/* Partition owning row (jc, j) of a row-partitioned walk: blocks of
 * part_rows rows for jc = 0, j < N; a hash of (jc, j) otherwise (the rows
 * only states outside the walk's subspace reach). */
__host__ __device__ static inline int qw_part_owner_of(const QwSimDev &d, uint32_t jc, uint32_t j)
{
    if (jc == 0 && j < (uint32_t)d.n_single) return (int)((int64_t)j / d.part_rows);
    uint64_t x = ((uint64_t)jc << 20) | (uint64_t)j;
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    return (int)(x % (uint64_t)d.nparts);
}

/* packed row key: inst << 40 | jc << 20 | j << 1 | b1  (nb <= 19) */
__host__ __device__ static inline uint64_t qw_rowkey(uint32_t inst, uint32_t jc, uint32_t j,
                                                     uint32_t b1)
{
    return ((uint64_t)inst << 40) | ((uint64_t)jc << 20) | ((uint64_t)j << 1) | (uint64_t)b1;
}

#endif /* QW_INTERNAL_H */
