/*
 * qwalk.h -- C ABI of the GB300 sparse-state quantum-walk simulator.
 *
 * The library simulates, on one GPU, the quantum walk on a sparse real
 * symmetric matrix stored in QRAM in compressed-sparse-column form and the
 * CKS quantum linear solver built on it (arXiv 2303.06890, Secs. II-V).  The
 * quantum state is a list of branches: one packed register key and one complex
 * amplitude each (Sec. V-A, "Main idea").
 *
 * Registers (Sec. IV, "Implementation of the quantum walk"): jc, j, b1, kc, k,
 * b2 of widths nb, nb, 1, nb, nb, 1 with nb = ceil(log2 N) (the largest N of
 * the simulation), plus the 16-bit element register A that is live only
 * inside T~ and T~^dag.
 *
 * Conventions for every function:
 *   - the return value is QW_OK (0) or a negative QW_ERR_* code; nothing
 *     throws across the ABI; qw_last_error() gives a message for the last
 *     failure on that simulator;
 *   - host arrays belong to the caller and are copied during the call (the
 *     copy may be asynchronous from pinned memory; the call still returns
 *     only when it no longer reads them);
 *     device memory belongs to the simulator and is freed by qw_sim_destroy;
 *   - work is issued in order on the stream given at creation; functions that
 *     return data to host arrays synchronise that stream before returning.
 */
#ifndef QWALK_H
#define QWALK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QW_OK 0
#define QW_ERR_ARG (-1)           /* bad argument (null pointer, size, index) */
#define QW_ERR_CSC (-2)           /* matrix rejected, see qw_sim_create */
#define QW_ERR_CAPACITY (-3)      /* a row or the on-chip row buffer overflowed */
#define QW_ERR_CUDA (-4)          /* a CUDA runtime call failed */
#define QW_ERR_DEVICE_STATUS (-5) /* a device-side self-check tripped */
#define QW_ERR_STATE (-6)         /* call out of order (e.g. no state yet) */

#define QW_FP64 0     /* complex128 amplitudes, FP64 arithmetic */
#define QW_FP32_AMP 1 /* complex64 amplitudes in memory; rotations and the reflection
                         sum from error-free FP32 products and sums (~48-bit float
                         pairs); each thread's share of the norm as a float pair,
                         its reductions, the renormalisation factor, the QLS
                         read-out and the success probability in FP64 */

/* Register ids for qw_measure_register. */
#define QW_REG_JC 0
#define QW_REG_J 1
#define QW_REG_B1 2
#define QW_REG_KC 3
#define QW_REG_K 4
#define QW_REG_B2 5

typedef struct qw_sim qw_sim; /* opaque; owns all device memory */

/*
 * One real symmetric matrix in CSC form (Sec. II-C).  Column c holds its
 * non-zero rows rowidx[colptr[c] .. colptr[c+1]) in strictly increasing order
 * with values val_q15[...] in Q1.15 two's complement (value = q / 32768).
 * By symmetry column j is also row j, which is what the QRAM stores.
 * s_pad: padded sparsity s, a power of two >= the largest column count and
 * <= n; 0 selects the smallest such power of two (Table 1, note b).
 */
typedef struct {
    int32_t n;
    int32_t nnz;
    const int32_t *colptr;  /* n + 1 entries, colptr[0] = 0, colptr[n] = nnz */
    const int32_t *rowidx;  /* nnz entries */
    const int16_t *val_q15; /* nnz entries */
    int32_t s_pad;
} qw_csc;

typedef struct {
    int32_t precision;       /* QW_FP64 (default) or QW_FP32_AMP */
    int32_t fuse_reflection; /* 1 (default): H P H of one walk step as the per-group
                                reflection 2|+><+| - 1; 0: H, P, H as three ops */
    double prune_tau;        /* branches with |a| <= tau are removed after each
                                interference op; 0 = 1e-13 (FP64), 2^-24 (FP32_AMP) */
    int32_t row_capacity;    /* branches per (jc, j, b1) row between steps; 0 = auto (4 s) */
    int32_t warp_capacity;   /* entries of a warp's on-chip buffers while it runs a row
                                (or a segment of two rows) through a step: branches at
                                load and after T~, b2-pairs between T~^dag and T~; 0 = auto:
                                2 row_capacity rounded up to a power of two, at least 64
                                (fuse_reflection = 1), halved while the buffers do not
                                fit the device's shared memory per block */
    int32_t renorm;          /* -1 = default (on for FP32_AMP, off for FP64) */
    void *stream;            /* cudaStream_t to issue on; NULL = the default stream */
    int32_t walk_variant;    /* step kernel with fuse_reflection = 1 (see qw_autotune):
                                0 = one row at a time (default), 1 = rows with a
                                software-pipelined loop, 2 = the two rows of a j as one
                                segment, 3 = segments, software-pipelined, 4 = one lane
                                per QRAM slot over groups of 32 / s consecutive j
                                (s = 8, 16 or 32 and warp_capacity >= 2 row_capacity;
                                what its lanes do not cover runs as in 2), 5 = the flat
                                path: the paper's literal schedule on one list of all
                                branches in device memory, each interference op a
                                global radix sort by key, a per-group transform and a
                                compaction (no capacity limit; the host synchronises
                                between its stages, so no CUDA graph is used; its
                                scratch comes from a device memory pool of the
                                simulator's own, which keeps the memory once used
                                until qw_sim_destroy), 6 = the
                                register-faithful schedule: the flat path with every
                                working register of O_s', O_A' and Alg. 1 held in the
                                state between sub-operations (the QW_FQ_STEP sequence
                                below; any fuse_reflection), 7 = the positional layout:
                                s = 8, 16, 32 or 64, any number of instances; every
                                branch the walk reaches from T~|b~> is held at a fixed
                                position of its row (no key, no count), one lane per
                                QRAM slot (two for s = 64) writes each output to its
                                position, so a step has no search, atomic or clearing;
                                a state with branches outside those positions (e.g.
                                from qw_state_import) runs on the kernel of variant 4
                                (2 for s = 64).  qw_state_init with apply_T = 1 writes
                                T~|b~> straight into the layout and the register
                                marginals read it in place; any other state moves into
                                it at the first walk step (a synchronisation), and it
                                moves back into the row buckets before qw_state_size,
                                qw_state_export, qw_state_import or a register-faithful
                                session; row_capacity grows to 2 s + 2 E (E: the most
                                unpaired padded columns pointing at one row) */
    int32_t graphs;          /* 1 (default): runs of >= 6 walk steps are issued as replays
                                of a captured 6-step CUDA graph; 0: one launch per step */
    int32_t spill_rows;      /* slots of the table holding rows with jc != 0 (reached only
                                from states outside the walk's physical subspace, e.g. by
                                qw_state_import); a power of two, 0 = auto (2N/8 over all
                                instances, clamped to [256, 4096]) */
    int32_t rot_bits;        /* 0 (default): the rotation's f = sqrt(|a|), g = sqrt(1 - |a|)
                                in FP64; 1..52: the angle theta = arccos(sqrt(|a|)) held
                                in a fixed-point register of rot_bits bits over [0, pi/2]
                                (rounded half to even), f = cos, g = sin of it -- the
                                square-root and arccos registers Table 2 lists for the
                                conditional rotation */
    int32_t overflow_fallback; /* 1 (default): a walk step whose rows outgrow row_capacity
                                or the on-chip buffers is run again from its input on the
                                flat path (walk_variant 5), and row_capacity grows to the
                                largest row it produces (the row buckets are reallocated);
                                qw_state_import grows it the same way.  0: such a step
                                fails with QW_ERR_CAPACITY and the state is kept at the
                                last completed step */
    int32_t nparts;          /* row-partitioned walk: the rows are split among nparts
                                simulators (1, the default: one simulator holds all) */
    int32_t part;            /* this simulator's partition, 0 .. nparts - 1 */
    int64_t outbox_capacity; /* branches each outbox segment (one per other partition)
                                holds; 0 = auto (2 N s) */
} qw_sim_opts;

/* Fill *opts with the defaults above. */
void qw_sim_opts_default(qw_sim_opts *opts);

/*
 * Create a simulator for num_instances independent walks, instance i on
 * matrix mats[i] (batched form: every instance is advanced by each call of
 * qw_apply_walk_step).  All instances must have the same padded sparsity s.
 * The matrices are validated and copied to device memory as the padded QRAM
 * image of Fig. 1: per row j, s (column, value) slots at j*s..j*s+s-1, sorted
 * by column; a row with fewer than s non-zeros is completed with explicit
 * zero elements at the first columns j+1, j+2, ... (cyclically) not already in
 * the row.
 * Errors: QW_ERR_ARG (null, num_instances < 1, n < 2, n > 65536, or row
 * buffers -- 8 warps x 2 x warp_capacity branches -- larger than the
 * device's shared memory per block);
 * QW_ERR_CSC (unsorted or duplicate rows in a column, index out of range,
 * column count > s_pad, s_pad not a power of two or > n, matrix not
 * symmetric, negative diagonal element -- which the walk's isometry cannot
 * encode, Eq. psi_j -- or instances with different s); QW_ERR_CUDA.
 * On success *out owns the simulator; on failure *out is NULL.
 */
int qw_sim_create(const qw_csc *mats, int32_t num_instances, const qw_sim_opts *opts,
                  qw_sim **out);

/*
 * Set instance inst to |b~> = sum_j b_j |jc=0, j, b1=0, kc=0, k=0, b2=0>
 * (Sec. IV, |j~>), b = b_re + i b_im (b_im may be NULL), n = that instance's N;
 * exact zeros are not stored.  With apply_T != 0 the state becomes T~|b~>
 * (Alg. T~).  Other instances are not touched.  b_re and b_im are copied to
 * the device directly (an asynchronous copy when they are pinned); the call
 * synchronises the simulator's stream before it returns, so they may be
 * reused afterwards.
 * Errors: QW_ERR_ARG, QW_ERR_CAPACITY, QW_ERR_CUDA, QW_ERR_DEVICE_STATUS (T~
 * met a row of the instance that was not |b~>).
 */
int qw_state_init(qw_sim *sim, int32_t inst, const double *b_re, const double *b_im, int32_t n,
                  int32_t apply_T);

/*
 * Apply nsteps walk steps W = S T~ P T~^dag (Alg. "Quantum walk operator")
 * to every instance.  Each step is one launch over all rows; no host
 * synchronisation happens between steps.  The call synchronises once at the
 * end to read the device status word.  With overflow_fallback, steps that
 * outgrew the row buckets or the on-chip buffers are run again on the flat
 * path (then the call synchronises between those steps).
 * Errors: QW_ERR_STATE (no state), QW_ERR_CAPACITY (without overflow_fallback,
 * or when the grown buckets would not fit in device memory; state kept at the
 * last completed step), QW_ERR_DEVICE_STATUS, QW_ERR_CUDA.
 */
int qw_apply_walk_step(qw_sim *sim, int64_t nsteps);

/*
 * Issue nsteps walk steps on the simulator's stream and return without
 * synchronising (for pipelining, timing and stream capture).  Device errors
 * of these steps are reported by the next call that synchronises (qw_sync,
 * qw_apply_walk_step, the measurement and export calls).  Exception: with
 * walk_variant 7, a call made while the stream is not being captured first
 * moves a state that is not yet in the positional layout into it, which
 * synchronises once; during a capture such a state runs on the bucket
 * kernel of variant 4 (2 for s = 64) instead.  The flat and register-faithful schedules (variants 5
 * and 6) synchronise between their stages.
 * Errors: QW_ERR_ARG, QW_ERR_STATE, QW_ERR_CUDA (launch failure).
 */
int qw_enqueue_walk_steps(qw_sim *sim, int64_t nsteps);

/*
 * Synchronise the stream and read the device status word.  On a device
 * error the state is the output of the last step that completed cleanly
 * (later steps did nothing) and the error code is returned:
 * QW_ERR_CAPACITY, QW_ERR_DEVICE_STATUS or QW_ERR_CUDA.  With
 * overflow_fallback, steps enqueued since the last synchronising call that
 * outgrew the buckets are first run again on the flat path.
 */
int qw_sync(qw_sim *sim);

/* Number of step-kernel variants (walk_variant 0 .. QW_WALK_VARIANTS - 1). */
#define QW_WALK_VARIANTS 8

/*
 * Autotuner of the fused step kernel: runs steps_per_candidate walk steps with
 * each variant of walk_variant (rows or segments of two rows, plain or
 * software-pipelined, one lane per QRAM slot, the positional layout), times
 * them with CUDA events on the simulator's stream, and keeps the fastest for
 * all later steps.  Segments are tried only when warp_capacity >= 2
 * row_capacity (true by default), the slot kernel only then and for s = 8, 16
 * or 32, the positional layout (variant 7) for s = 8, 16, 32 or 64 without
 * partitions (its tables are built first, and the move of the state into it
 * is not timed); the flat path and the register-faithful
 * schedule (variants 5 and 6) are never chosen; variants not tried are
 * reported as 0 us.  The state advances by steps_per_candidate walk steps per
 * variant tried (the variants give the same results).  *choice (nullable)
 * receives the variant, *us_per_step (nullable, QW_WALK_VARIANTS doubles) the
 * measured times.  Synchronises.  Has no effect with fuse_reflection = 0.
 * Errors: QW_ERR_ARG, QW_ERR_STATE, QW_ERR_CAPACITY, QW_ERR_CUDA.
 */
int qw_autotune(qw_sim *sim, int32_t steps_per_candidate, int32_t *choice, double *us_per_step);

/*
 * CKS coefficients of Eq. (fx): b = ceil(kappa^2 ln(kappa/eps)),
 * j0 = ceil(sqrt(b ln(4 b / eps))), a_j = 4 (-1)^j sum_{i=j+1}^{b} C(2b, b+i) / 2^(2b)
 * for j = 0..j0, computed in log space.  Writes min(j0+1, cap) coefficients;
 * *j0_out and *b_out (nullable) receive j0 and b.
 * Errors: QW_ERR_ARG (kappa < 1, eps not in (0, 1), coeffs NULL with cap > 0).
 */
int qw_cks_coefficients(double kappa, double eps, double *coeffs, int64_t cap, int64_t *j0_out,
                        int64_t *b_out);

/*
 * CKS linear solver (Sec. IV, Eq. (fx); Sec. V-B).  Requires instance inst in
 * state T~|b~> (qw_state_init with apply_T = 1) and a single-instance
 * simulator.  Runs walk steps and, at every other step, reads the flag-0 block
 * of tau_j = T~^dag W^(2j+1) T~ |b~> (whose value is T_{2j+1}(A/s) b) in FP64:
 * Y += coeffs[j] * Pi_0 tau_j for j = 0..j0.  Outputs: y_out (2 N doubles,
 * interleaved re/im) = Y; psucc_out (j0+1 doubles, nullable) =
 * || Pi_0 sum_{k<=j} coeffs[k] tau_k ||^2 for each j.  Three launches per
 * term (two walk steps, one norm); with opts.graphs, runs of 3 terms replay a
 * captured CUDA graph (the coefficient index lives on the device).
 * Errors: QW_ERR_ARG, QW_ERR_STATE, QW_ERR_CAPACITY, QW_ERR_CUDA.
 */
int qw_apply_qls(qw_sim *sim, int32_t inst, const double *coeffs, int64_t j0, double *y_out,
                 double *psucc_out);

/*
 * Marginal distribution of one register of instance inst (the read-out of
 * Sec. V-B: the success probability p_j of the post-selection is the weight
 * of the flag registers' zero value, a marginal of the state):
 * probs[v] = sum over branches with register value v of |a|^2, v < len.
 * reg_id is one of QW_REG_*.  The histogram is accumulated in a device
 * scratch array that the simulator keeps for later calls; the call allocates
 * it with cudaMalloc when len exceeds every earlier len of this simulator.
 * The result is copied straight into probs (asynchronous when probs is
 * pinned); the call synchronises before it returns.
 * Errors: QW_ERR_ARG, QW_ERR_STATE, QW_ERR_CUDA.
 */
int qw_measure_register(qw_sim *sim, int32_t inst, int32_t reg_id, double *probs, int64_t len);

/*
 * Largest len accepted by qw_measure_register_noalloc: 65536 bins, enough for
 * any register of a simulator (N <= 65536).
 */
#define QW_MEASURE_NOALLOC_MAX_LEN 65536

/*
 * qw_measure_register without any device allocation.  No counterpart in the
 * paper: a service of the library for callers that cannot call cudaMalloc or
 * cudaMallocAsync when they measure -- a runtime whose device memory is owned
 * by another allocator that has no headroom left (a cudaMalloc there fails,
 * or evicts the owner's cached blocks), or a loop that must not enter the
 * allocator for latency reasons (a cudaMalloc may synchronise the device).
 * qw_measure_register may allocate its histogram (the first time a len is
 * larger than every earlier one); this entry point never allocates: it
 * accumulates into a fixed 512 KiB array of the library's device image,
 * which every GPU that loads the library keeps until the process exits.  Same
 * arguments and result (probs is a host array of len doubles).
 * Limits and caveats:
 *   - len must be <= QW_MEASURE_NOALLOC_MAX_LEN, else QW_ERR_ARG;
 *   - the first call on a device looks up the array's device address once
 *     (cudaGetSymbolAddress, with that device current); make that first call
 *     before any stream capture begins;
 *   - all calls share the one array and it keeps the last call's contents:
 *     each call zeroes the bins it uses before accumulating, but calls whose
 *     GPU work overlaps (issued on different streams with no ordering between
 *     them) race on it and give wrong results;
 *   - like qw_measure_register it synchronises the simulator's stream.
 * Errors: QW_ERR_ARG, QW_ERR_STATE, QW_ERR_CUDA.
 */
int qw_measure_register_noalloc(qw_sim *sim, int32_t inst, int32_t reg_id, double *probs,
                                int64_t len);

/*
 * Row-partitioned walk (no counterpart in the paper's single-core simulator;
 * it follows from Sec. IV: T~^dag, P and T~ never change (jc, j, b1) and read
 * only row j of the QRAM, so a simulator holding a set of rows advances them
 * alone, and S, which moves a branch to row (kc, k, b2), is the one exchange
 * of a step).  Partition p of nparts (qw_sim_opts.nparts, .part; one instance,
 * fuse_reflection = 1, walk_variant <= 4, no QLS) owns the rows (0, j, b1)
 * with j in [p R, (p + 1) R), R = ceil(N / nparts), and the garbage rows
 * (jc != 0 or j >= N) whose (jc, j) hashes to p (qw_part_owner).
 * qw_state_init stores only the owned rows of |b~>.  A walk step of a
 * partition leaves the branches S sends to another partition's rows in that
 * partition's outbox segment; they join the state once delivered to it with
 * qw_part_inbox, before its next step.  Each partition's step records the
 * norm of what it emitted (qw_part_norm); the renormalisation of the next
 * step needs the global norm (qw_part_set_norm).  Steps are issued one at a
 * time (no CUDA graph).
 * Outbox entries (32 bytes): uint64 row key inst << 40 | jc << 20 | j << 1 |
 * b1, uint64 local registers b2 | k << 1 | kc << (1 + nb), double re, im.
 */
typedef struct {
    uint64_t rowkey, local;
    double re, im;
} qw_part_entry;

/* Partition owning row (jc, j) of a walk on an N-row matrix split nparts
 * ways (the rule above; host-only arithmetic, no device needed); -1 on a bad
 * argument. */
int qw_part_owner(int32_t n, int32_t nparts, int32_t jc, int32_t j);

/*
 * Copy the outbox segment toward partition dest, as left by the last walk
 * step, into the caller's device buffer dst (cap entries); *count receives
 * its length (more than cap: only cap copied).  Synchronises.
 * Errors: QW_ERR_ARG, QW_ERR_STATE (not partitioned), QW_ERR_CUDA.
 */
int qw_part_outbox(qw_sim *sim, int32_t dest, qw_part_entry *dst, int64_t cap, int64_t *count);

/*
 * Append count entries received from other partitions (device memory,
 * caller-owned) to the state; entries must name rows this partition owns.
 * Synchronises.  Errors: QW_ERR_ARG, QW_ERR_STATE, QW_ERR_CAPACITY, QW_ERR_CUDA.
 */
int qw_part_inbox(qw_sim *sim, const qw_part_entry *entries, int64_t count);

/* ||.||^2 of what this partition's last step emitted (its rows and its
 * outboxes), in FP64.  Synchronises. */
int qw_part_norm(qw_sim *sim, double *local_norm2);

/* Set the renormalisation of the next step from the global norm (the sum of
 * every partition's qw_part_norm): scale sqrt(target / global_norm2) when
 * renormalising, else 1. */
int qw_part_set_norm(qw_sim *sim, double global_norm2);

/*
 * nsteps steps of a walk partitioned among nparts simulators of one process
 * on one device: each step runs every partition's step kernel on its stream;
 * then, on each partition's stream once every step kernel is done (CUDA
 * events), the entries the others' S sent to it are appended straight from
 * their outbox segments (the counts read on the device) and its
 * renormalisation factor is set from the summed norms of all partitions'
 * outputs; a partition's next step waits for every exchange of the previous
 * one.  No host synchronisation between steps: the call synchronises once at
 * the end and reads every partition's device status.  After a device error
 * (an outbox or a row overflow) the partitions are not at a common step:
 * initialise them again.
 * Errors: QW_ERR_ARG (not a set of partitions 0 .. nparts - 1 of one walk),
 * QW_ERR_STATE, QW_ERR_CAPACITY, QW_ERR_DEVICE_STATUS, QW_ERR_CUDA.
 */
int qw_part_walk(qw_sim **sims, int32_t nparts, int64_t nsteps);

/* Number of branches of instance inst (inst = -1: all instances). */
int qw_state_size(qw_sim *sim, int32_t inst, int64_t *count);

/*
 * Export instance inst (-1: all): the simulator's state array -- the list of
 * (register key, amplitude) branches of Sec. V-A ("Main idea": the packed
 * registers of a basis state, and its complex amplitude) -- in canonical
 * order, keys ascending.  Each
 * key occupies key_words (1..10) uint64 words, least significant word first,
 * zero-extended; the packed layout from bit 0 up is
 *   b2 (1) | k (nb) | kc (nb) | b1 (1) | j (nb) | jc (nb) | A (16) | inst (16).
 * amps receives 2 doubles (re, im) per branch.  Writes min(count, cap)
 * branches; *count receives the total.  nb is reported by qw_sim_info.
 * Errors: QW_ERR_ARG (key_words too small for the layout), QW_ERR_STATE, QW_ERR_CUDA.
 */
int qw_state_export(qw_sim *sim, int32_t inst, int32_t key_words, uint64_t *keys, double *amps,
                    int64_t cap, int64_t *count);

/*
 * Replace the whole state (every instance) -- the branch list of Sec. V-A --
 * by the count branches given in the packed layout of qw_state_export (key_words words per key, the instance
 * field included) with amplitudes amps (2 doubles each): checkpoint / resume,
 * or any state of the register space.  Keys must be distinct, name existing
 * instances, and hold A = 0 (A is zero between walk steps).  The
 * renormalisation target becomes the imported norm.
 * Errors: QW_ERR_ARG (layout, duplicate key, A != 0, instance out of range),
 * QW_ERR_CAPACITY (a row exceeds row_capacity or the garbage-row table),
 * QW_ERR_CUDA.
 */
int qw_state_import(qw_sim *sim, int32_t key_words, const uint64_t *keys, const double *amps,
                    int64_t count);

/*
 * Register-faithful sub-operations (Sec. V-A, the working-qubit count of
 * Sec. V-C-1, Alg. 1, Eq. "Newprocess").  The paper's simulator keeps every
 * working register of a semi-quantum operation in the state: the QRAM
 * address that O_s' and O_A' compute out of place, and the quantum binary
 * search's left, right, mid, midval, flag and comparison bits with the
 * push/pop stack of one (mid, midval, cl, ce) frame per probe.  These calls
 * run the walk at that granularity on one list of all branches in device
 * memory (the flat path of walk_variant 5) whose keys hold those registers
 * beside the base ones (QW_FQ_KEY_WORDS 64-bit words per branch).
 *
 * QRAM addresses (Fig. 1): the value segment [0, N s) holds A_jl at j s + l,
 * the column segment [N s, 2 N s) holds the column index of slot l of row j
 * at N s + j s + l; a read outside its segment gives 0.  Sub-operations:
 *   QW_FQ_ADDR_COL  addr ^= N s + j s + k
 *   QW_FQ_QRAM_COL  kc ^= QRAM[addr] (column segment)
 *   QW_FQ_QBS_FWD   Alg. 1 with target kc on row j's column segment,
 *                   k ^= the index found; left, right, flag and L + 1 stack
 *                   frames (L = ceil(log2 s)) stay
 *   QW_FQ_QBS_BWD   Alg. 1 undone in reverse: the working registers back to
 *                   0 (k kept)
 *   QW_FQ_SWAP      swap(k, kc)
 *   QW_FQ_ADDR_VAL  addr ^= j s + k           (only where jc = kc = 0)
 *   QW_FQ_QRAM_VAL  A ^= QRAM[addr] (value segment; only where jc = kc = 0)
 *   QW_FQ_R, QW_FQ_RDAG, QW_FQ_H, QW_FQ_P, QW_FQ_S  the walk's operators
 *   QW_FQ_ALLOC_A, QW_FQ_FREE_A  A's allocation (FREE_A checks A = 0)
 * so O_s' = ADDR_COL QRAM_COL ADDR_COL QBS_FWD QBS_BWD SWAP, O_s'^dag =
 * SWAP QBS_FWD QBS_BWD ADDR_COL QRAM_COL ADDR_COL (the search with its
 * uncomputation is k ^= index, its own inverse, so that pair keeps its order)
 * and O_A' = ADDR_VAL QRAM_VAL ADDR_VAL.  The operators
 * R .. FREE_A act on the base registers and need every working register at 0.
 * QW_FQ_STEP_LEN codes in QW_FQ_STEP are W = S T~ P T~^dag (Alg. "Quantum
 * walk operator"); walk_variant 6 runs them as one walk step.
 */
#define QW_FQ_ADDR_COL 1
#define QW_FQ_QRAM_COL 2
#define QW_FQ_QBS_FWD 3
#define QW_FQ_QBS_BWD 4
#define QW_FQ_SWAP 5
#define QW_FQ_ADDR_VAL 6
#define QW_FQ_QRAM_VAL 7
#define QW_FQ_R 8
#define QW_FQ_RDAG 9
#define QW_FQ_H 10
#define QW_FQ_P 11
#define QW_FQ_S 12
#define QW_FQ_ALLOC_A 13
#define QW_FQ_FREE_A 14
#define QW_FQ_KEY_WORDS 10
#define QW_FQ_FRAMES 8 /* stack frames in an exported row: s <= 128 */
#define QW_FQ_COLS (16 + 4 * QW_FQ_FRAMES)
#define QW_FQ_STEP_LEN 58
#define QW_FQ_OS_SEQ QW_FQ_ADDR_COL, QW_FQ_QRAM_COL, QW_FQ_ADDR_COL, QW_FQ_QBS_FWD, QW_FQ_QBS_BWD, QW_FQ_SWAP
#define QW_FQ_OSDAG_SEQ QW_FQ_SWAP, QW_FQ_QBS_FWD, QW_FQ_QBS_BWD, QW_FQ_ADDR_COL, QW_FQ_QRAM_COL, QW_FQ_ADDR_COL
#define QW_FQ_OA_SEQ QW_FQ_ADDR_VAL, QW_FQ_QRAM_VAL, QW_FQ_ADDR_VAL
#define QW_FQ_STEP                                                                                               \
    {QW_FQ_ALLOC_A, QW_FQ_OSDAG_SEQ, QW_FQ_OA_SEQ, QW_FQ_OS_SEQ, QW_FQ_RDAG, QW_FQ_OSDAG_SEQ, QW_FQ_OA_SEQ,        \
     QW_FQ_H,       QW_FQ_FREE_A,    QW_FQ_P,      QW_FQ_ALLOC_A, QW_FQ_H,   QW_FQ_OA_SEQ,    QW_FQ_OS_SEQ,        \
     QW_FQ_R,       QW_FQ_OSDAG_SEQ, QW_FQ_OA_SEQ, QW_FQ_OS_SEQ,  QW_FQ_FREE_A, QW_FQ_S}

/*
 * Layout of the register-faithful keys for this simulator: *addr_bits the
 * width of the address and of left / right / mid, *key_bits the bits a key
 * uses (the base registers' 128, the working registers, L + 1 frames),
 * *live_bits the qubits of the schedule at its widest (inside Alg. 1 with a
 * full stack: the base registers, A, the address and Alg. 1's registers).
 * All nullable.  Returns QW_OK when the layout fits QW_FQ_KEY_WORDS words and
 * QW_FQ_FRAMES frames, QW_ERR_ARG otherwise (the register-faithful calls are
 * then refused).
 */
int qw_faithful_info(const qw_sim *sim, int32_t *addr_bits, int32_t *key_bits, int64_t *live_bits);

/*
 * Open a register-faithful session: the state (with its pending
 * renormalisation) becomes a list of branches, every working register 0.
 * Until qw_faithful_end the row buckets keep the state as it was here, and
 * walk steps, QLS, qw_state_init and qw_state_import are refused
 * (QW_ERR_STATE).  Synchronises.  Errors: QW_ERR_ARG (layout too wide, see
 * qw_faithful_info), QW_ERR_STATE (no state, or a session is open),
 * QW_ERR_CUDA.
 */
int qw_faithful_begin(qw_sim *sim);

/*
 * Apply nops sub-operations (QW_FQ_* codes) in order to the open session's
 * list.  R, R^dag and H drop outputs with |a| <= prune_tau, as a walk step
 * does.  Synchronises.  Errors: QW_ERR_ARG (unknown code), QW_ERR_STATE (no
 * session), QW_ERR_DEVICE_STATUS (a working register was not 0 where it must
 * be, or A not 0 at FREE_A; the list is then as after the failing
 * sub-operation), QW_ERR_CUDA.
 */
int qw_faithful_apply(qw_sim *sim, const int32_t *ops, int32_t nops);

/*
 * The open session's list as a table: *count = its branches; the first
 * min(count, cap) rows, sorted ascending by their columns, are written to
 * regs (QW_FQ_COLS uint64 per branch, host memory: inst, jc, j, b1, kc, k, b2,
 * A, addr, left, right, mid, midval, flag, cl, ce, then QW_FQ_FRAMES frames of
 * (mid, midval, cl, ce), frames past L + 1 zero) and amps (2 doubles each).
 * cap = 0 only counts.  Synchronises.  Errors: QW_ERR_ARG, QW_ERR_STATE,
 * QW_ERR_CUDA.
 */
int qw_faithful_export(qw_sim *sim, uint64_t *regs, double *amps, int64_t cap, int64_t *count);

/*
 * Close the session.  keep != 0: the list becomes the state as the output of
 * one walk step (the step counter and qw_step_stats advance; with
 * renormalisation on, the next step rescales it to the target norm); every
 * working register and A must be 0, and with overflow_fallback the row
 * buckets grow to the largest row.  keep = 0: the list is dropped and the
 * state is the one at qw_faithful_begin.  Synchronises.  Errors: QW_ERR_STATE
 * (no session), QW_ERR_DEVICE_STATUS (a register not 0: the session stays
 * open), QW_ERR_CAPACITY (a row does not fit and overflow_fallback = 0: the
 * session is closed, the state is the one at qw_faithful_begin), QW_ERR_CUDA.
 */
int qw_faithful_end(qw_sim *sim, int32_t keep);

/* nb, s, number of instances, and the total device bytes held (all nullable). */
int qw_sim_info(const qw_sim *sim, int32_t *nb, int32_t *s, int32_t *num_instances,
                int64_t *device_bytes);

/*
 * Branch counters of the walk steps run since creation or the last reset,
 * summed over steps: out[0] row items processed (a row, or the two rows of a j
 * run as one segment), out[1] branches entering the
 * steps (input of R^dag), out[2] after R^dag, out[3] after the first H (only
 * with fuse_reflection = 0), out[4] after H P H, out[5] after R (branches
 * written), out[6] steps counted.  Writes min(len, 8) values; reset != 0
 * zeroes the counters afterwards.  Errors: QW_ERR_ARG, QW_ERR_CUDA.
 */
int qw_step_stats(qw_sim *sim, int64_t *out, int32_t len, int32_t reset);

/* Kernel launches issued by this simulator since creation (for accounting). */
int64_t qw_launch_count(const qw_sim *sim);

/* Free all device memory of the simulator.  Accepts NULL. */
int qw_sim_destroy(qw_sim *sim);

/* Message of the last failure on sim (a static string if sim is NULL). */
const char *qw_last_error(const qw_sim *sim);

#ifdef __cplusplus
}
#endif

#endif /* QWALK_H */
