/*
 * qw_oracle.c -- plain, slow CPU FP64 reference of the register-level
 * sparse-state simulation of the quantum walk on a CSC matrix in QRAM
 * (arXiv 2303.06890).  TEST INFRASTRUCTURE ONLY: the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg load this library; the product
 * never does.  It shares no code with the CUDA path.
 *
 * State (Sec. V-A, "Main idea"): a list of branches, each holding one value
 * per register (the state array) and one complex amplitude (the amplitude
 * vector), plus per-register metadata (width, live flag).
 *
 * Registers of the walk (Sec. IV, "Implementation of the quantum walk"):
 *   jc, j, b1, kc, k, b2   widths nb, nb, 1, nb, nb, 1   (nb = ceil(log2 N))
 *   A                      width 16, allocated inside T~ and T~^dag only.
 *
 * Operations follow the paper literally:
 *   - semi-quantum ops (Sec. V-A, Fig. 8b): per-branch reversible register
 *     maps: QRAM XOR-lookup, address arithmetic, the quantum binary search of
 *     Alg. 1 with its push/pop garbage stack and full uncomputation, swaps and
 *     the controlled phase flip;
 *   - interference ops (Sec. V-A, "Classical simulation of the interference
 *     operation"): (1) sort the branches so that those equal on every idle
 *     register are contiguous, (2) apply the small dense unitary to each
 *     group's zero-filled vector, (3) drop branches whose |amplitude| <= tau.
 *
 * Readings where the paper is silent or garbled (each is shared with the
 * CUDA path by specification, not by code):
 *   - QRAM image (Fig. 1): value segment [0, N s) then column-index segment
 *     [N s, 2 N s); row j's slot l at j*s + l.  Rows with fewer than s
 *     non-zeros are padded with explicit zero elements ("fill zeros",
 *     Sec. II-C) placed at the first columns not already in the row, scanning
 *     j+1, j+2, ... cyclically; each row's column list is then sorted, so the
 *     list is unique and sorted as the QBS definition (Def. 1) requires.
 *   - A read outside its segment returns 0 (garbage subspaces reach l >= s
 *     and rows j >= N).
 *   - QBS output is the in-row index mid - offset (Def. 1 defines i(d) as the
 *     list index, while Alg. 1 XORs the absolute address mid); floor
 *     midpoint, right end exclusive,
 *     ceil(log2 s)+1 probes, stop at the first equal element.
 *   - O_s' computes the QRAM address out of place (Eq. "Newprocess").
 *   - Conditional rotation (Alg. T~ and the footnote of Sec. IV): for A's Q1.15
 *     value a, g = sqrt(1-|a|); f = sqrt(a) if a >= 0, else i*sigma*sqrt(|a|)
 *     with sigma = +1 when j <= k and -1 when j > k; R = [[f, -g], [g, conj f]]
 *     acting on b2, R^dag its conjugate transpose.
 *   - P = 2 Pi - 1: the sign flips unless b1, k, b2, jc, kc are all zero
 *     (Alg. "Quantum walk operator"; Eq. (impl)).
 *     Optionally (or_set_rot_bits) the angle arccos(sqrt|a|) is first rounded
 *     to a multiple of (pi/2) / 2^bits, a fixed-point angle register as in
 *     Table 2, and f, g are its cosine and sine.
 *   - H of T~ acts on the low log2(s) bits of register k (Sec. IV, T~).
 *
 * Pins: the test-suite checks this oracle against closed forms, brute force
 * and the paper's printed examples.  Parity unpinned: the amplitudes of
 * garbage branches (jc or kc != 0, rows j >= N) follow only from the readings
 * above -- no closed form of the paper reaches them -- and are compared with
 * the CUDA path as they stand; what pins them is an invariant only: on random
 * states over the whole register space each op of W is undone by its
 * inverse, and W by T~ P T~^dag S.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { R_JC = 0, R_J, R_B1, R_KC, R_K, R_B2, R_A, NREG };

typedef struct {
    uint64_t r[NREG];
    double complex a;
} branch;

typedef struct {
    int width;
    int live;
} reg_meta;

typedef struct oracle {
    int64_t n, s, L, nb, w;
    int64_t ns;         /* N * s: words per segment */
    int64_t val_base;   /* start of the matrix-element segment */
    int64_t col_base;   /* start of the sparsity (column index) segment */
    uint32_t *mem;      /* QRAM words, 2 * N * s */
    branch *st;         /* state */
    int64_t m, cap;
    double tau;
    int rot_bits; /* 0: exact f, g; > 0: the rotation angle held in rot_bits bits */
    reg_meta meta[NREG];
    int64_t live_bits, max_live_bits;
    int64_t violations; /* ancilla-not-zero and other self-check failures */
    uint64_t *g;        /* register-faithful sub-operations: NG working registers per branch */
    int64_t gm;         /* rows of g (0: none allocated, all working registers zero) */
} oracle;

/* ------------------------------------------------------------------------- */
/* memory                                                                    */

static int reserve(oracle *o, int64_t need)
{
    if (need <= o->cap) return 0;
    int64_t cap = o->cap ? o->cap : 1024;
    while (cap < need) cap *= 2;
    branch *p = (branch *)realloc(o->st, (size_t)cap * sizeof(branch));
    if (!p) return -1;
    o->st = p;
    o->cap = cap;
    return 0;
}

static void check(oracle *o, int ok)
{
    if (!ok) o->violations++;
}

/* register allocation and the working-qubit counter (Sec. V-C-1) */
static void reg_alloc(oracle *o, int r, int width)
{
    check(o, !o->meta[r].live);
    for (int64_t i = 0; i < o->m; ++i) check(o, o->st[i].r[r] == 0);
    o->meta[r].live = 1;
    o->meta[r].width = width;
    o->live_bits += width;
    if (o->live_bits > o->max_live_bits) o->max_live_bits = o->live_bits;
}

static void reg_free(oracle *o, int r)
{
    /* safe discard: every branch must hold 0 in the register */
    for (int64_t i = 0; i < o->m; ++i) check(o, o->st[i].r[r] == 0);
    o->meta[r].live = 0;
    o->live_bits -= o->meta[r].width;
}

static void note_transient_bits(oracle *o, int64_t bits)
{
    if (o->live_bits + bits > o->max_live_bits) o->max_live_bits = o->live_bits + bits;
}

/* ------------------------------------------------------------------------- */
/* QRAM: U|i>|z> = |i>|z xor d_i>  (Sec. V-A, QRAM paragraph)                 */

static uint64_t qram(const oracle *o, uint64_t addr, int64_t seg_base)
{
    if ((int64_t)addr < seg_base || (int64_t)addr >= seg_base + o->ns) return 0;
    return o->mem[addr];
}

/* ------------------------------------------------------------------------- */
/* Quantum binary search, Alg. 1, with the push/pop garbage stack (Fig. 2).  */
/* Returns out xor i(target) and checks that every ancilla returns to 0.     */

typedef struct {
    uint64_t mid, midval;
    int cl, ce;
} qbs_frame;

static uint64_t qbs(oracle *o, uint64_t offset, uint64_t target, uint64_t out)
{
    uint64_t left = 0, right = 0, mid = 0, midval = 0;
    int flag = 0, cl = 0, ce = 0;
    qbs_frame stack[72];
    int sp = 0;
    const int iters = (int)o->L + 1; /* for i = 0 : ceil(log s) */

    /* allocate and initialise the search window and the loop flag */
    left ^= offset;
    right ^= left + (uint64_t)o->s;
    flag ^= 1;
    for (int it = 0; it < iters; ++it) {
        if (flag) mid ^= (left + right) / 2;                 /* midpoint */
        if (flag) midval ^= qram(o, mid, o->col_base);       /* QRAM probe */
        if (flag) {                                          /* compare */
            cl ^= (midval < target);
            ce ^= (midval == target);
        }
        if (ce) out ^= mid - offset;                         /* found: write output */
        if (ce) flag ^= 1;                                   /* found: stop */
        if (flag && cl) { uint64_t t = mid; mid = left; left = t; }   /* go right */
        if (flag) cl ^= 1;
        if (flag && cl) { uint64_t t = mid; mid = right; right = t; } /* go left */
        /* push: the loop variables move onto the garbage stack, zeros remain */
        stack[sp].mid = mid;
        stack[sp].midval = midval;
        stack[sp].cl = cl;
        stack[sp].ce = ce;
        sp++;
        mid = 0;
        midval = 0;
        cl = 0;
        ce = 0;
    }
    /* uncompute every loop step except the output write, in reverse order */
    for (int it = iters - 1; it >= 0; --it) {
        sp--;
        mid = stack[sp].mid;
        midval = stack[sp].midval;
        cl = stack[sp].cl;
        ce = stack[sp].ce;
        if (flag && cl) { uint64_t t = mid; mid = right; right = t; }
        if (flag) cl ^= 1;
        if (flag && cl) { uint64_t t = mid; mid = left; left = t; }
        if (ce) flag ^= 1;
        if (flag) {
            cl ^= (midval < target);
            ce ^= (midval == target);
        }
        if (flag) midval ^= qram(o, mid, o->col_base);
        if (flag) mid ^= (left + right) / 2;
        check(o, mid == 0 && midval == 0 && cl == 0 && ce == 0);
    }
    flag ^= 1;
    right ^= left + (uint64_t)o->s;
    left ^= offset;
    check(o, left == 0 && right == 0 && flag == 0);
    return out;
}

/* ------------------------------------------------------------------------- */
/* Oracles on one branch                                                     */

/* O_A' (Alg. O_A'): A ^= a_{j,l} with l in register k, controlled by jc = kc = 0
 * (Sec. III-B: O_A' controlled by the two added registers). */
static void oa_branch(oracle *o, branch *e)
{
    if (e->r[R_JC] != 0 || e->r[R_KC] != 0) return;
    uint64_t anc = 0;
    anc ^= (uint64_t)o->val_base + e->r[R_J] * (uint64_t)o->s + e->r[R_K];
    e->r[R_A] ^= qram(o, anc, o->val_base);
    anc ^= (uint64_t)o->val_base + e->r[R_J] * (uint64_t)o->s + e->r[R_K];
    check(o, anc == 0);
}

/* O_s' (Eq. "Newprocess"): |j>|l>|z> -> |j>|z^K(j,l)>|l^I(j, z^K(j,l))>,
 * with l in register k and z in register kc. */
static void os_branch(oracle *o, branch *e)
{
    uint64_t j = e->r[R_J];
    uint64_t anc = 0;
    anc ^= (uint64_t)o->col_base + j * (uint64_t)o->s + e->r[R_K]; /* address */
    e->r[R_KC] ^= qram(o, anc, o->col_base);                        /* QRAM */
    anc ^= (uint64_t)o->col_base + j * (uint64_t)o->s + e->r[R_K]; /* uncompute */
    check(o, anc == 0);
    e->r[R_K] = qbs(o, (uint64_t)o->col_base + j * (uint64_t)o->s, e->r[R_KC], e->r[R_K]);
    uint64_t t = e->r[R_K];                                          /* swap */
    e->r[R_K] = e->r[R_KC];
    e->r[R_KC] = t;
}

/* O_s'^dag: the three steps of O_s' undone in reverse order. */
static void osdag_branch(oracle *o, branch *e)
{
    uint64_t j = e->r[R_J];
    uint64_t t = e->r[R_K];
    e->r[R_K] = e->r[R_KC];
    e->r[R_KC] = t;
    e->r[R_K] = qbs(o, (uint64_t)o->col_base + j * (uint64_t)o->s, e->r[R_KC], e->r[R_K]);
    uint64_t anc = 0;
    anc ^= (uint64_t)o->col_base + j * (uint64_t)o->s + e->r[R_K];
    e->r[R_KC] ^= qram(o, anc, o->col_base);
    anc ^= (uint64_t)o->col_base + j * (uint64_t)o->s + e->r[R_K];
    check(o, anc == 0);
}

/* P = 2 sum_j |j~><j~| - 1: flip unless b1, k, b2, jc, kc are all zero. */
static void p_branch(oracle *o, branch *e)
{
    (void)o;
    int zero = e->r[R_B1] == 0 && e->r[R_K] == 0 && e->r[R_B2] == 0 &&
               e->r[R_JC] == 0 && e->r[R_KC] == 0;
    if (!zero) e->a = -e->a;
}

/* S: swap (jc, j, b1) with (kc, k, b2). */
static void s_branch(oracle *o, branch *e)
{
    (void)o;
    uint64_t t;
    t = e->r[R_J];  e->r[R_J] = e->r[R_K];   e->r[R_K] = t;
    t = e->r[R_JC]; e->r[R_JC] = e->r[R_KC]; e->r[R_KC] = t;
    t = e->r[R_B1]; e->r[R_B1] = e->r[R_B2]; e->r[R_B2] = t;
}

static void for_each(oracle *o, void (*fn)(oracle *, branch *))
{
    for (int64_t i = 0; i < o->m; ++i) fn(o, &o->st[i]);
}

/* ------------------------------------------------------------------------- */
/* Interference operation (grouping, computing, clearing)                    */

typedef void (*unitary_fn)(const oracle *o, const branch *idle, int dim, double complex *u);

static const oracle *g_sort_o;
static int g_sort_reg;
static uint64_t g_sort_mask;

static int cmp_grouping(const void *pa, const void *pb)
{
    const branch *x = (const branch *)pa, *y = (const branch *)pb;
    for (int r = 0; r < NREG; ++r) {
        uint64_t mx = (r == g_sort_reg) ? (x->r[r] & ~g_sort_mask) : x->r[r];
        uint64_t my = (r == g_sort_reg) ? (y->r[r] & ~g_sort_mask) : y->r[r];
        if (mx != my) return mx < my ? -1 : 1;
    }
    uint64_t tx = x->r[g_sort_reg] & g_sort_mask, ty = y->r[g_sort_reg] & g_sort_mask;
    return (tx > ty) - (tx < ty);
}

static int same_group(const branch *x, const branch *y, int reg, uint64_t mask)
{
    for (int r = 0; r < NREG; ++r) {
        uint64_t mx = (r == reg) ? (x->r[r] & ~mask) : x->r[r];
        uint64_t my = (r == reg) ? (y->r[r] & ~mask) : y->r[r];
        if (mx != my) return 0;
    }
    return 1;
}

/* Apply the 2^nbits x 2^nbits unitary u(idle) to bits [bitlo, bitlo+nbits) of
 * register `reg`; u is row-major, u[out*dim + in]. */
static int interfere(oracle *o, int reg, int bitlo, int nbits, unitary_fn fn)
{
    const int dim = 1 << nbits;
    const uint64_t mask = ((uint64_t)(dim - 1)) << bitlo;
    /* grouping */
    g_sort_o = o;
    g_sort_reg = reg;
    g_sort_mask = mask;
    qsort(o->st, (size_t)o->m, sizeof(branch), cmp_grouping);

    branch *out = NULL;
    int64_t mo = 0, cap = 0;
    double complex *u = (double complex *)malloc(sizeof(double complex) * (size_t)dim * dim);
    double complex *v = (double complex *)malloc(sizeof(double complex) * (size_t)dim);
    if (!u || !v) { free(u); free(v); return -1; }
    int64_t i = 0;
    while (i < o->m) {
        int64_t g = i + 1;
        while (g < o->m && same_group(&o->st[i], &o->st[g], reg, mask)) ++g;
        /* computing, on the zero-filled group vector */
        for (int t = 0; t < dim; ++t) v[t] = 0;
        for (int64_t q = i; q < g; ++q) v[(o->st[q].r[reg] & mask) >> bitlo] = o->st[q].a;
        fn(o, &o->st[i], dim, u);
        if (mo + dim > cap) {
            cap = cap ? cap * 2 : 1024;
            while (mo + dim > cap) cap *= 2;
            branch *p = (branch *)realloc(out, (size_t)cap * sizeof(branch));
            if (!p) { free(out); free(u); free(v); return -1; }
            out = p;
        }
        for (int t = 0; t < dim; ++t) {
            double complex acc = 0;
            for (int q = 0; q < dim; ++q) acc += u[t * dim + q] * v[q];
            /* clearing zero elements */
            if (creal(acc) * creal(acc) + cimag(acc) * cimag(acc) <= o->tau * o->tau) continue;
            branch e = o->st[i];
            e.r[reg] = (e.r[reg] & ~mask) | ((uint64_t)t << bitlo);
            e.a = acc;
            out[mo++] = e;
        }
        i = g;
    }
    free(u);
    free(v);
    free(o->st);
    o->st = out;
    o->m = mo;
    o->cap = cap;
    return 0;
}

/* Hadamard on log2(s) bits: u[t][q] = (-1)^{popcount(t & q)} / sqrt(s). */
static void u_hadamard(const oracle *o, const branch *idle, int dim, double complex *u)
{
    (void)o;
    (void)idle;
    double h = 1.0 / sqrt((double)dim);
    for (int t = 0; t < dim; ++t)
        for (int q = 0; q < dim; ++q)
            u[t * dim + q] = (__builtin_popcount((unsigned)(t & q)) & 1) ? -h : h;
}

/* f and g of the conditional rotation from A's Q1.15 code and (j, k).
 * Exact (rot_bits = 0): |f| = sqrt(|a|), g = sqrt(1 - |a|).  With the angle in
 * a fixed-point register (the square root and arccos registers that Table 2
 * lists for the conditional rotation): theta = arccos(sqrt(|a|)) in [0, pi/2]
 * rounded to a multiple of (pi/2) / 2^rot_bits (half to even), |f| = cos,
 * g = sin of the rounded angle. */
static void rotation_fg(const oracle *o, const branch *e, double complex *f, double *g)
{
    int16_t q = (int16_t)(uint16_t)e->r[R_A];
    double a = (double)q / 32768.0;
    double mag = fabs(a);
    double fm;
    if (o->rot_bits > 0) {
        double step = ldexp(1.5707963267948966, -o->rot_bits);
        double th = nearbyint(acos(sqrt(mag)) / step) * step;
        fm = cos(th);
        *g = sin(th);
    } else {
        fm = sqrt(mag);
        *g = sqrt(1.0 - mag);
    }
    if (q >= 0) {
        *f = fm;
    } else {
        double sigma = (e->r[R_J] <= e->r[R_K]) ? 1.0 : -1.0;
        *f = I * (sigma * fm);
    }
}

static void u_rot(const oracle *o, const branch *idle, int dim, double complex *u)
{
    (void)o;
    (void)dim;
    double complex f;
    double g;
    rotation_fg(o, idle, &f, &g);
    u[0] = f;  u[1] = -g;       /* R|0> = f|0> + g|1> */
    u[2] = g;  u[3] = conj(f);  /* R|1> = -g|0> + conj(f)|1> */
}

static void u_rotdag(const oracle *o, const branch *idle, int dim, double complex *u)
{
    (void)o;
    (void)dim;
    double complex f;
    double g;
    rotation_fg(o, idle, &f, &g);
    u[0] = conj(f); u[1] = g;
    u[2] = -g;      u[3] = f;
}

/* ------------------------------------------------------------------------- */
/* Composite operators                                                       */

static int op_h(oracle *o) { return interfere(o, R_K, 0, (int)o->L, u_hadamard); }
static int op_r(oracle *o) { return interfere(o, R_B2, 0, 1, u_rot); }
static int op_rdag(oracle *o) { return interfere(o, R_B2, 0, 1, u_rotdag); }

static void op_os(oracle *o)
{
    /* O_s' needs one address ancilla and QBS's registers and stack */
    int64_t addr_w = 1;
    while (((int64_t)1 << addr_w) < 2 * o->ns + 1) addr_w++;
    note_transient_bits(o, addr_w + 3 * addr_w + o->w + 3 + (o->L + 1) * (addr_w + o->w + 2));
    for_each(o, os_branch);
}

static void op_osdag(oracle *o)
{
    for_each(o, osdag_branch);
}

/* T~ (Alg. T~): H, O_A', O_s', R, O_s'^dag, O_A' (uncompute), O_s'. */
static int op_t(oracle *o)
{
    reg_alloc(o, R_A, (int)o->w);
    if (op_h(o)) return -1;
    for_each(o, oa_branch);
    op_os(o);
    if (op_r(o)) return -1;
    op_osdag(o);
    for_each(o, oa_branch);
    op_os(o);
    reg_free(o, R_A);
    return 0;
}

/* T~^dag: the steps of T~ inverted in reverse order. */
static int op_tdag(oracle *o)
{
    reg_alloc(o, R_A, (int)o->w);
    op_osdag(o);
    for_each(o, oa_branch);
    op_os(o);
    if (op_rdag(o)) return -1;
    op_osdag(o);
    for_each(o, oa_branch);
    if (op_h(o)) return -1;
    reg_free(o, R_A);
    return 0;
}

/* W = S T~ P T~^dag (Alg. "Quantum walk operator"). */
static int op_w(oracle *o)
{
    if (op_tdag(o)) return -1;
    for_each(o, p_branch);
    if (op_t(o)) return -1;
    for_each(o, s_branch);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Register-faithful sub-operations                                          */
/*
 * The paper's simulator holds every working register of a semi-quantum op in
 * the state (Sec. V-A; the qubit count of Sec. V-C-1): the QRAM address of
 * O_s' and O_A' (Eq. "Newprocess", computed out of place), and Alg. 1's
 * left, right, mid, midval and flags with its push/pop garbage stack.  Here
 * each of those steps is an operation of its own, the working registers kept
 * per branch between them in g (NG values per branch, zero when idle):
 *   FQ_ADDR_COL  addr ^= col_base + j s + k
 *   FQ_QRAM_COL  kc ^= QRAM[addr] over the column segment
 *   FQ_QBS_FWD   Alg. 1's loop with target kc, output k ^= index: left,
 *                right, flag and the stack of (mid, midval, cl, ce) frames stay
 *   FQ_QBS_BWD   Alg. 1's uncomputation: every working register back to 0
 *   FQ_SWAP      swap(k, kc)
 *   FQ_ADDR_VAL  addr ^= val_base + j s + k           (controlled by jc = kc = 0)
 *   FQ_QRAM_VAL  A ^= QRAM[addr] over the value segment (controlled likewise)
 * so O_s' = ADDR_COL QRAM_COL ADDR_COL QBS_FWD QBS_BWD SWAP, O_s'^dag the same
 * in reverse, O_A' = ADDR_VAL QRAM_VAL ADDR_VAL.  The interference ops, P and
 * S act on the base registers; the working registers must be 0 there.
 */
enum { G_ADDR = 0, G_LEFT, G_RIGHT, G_MID, G_MIDVAL, G_FLAG, G_CL, G_CE, G_STK, NG = G_STK + 4 * 8 };
enum {
    FQ_ADDR_COL = 1, FQ_QRAM_COL, FQ_QBS_FWD, FQ_QBS_BWD, FQ_SWAP, FQ_ADDR_VAL, FQ_QRAM_VAL,
    FQ_R, FQ_RDAG, FQ_H, FQ_P, FQ_S, FQ_ALLOC_A, FQ_FREE_A
};

static int g_reserve(oracle *o)
{
    if (o->gm == o->m && o->g) return 0;
    free(o->g);
    o->g = (uint64_t *)calloc((size_t)(o->m ? o->m : 1) * NG, sizeof(uint64_t));
    o->gm = o->m;
    return o->g ? 0 : -1;
}

/* the working registers are 0 on every branch (an interference op, P and S
   act on the base registers only) */
static void g_check_free(oracle *o)
{
    if (!o->g) return;
    for (int64_t i = 0; i < o->gm * NG; ++i) check(o, o->g[i] == 0);
    free(o->g);
    o->g = NULL;
    o->gm = 0;
}

static void fq_branch(oracle *o, branch *e, uint64_t *g, int op)
{
    const uint64_t j = e->r[R_J];
    const uint64_t offset = (uint64_t)o->col_base + j * (uint64_t)o->s;
    switch (op) {
    case FQ_ADDR_COL: g[G_ADDR] ^= offset + e->r[R_K]; break;
    case FQ_QRAM_COL: e->r[R_KC] ^= qram(o, g[G_ADDR], o->col_base); break;
    case FQ_ADDR_VAL:
        if (e->r[R_JC] == 0 && e->r[R_KC] == 0) g[G_ADDR] ^= (uint64_t)o->val_base + j * (uint64_t)o->s + e->r[R_K];
        break;
    case FQ_QRAM_VAL:
        if (e->r[R_JC] == 0 && e->r[R_KC] == 0) e->r[R_A] ^= qram(o, g[G_ADDR], o->val_base);
        break;
    case FQ_SWAP: {
        uint64_t t = e->r[R_K];
        e->r[R_K] = e->r[R_KC];
        e->r[R_KC] = t;
        break;
    }
    case FQ_QBS_FWD: { /* Alg. 1, target kc, output into k */
        const uint64_t target = e->r[R_KC];
        g[G_LEFT] ^= offset;
        g[G_RIGHT] ^= g[G_LEFT] + (uint64_t)o->s;
        g[G_FLAG] ^= 1;
        for (int it = 0; it <= o->L; ++it) {
            uint64_t *fr = g + G_STK + 4 * it;
            if (g[G_FLAG]) g[G_MID] ^= (g[G_LEFT] + g[G_RIGHT]) / 2;
            if (g[G_FLAG]) g[G_MIDVAL] ^= qram(o, g[G_MID], o->col_base);
            if (g[G_FLAG]) {
                g[G_CL] ^= (g[G_MIDVAL] < target);
                g[G_CE] ^= (g[G_MIDVAL] == target);
            }
            if (g[G_CE]) e->r[R_K] ^= g[G_MID] - offset;
            if (g[G_CE]) g[G_FLAG] ^= 1;
            if (g[G_FLAG] && g[G_CL]) { uint64_t t = g[G_MID]; g[G_MID] = g[G_LEFT]; g[G_LEFT] = t; }
            if (g[G_FLAG]) g[G_CL] ^= 1;
            if (g[G_FLAG] && g[G_CL]) { uint64_t t = g[G_MID]; g[G_MID] = g[G_RIGHT]; g[G_RIGHT] = t; }
            /* push: the loop registers move into frame it, zeros remain */
            fr[0] = g[G_MID];
            fr[1] = g[G_MIDVAL];
            fr[2] = g[G_CL];
            fr[3] = g[G_CE];
            g[G_MID] = g[G_MIDVAL] = g[G_CL] = g[G_CE] = 0;
        }
        break;
    }
    case FQ_QBS_BWD: { /* the loop undone in reverse, all but the output */
        const uint64_t target = e->r[R_KC];
        for (int it = (int)o->L; it >= 0; --it) {
            uint64_t *fr = g + G_STK + 4 * it;
            g[G_MID] = fr[0];
            g[G_MIDVAL] = fr[1];
            g[G_CL] = fr[2];
            g[G_CE] = fr[3];
            fr[0] = fr[1] = fr[2] = fr[3] = 0;
            if (g[G_FLAG] && g[G_CL]) { uint64_t t = g[G_MID]; g[G_MID] = g[G_RIGHT]; g[G_RIGHT] = t; }
            if (g[G_FLAG]) g[G_CL] ^= 1;
            if (g[G_FLAG] && g[G_CL]) { uint64_t t = g[G_MID]; g[G_MID] = g[G_LEFT]; g[G_LEFT] = t; }
            if (g[G_CE]) g[G_FLAG] ^= 1;
            if (g[G_FLAG]) {
                g[G_CL] ^= (g[G_MIDVAL] < target);
                g[G_CE] ^= (g[G_MIDVAL] == target);
            }
            if (g[G_FLAG]) g[G_MIDVAL] ^= qram(o, g[G_MID], o->col_base);
            if (g[G_FLAG]) g[G_MID] ^= (g[G_LEFT] + g[G_RIGHT]) / 2;
            check(o, g[G_MID] == 0 && g[G_MIDVAL] == 0 && g[G_CL] == 0 && g[G_CE] == 0);
        }
        g[G_FLAG] ^= 1;
        g[G_RIGHT] ^= g[G_LEFT] + (uint64_t)o->s;
        g[G_LEFT] ^= offset;
        check(o, g[G_LEFT] == 0 && g[G_RIGHT] == 0 && g[G_FLAG] == 0);
        break;
    }
    default: break;
    }
}

/* address register width of the layout: every address a branch can form */
static int faithful_addr_bits(const oracle *o)
{
    uint64_t top = (uint64_t)o->ns + (((uint64_t)1 << o->nb) * (uint64_t)o->s) + ((uint64_t)1 << o->nb) + 1;
    int b = 0;
    while (((uint64_t)1 << b) < top) b++;
    return b;
}

/* live bits of the faithful schedule at its widest (inside O_s'): the base
   registers, A, the address and Alg. 1's registers with a full stack
   (Sec. V-C-1's count of working qubits, for this register layout) */
int64_t or_faithful_live_bits(const oracle *o)
{
    const int aw = faithful_addr_bits(o);
    return 4 * o->nb + 2 + o->w + aw + 3 * aw + 16 + 3 + (o->L + 1) * (aw + 16 + 2);
}

int or_apply_faithful(oracle *o, int op)
{
    switch (op) {
    case FQ_R: g_check_free(o); return op_r(o);
    case FQ_RDAG: g_check_free(o); return op_rdag(o);
    case FQ_H: g_check_free(o); return op_h(o);
    case FQ_P: g_check_free(o); for_each(o, p_branch); return 0;
    case FQ_S: g_check_free(o); for_each(o, s_branch); return 0;
    case FQ_ALLOC_A: g_check_free(o); reg_alloc(o, R_A, (int)o->w); return 0;
    case FQ_FREE_A: g_check_free(o); reg_free(o, R_A); return 0;
    default: break;
    }
    if (op < FQ_ADDR_COL || op > FQ_QRAM_VAL) return -1;
    if (g_reserve(o)) return -1;
    if (op == FQ_QBS_FWD) {
        const int aw = faithful_addr_bits(o);
        note_transient_bits(o, aw + 3 * aw + 16 + 3 + (o->L + 1) * (aw + 16 + 2));
    }
    for (int64_t i = 0; i < o->m; ++i) fq_branch(o, &o->st[i], o->g + i * NG, op);
    return 0;
}

/* Export with the working registers: regs m x (7 + NG) (jc, j, b1, kc, k, b2,
   A, then g), amps m x 2. */
int64_t or_export_faithful(const oracle *o, uint64_t *regs, double *amps, int64_t cap)
{
    int64_t m = o->m < cap ? o->m : cap;
    for (int64_t i = 0; i < m; ++i) {
        for (int r = 0; r < NREG; ++r) regs[i * (NREG + NG) + r] = o->st[i].r[r];
        for (int r = 0; r < NG; ++r) regs[i * (NREG + NG) + NREG + r] = (o->g && i < o->gm) ? o->g[i * NG + r] : 0;
        amps[2 * i] = creal(o->st[i].a);
        amps[2 * i + 1] = cimag(o->st[i].a);
    }
    return o->m;
}

int or_faithful_ng(void) { return NG; }
int or_faithful_addr_bits(const oracle *o) { return faithful_addr_bits(o); }

/* ------------------------------------------------------------------------- */
/* Public interface (ctypes)                                                 */

enum {
    OR_T = 0, OR_TDAG, OR_W, OR_P, OR_S, OR_H, OR_R, OR_RDAG, OR_OA, OR_OS, OR_OSDAG,
    OR_ALLOC_A, OR_FREE_A
};

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* CSC of a real symmetric matrix -> padded QRAM image (Fig. 1). */
oracle *or_create(int32_t n, const int32_t *colptr, const int32_t *rowidx, const int16_t *val_q15,
                  int32_t s, double tau)
{
    if (n < 1 || s < 1 || s > n || (s & (s - 1))) return NULL;
    oracle *o = (oracle *)calloc(1, sizeof(oracle));
    if (!o) return NULL;
    o->n = n;
    o->s = s;
    o->L = 0;
    while ((1 << o->L) < s) o->L++;
    o->nb = 0;
    while (((int64_t)1 << o->nb) < n) o->nb++;
    o->w = 16;
    o->ns = (int64_t)n * s;
    o->val_base = 0;
    o->col_base = o->ns;
    o->tau = tau;
    o->mem = (uint32_t *)calloc((size_t)(2 * o->ns), sizeof(uint32_t));
    int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * (size_t)s);
    int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * (size_t)s);
    uint16_t *vals = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)s);
    char *used = (char *)calloc((size_t)n, 1);
    if (!o->mem || !cols || !vals || !used || !ord) goto fail;
    for (int32_t j = 0; j < n; ++j) {
        int32_t lo = colptr[j], hi = colptr[j + 1];
        int32_t r = hi - lo;
        if (r > s) goto fail;
        /* column j of a symmetric matrix is row j */
        for (int32_t t = 0; t < r; ++t) {
            cols[t] = rowidx[lo + t];
            vals[t] = (uint16_t)val_q15[lo + t];
            used[cols[t]] = 1;
        }
        /* pad with explicit zeros at free columns j+1, j+2, ... (cyclic) */
        int32_t c = j;
        for (int32_t t = r; t < s; ++t) {
            do { c = (c + 1) % n; } while (used[c]);
            cols[t] = c;
            vals[t] = 0;
            used[c] = 1;
        }
        /* sort the row's (column, value) pairs by column */
        for (int32_t t = 0; t < s; ++t) ord[t] = cols[t];
        qsort(ord, (size_t)s, sizeof(int32_t), cmp_i32);
        for (int32_t t = 0; t < s; ++t) {
            int32_t col = ord[t];
            uint16_t val = 0;
            for (int32_t q = 0; q < s; ++q)
                if (cols[q] == col) val = vals[q];
            o->mem[o->val_base + (int64_t)j * s + t] = val;
            o->mem[o->col_base + (int64_t)j * s + t] = (uint32_t)col;
        }
        for (int32_t t = 0; t < s; ++t) used[cols[t]] = 0;
    }
    free(cols);
    free(ord);
    free(vals);
    free(used);
    for (int r = 0; r < NREG; ++r) o->meta[r].live = 0;
    int widths[NREG] = {(int)o->nb, (int)o->nb, 1, (int)o->nb, (int)o->nb, 1, (int)o->w};
    for (int r = 0; r < R_A; ++r) {
        o->meta[r].width = widths[r];
        o->meta[r].live = 1;
        o->live_bits += widths[r];
    }
    o->meta[R_A].width = widths[R_A];
    o->max_live_bits = o->live_bits;
    return o;
fail:
    free(cols);
    free(ord);
    free(vals);
    free(used);
    free(o->mem);
    free(o);
    return NULL;
}

void or_destroy(oracle *o)
{
    if (!o) return;
    free(o->mem);
    free(o->st);
    free(o->g);
    free(o);
}

int64_t or_nb(const oracle *o) { return o->nb; }
int64_t or_size(const oracle *o) { return o->m; }
int64_t or_violations(const oracle *o) { return o->violations; }
int64_t or_max_live_bits(const oracle *o) { return o->max_live_bits; }
void or_set_tau(oracle *o, double tau) { o->tau = tau; }
void or_set_rot_bits(oracle *o, int bits) { o->rot_bits = bits; }

/* QRAM image readback (value word, column word) of row j, slot l. */
void or_image(const oracle *o, int64_t j, int64_t l, uint32_t *val, uint32_t *col)
{
    *val = (uint32_t)qram(o, (uint64_t)(o->val_base + j * o->s + l), o->val_base);
    *col = (uint32_t)qram(o, (uint64_t)(o->col_base + j * o->s + l), o->col_base);
}

/* |b~> = sum_j b_j |0, j, 0, 0, 0, 0> (exact zeros are not stored). */
int or_init_b(oracle *o, const double *b_re, const double *b_im)
{
    free(o->g);
    o->g = NULL;
    o->gm = 0;
    o->m = 0;
    if (reserve(o, o->n)) return -1;
    for (int64_t j = 0; j < o->n; ++j) {
        double complex a = b_re[j] + I * (b_im ? b_im[j] : 0.0);
        if (a == 0) continue;
        branch e;
        memset(&e, 0, sizeof e);
        e.r[R_J] = (uint64_t)j;
        e.a = a;
        o->st[o->m++] = e;
    }
    return 0;
}

/* Replace the state: regs is m x 6 (jc, j, b1, kc, k, b2), amps m x 2. */
int or_import(oracle *o, const uint64_t *regs, const double *amps, int64_t m)
{
    free(o->g);
    o->g = NULL;
    o->gm = 0;
    if (reserve(o, m)) return -1;
    for (int64_t i = 0; i < m; ++i) {
        branch e;
        memset(&e, 0, sizeof e);
        for (int r = 0; r < 6; ++r) e.r[r] = regs[i * 6 + r];
        e.a = amps[2 * i] + I * amps[2 * i + 1];
        o->st[i] = e;
    }
    o->m = m;
    return 0;
}

/* Export: regs m x 7 (jc, j, b1, kc, k, b2, A), amps m x 2. */
int64_t or_export(const oracle *o, uint64_t *regs, double *amps, int64_t cap)
{
    int64_t m = o->m < cap ? o->m : cap;
    for (int64_t i = 0; i < m; ++i) {
        for (int r = 0; r < NREG; ++r) regs[i * NREG + r] = o->st[i].r[r];
        amps[2 * i] = creal(o->st[i].a);
        amps[2 * i + 1] = cimag(o->st[i].a);
    }
    return o->m;
}

int or_apply(oracle *o, int op)
{
    g_check_free(o); /* the whole ops need the working registers idle */
    switch (op) {
    case OR_T: return op_t(o);
    case OR_TDAG: return op_tdag(o);
    case OR_W: return op_w(o);
    case OR_P: for_each(o, p_branch); return 0;
    case OR_S: for_each(o, s_branch); return 0;
    case OR_H: return op_h(o);
    case OR_R: return op_r(o);
    case OR_RDAG: return op_rdag(o);
    case OR_OA: for_each(o, oa_branch); return 0;
    case OR_OS: op_os(o); return 0;
    case OR_OSDAG: op_osdag(o); return 0;
    case OR_ALLOC_A: reg_alloc(o, R_A, (int)o->w); return 0;
    case OR_FREE_A: reg_free(o, R_A); return 0;
    default: return -1;
    }
}

/* Flag-0 block: y[j] = amplitude of |0, j, 0, 0, 0, 0> for j < N (Sec. V-B). */
void or_flag0(const oracle *o, double *y)
{
    memset(y, 0, sizeof(double) * 2 * (size_t)o->n);
    for (int64_t i = 0; i < o->m; ++i) {
        const branch *e = &o->st[i];
        if (e->r[R_JC] || e->r[R_B1] || e->r[R_KC] || e->r[R_K] || e->r[R_B2] || e->r[R_A]) continue;
        if ((int64_t)e->r[R_J] >= o->n) continue;
        y[2 * e->r[R_J]] = creal(e->a);
        y[2 * e->r[R_J] + 1] = cimag(e->a);
    }
}

/* Marginal distribution of register `reg` (0..5 = jc, j, b1, kc, k, b2). */
int or_marginal(const oracle *o, int reg, double *probs, int64_t len)
{
    if (reg < 0 || reg >= NREG) return -1;
    memset(probs, 0, sizeof(double) * (size_t)len);
    for (int64_t i = 0; i < o->m; ++i) {
        uint64_t v = o->st[i].r[reg];
        if ((int64_t)v < len) probs[v] += creal(o->st[i].a) * creal(o->st[i].a) +
                                          cimag(o->st[i].a) * cimag(o->st[i].a);
    }
    return 0;
}

double or_norm2(const oracle *o)
{
    double acc = 0;
    for (int64_t i = 0; i < o->m; ++i)
        acc += creal(o->st[i].a) * creal(o->st[i].a) + cimag(o->st[i].a) * cimag(o->st[i].a);
    return acc;
}

/* Single-branch probes used by the unit tests. */
uint64_t or_qbs(oracle *o, uint64_t j, uint64_t target)
{
    return qbs(o, (uint64_t)o->col_base + j * (uint64_t)o->s, target, 0);
}

void or_os_single(oracle *o, uint64_t j, uint64_t k, uint64_t kc, int dagger, uint64_t *k_out,
                  uint64_t *kc_out)
{
    branch e;
    memset(&e, 0, sizeof e);
    e.r[R_J] = j;
    e.r[R_K] = k;
    e.r[R_KC] = kc;
    if (dagger) osdag_branch(o, &e);
    else os_branch(o, &e);
    *k_out = e.r[R_K];
    *kc_out = e.r[R_KC];
}
