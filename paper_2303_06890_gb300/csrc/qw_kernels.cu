/*
 * qw_kernels.cu -- sm_103a kernels of the sparse-state quantum walk.
 *
 * One walk step W = S T~ P T~^dag (Alg. "Quantum walk operator") is one launch
 * of k_step.  T~^dag, P and T~ never change the registers (jc, j, b1) and every
 * QRAM read they make (O_A', O_s', QBS) indexes row j, so each (jc, j, b1) row
 * of the state evolves independently until S.  One warp takes one row: it
 * loads the row's branches into its slice of shared memory together with the
 * row's s QRAM words, runs the whole T~^dag P T~ on chip -- the per-branch
 * register maps (semi-quantum ops, Sec. V-A), and the interference ops R^dag,
 * H P H and R as sort + per-group transform + pruning (Sec. V-A, interference
 * paragraph) -- then applies S and appends every branch to the bucket of its
 * new row with one atomic per branch.  The HBM traffic of a step is one read
 * and one write of the state.
 *
 * Arithmetic: register maps are exact integer work; amplitudes are combined in
 * FP64 whatever the storage type; the prune decision |a|^2 <= tau^2 is taken
 * with un-fused FP64 multiplies and adds.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include "qw_internal.h"

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int WARPS = 8; /* warps per block of the step kernel */

struct Row {
    uint32_t inst, jc, j, b1;
    uint32_t n_inst;
    int64_t img_base;
    bool valid; /* j < N: the row has a QRAM image */
    const uint32_t *simg;
};

struct Regs {
    uint32_t k, kc, A, b2;
};

/* ---- complex helpers (FP64) ------------------------------------------------ */

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cneg(double2 a) { return make_double2(-a.x, -a.y); }

/* clearing step of an interference op: keep a branch iff |a|^2 > tau^2 */
__device__ __forceinline__ bool keep(double2 a, double tau2)
{
    return __dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y)) > tau2;
}

template <typename T> __device__ __forceinline__ double2 load_amp(const void *p, int64_t i);
template <> __device__ __forceinline__ double2 load_amp<double2>(const void *p, int64_t i)
{
    return static_cast<const double2 *>(p)[i];
}
template <> __device__ __forceinline__ double2 load_amp<float2>(const void *p, int64_t i)
{
    float2 v = static_cast<const float2 *>(p)[i];
    return make_double2((double)v.x, (double)v.y);
}
template <typename T> __device__ __forceinline__ double store_amp(void *p, int64_t i, double2 a);
template <> __device__ __forceinline__ double store_amp<double2>(void *p, int64_t i, double2 a)
{
    static_cast<double2 *>(p)[i] = a;
    return a.x * a.x + a.y * a.y;
}
template <> __device__ __forceinline__ double store_amp<float2>(void *p, int64_t i, double2 a)
{
    float2 v = make_float2((float)a.x, (float)a.y);
    static_cast<float2 *>(p)[i] = v;
    return (double)v.x * (double)v.x + (double)v.y * (double)v.y;
}

/* ---- warp primitives ---------------------------------------------------------- */

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ int warp_excl_scan(int v, int &total)
{
    const int lane = lane_id();
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    total = __shfl_sync(FULL, x, 31);
    return x - v;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

/* Grouping step of an interference op: sort the row's n branches by key.
 * Keys are distinct (every register map is a bijection and every
 * interference op emits one branch per key), so the rank of a key -- the
 * number of smaller keys -- is its position. */
__device__ void warp_sort(const uint64_t *ks, const double2 *as, int n, uint64_t *kd, double2 *ad)
{
    for (int i = lane_id(); i < n; i += 32) {
        const uint64_t ki = ks[i];
        int r = 0;
        for (int t = 0; t < n; ++t) r += (ks[t] < ki);
        kd[r] = ki;
        ad[r] = as[i];
    }
    __syncwarp();
}

/* ---- register layouts --------------------------------------------------------- */

__device__ __forceinline__ Regs decode_r(uint64_t key, int nb)
{
    const uint64_t m = (1ull << nb) - 1;
    Regs x;
    x.b2 = (uint32_t)(key & 1);
    x.k = (uint32_t)((key >> 1) & m);
    x.kc = (uint32_t)((key >> (1 + nb)) & m);
    x.A = (uint32_t)((key >> (1 + 2 * nb)) & 0xffffu);
    return x;
}

__device__ __forceinline__ uint64_t encode_r(const Regs &x, int nb)
{
    return (uint64_t)x.b2 | ((uint64_t)x.k << 1) | ((uint64_t)x.kc << (1 + nb)) |
           ((uint64_t)x.A << (1 + 2 * nb));
}

__device__ __forceinline__ Regs decode_h(uint64_t key, int nb, int L)
{
    const uint64_t m = (1ull << nb) - 1;
    Regs x;
    const uint32_t klow = (uint32_t)(key & ((1ull << L) - 1));
    x.b2 = (uint32_t)((key >> L) & 1);
    const uint32_t khigh = (uint32_t)((key >> (L + 1)) & ((1ull << (nb - L)) - 1));
    x.k = (khigh << L) | klow;
    x.kc = (uint32_t)((key >> (1 + nb)) & m);
    x.A = (uint32_t)((key >> (1 + 2 * nb)) & 0xffffu);
    return x;
}

__device__ __forceinline__ uint64_t encode_h(const Regs &x, int nb, int L)
{
    const uint64_t klow = x.k & ((1u << L) - 1), khigh = x.k >> L;
    return klow | ((uint64_t)x.b2 << L) | (khigh << (L + 1)) | ((uint64_t)x.kc << (1 + nb)) |
           ((uint64_t)x.A << (1 + 2 * nb));
}

/* ---- QRAM and the register maps (semi-quantum operations) --------------------- */

/* QRAM word of row r.j, slot l: (column << 16) | value, 0 outside [0, N s).
 * Slots l < s of a row j < N come from the staged copy in shared memory. */
__device__ __forceinline__ uint32_t qword(const QwSimDev &d, const Row &r, uint32_t l)
{
    if (l < (uint32_t)d.s) return r.valid ? r.simg[l] : 0u;
    const uint64_t addr = (uint64_t)r.j * (uint64_t)d.s + l;
    if (addr < (uint64_t)r.n_inst * (uint64_t)d.s) return __ldg(d.img + r.img_base + addr);
    return 0u;
}

/* Quantum binary search (Def. 1), net effect of the reversible loop of
 * Alg. 1 after its uncomputation: ceil(log2 s)+1 probes with a floor midpoint
 * over [0, s), stop at the first equal column, in-row index or 0. */
__device__ __forceinline__ uint32_t qbs(const QwSimDev &d, const Row &r, uint32_t target)
{
    uint32_t lo = 0, hi = (uint32_t)d.s, found = 0;
    bool done = false;
    for (int it = 0; it <= d.L; ++it) {
        if (!done) {
            const uint32_t mid = (lo + hi) >> 1;
            const uint32_t v = r.valid ? (r.simg[mid] >> 16) : 0u;
            if (v == target) {
                found = mid;
                done = true;
            } else if (v < target) {
                lo = mid;
            } else {
                hi = mid;
            }
        }
    }
    return found;
}

/* O_A': A ^= a_{j,k}, controlled by jc = kc = 0 (Sec. III-B). */
__device__ __forceinline__ void op_oa(const QwSimDev &d, const Row &r, Regs &x)
{
    if (r.jc == 0 && x.kc == 0) x.A ^= (qword(d, r, x.k) & 0xffffu);
}

/* O_s' (Eq. "Newprocess"): kc ^= K(j, k); k ^= I(j, kc); swap(k, kc). */
__device__ __forceinline__ void op_os(const QwSimDev &d, const Row &r, Regs &x)
{
    x.kc ^= qword(d, r, x.k) >> 16;
    x.k ^= qbs(d, r, x.kc);
    const uint32_t t = x.k;
    x.k = x.kc;
    x.kc = t;
}

/* O_s'^dag: the three steps of O_s' in reverse. */
__device__ __forceinline__ void op_osdag(const QwSimDev &d, const Row &r, Regs &x)
{
    const uint32_t t = x.k;
    x.k = x.kc;
    x.kc = t;
    x.k ^= qbs(d, r, x.kc);
    x.kc ^= qword(d, r, x.k) >> 16;
}

/* ---- interference operations on one row ---------------------------------------- */

/* f, g of the conditional rotation on b2 (Alg. T~ and the footnote of Sec. IV):
 * g = sqrt(1-|a|); f = sqrt(a) for a >= 0, i sigma sqrt|a| for a < 0 with
 * sigma = +1 if j <= k else -1.  sqrt values come from a per-code table that
 * the host filled with IEEE-rounded square roots. */
__device__ __forceinline__ void rot_fg(const QwSimDev &d, uint32_t A, uint32_t j, uint32_t k,
                                       double2 &f, double &g)
{
    const double2 t = __ldg(d.fg + A);
    g = t.y;
    const int16_t q = (int16_t)(uint16_t)A;
    if (q >= 0) f = make_double2(t.x, 0.0);
    else f = make_double2(0.0, (j <= k) ? t.x : -t.x);
}

/* R (DAG = false) or R^dag on b2: groups are branch pairs differing in b2,
 * adjacent in the sorted R layout.  R = [[f, -g], [g, conj f]]. */
template <bool DAG>
__device__ int rot_op(const QwSimDev &d, const Row &r, const uint64_t *ks, const double2 *as, int n,
                      uint64_t *kd, double2 *ad, int cap, int32_t *status)
{
    const int lane = lane_id();
    int out = 0;
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        const bool valid = i < n;
        const uint64_t k = valid ? ks[i] : 0;
        const bool head = valid && (i == 0 || (ks[i - 1] >> 1) != (k >> 1));
        double2 o0 = make_double2(0, 0), o1 = make_double2(0, 0);
        bool c0 = false, c1 = false;
        if (head) {
            double2 a0 = make_double2(0, 0), a1 = make_double2(0, 0);
            if ((k & 1) == 0) {
                a0 = as[i];
                if (i + 1 < n && (ks[i + 1] >> 1) == (k >> 1)) a1 = as[i + 1];
            } else {
                a1 = as[i];
            }
            const Regs x = decode_r(k, d.nb);
            double2 f;
            double g;
            rot_fg(d, x.A, r.j, x.k, f, g);
            if (!DAG) {
                o0 = csub(cmul(f, a0), cscale(g, a1));
                o1 = cadd(cscale(g, a0), cmul(cconj(f), a1));
            } else {
                o0 = cadd(cmul(cconj(f), a0), cscale(g, a1));
                o1 = csub(cmul(f, a1), cscale(g, a0));
            }
            c0 = keep(o0, d.tau2);
            c1 = keep(o1, d.tau2);
        }
        int total;
        int pos = out + warp_excl_scan((int)c0 + (int)c1, total);
        if (head) {
            const uint64_t k0 = k & ~1ull;
            if (c0) {
                if (pos < cap) { kd[pos] = k0; ad[pos] = o0; }
                pos++;
            }
            if (c1) {
                if (pos < cap) { kd[pos] = k0 | 1ull; ad[pos] = o1; }
                pos++;
            }
        }
        out += total;
    }
    __syncwarp();
    if (out > cap) {
        if (lane == 0) atomicOr(status, QW_ST_WARP_OVERFLOW);
        out = cap;
    }
    return out;
}

/* H P H of one walk step as one op (input sorted in the H layout).  Per
 * Hadamard group (all registers equal except the low L bits of k): P keeps
 * the sign of the all-zero branch (b1 = k = b2 = jc = kc = 0) and flips the
 * rest, so on a group whose other registers are zero H P H = 2|+><+| - 1,
 * i.e. a_u -> (2/s) sum_v a_v - a_u for all s values of u, and on every other
 * group H P H = -1.  Optionally reads the flag-0 amplitude of T~^dag's output,
 * (1/sqrt s) sum_v a_v of the group whose key is 0, into the QLS accumulator. */
__device__ int reflect_op(const QwSimDev &d, const Row &r, const uint64_t *ks, const double2 *as,
                          int n, uint64_t *kd, double2 *ad, int cap, int32_t *status,
                          const QwStepArgs &a)
{
    const int lane = lane_id();
    const int L = d.L, s = d.s;
    const bool rowzero = (r.jc == 0 && r.b1 == 0);
    const uint64_t zmask = (1ull << (1 + 2 * d.nb - L)) - 1; /* b2, k_high, kc */
    const uint64_t umask = (uint64_t)s - 1;
    int out = 0;
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        const bool valid = i < n;
        const uint64_t k = valid ? ks[i] : 0;
        const uint64_t g = k >> L;
        const bool zt = valid && rowzero && ((g & zmask) == 0);
        const bool head = valid && (i == 0 || (ks[i - 1] >> L) != g);
        int cnt = 0;
        double2 sum = make_double2(0, 0);
        int gend = i;
        if (valid && !zt) cnt = keep(as[i], d.tau2) ? 1 : 0;
        if (zt && head) {
            while (gend < n && (ks[gend] >> L) == g) {
                sum = cadd(sum, as[gend]);
                gend++;
            }
            int m = i;
            for (int u = 0; u < s; ++u) {
                double2 au = make_double2(0, 0);
                if (m < gend && (ks[m] & umask) == (uint64_t)u) au = as[m++];
                cnt += keep(csub(cscale(d.two_over_s, sum), au), d.tau2) ? 1 : 0;
            }
            if (g == 0 && a.qls_readout && r.valid) {
                const double2 y = cscale(d.inv_sqrt_s, sum);
                double2 acc = a.qls_y[r.j];
                acc.x += a.qls_coef * y.x;
                acc.y += a.qls_coef * y.y;
                a.qls_y[r.j] = acc;
            }
        }
        int total;
        int pos = out + warp_excl_scan(cnt, total);
        if (valid && !zt && cnt) {
            if (pos < cap) { kd[pos] = k; ad[pos] = cneg(as[i]); }
        }
        if (zt && head) {
            int m = i;
            for (int u = 0; u < s; ++u) {
                double2 au = make_double2(0, 0);
                if (m < gend && (ks[m] & umask) == (uint64_t)u) au = as[m++];
                const double2 o = csub(cscale(d.two_over_s, sum), au);
                if (keep(o, d.tau2)) {
                    if (pos < cap) { kd[pos] = (g << L) | (uint64_t)u; ad[pos] = o; }
                    pos++;
                }
            }
        }
        out += total;
    }
    __syncwarp();
    if (out > cap) {
        if (lane == 0) atomicOr(status, QW_ST_WARP_OVERFLOW);
        out = cap;
    }
    return out;
}

/* Hadamard on the low L bits of k as a plain interference op (input sorted in
 * the H layout): each group emits the s outputs (1/sqrt s) sum_v (-1)^{u.v} a_v.
 * With readout set, the u = 0 output of the group whose key is 0 (the flag-0
 * amplitude) is added into the QLS accumulator. */
__device__ int hadamard_op(const QwSimDev &d, const Row &r, const uint64_t *ks, const double2 *as,
                           int n, uint64_t *kd, double2 *ad, int cap, int32_t *status,
                           const QwStepArgs &a, bool readout)
{
    const int lane = lane_id();
    const int L = d.L, s = d.s;
    const uint64_t umask = (uint64_t)s - 1;
    int out = 0;
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        const bool valid = i < n;
        const uint64_t k = valid ? ks[i] : 0;
        const uint64_t g = k >> L;
        const bool head = valid && (i == 0 || (ks[i - 1] >> L) != g);
        int gend = i;
        int cnt = 0;
        if (head) {
            while (gend < n && (ks[gend] >> L) == g) gend++;
            for (int u = 0; u < s; ++u) {
                double2 o = make_double2(0, 0);
                for (int m = i; m < gend; ++m) {
                    const double2 v = as[m];
                    o = (__popcll((uint64_t)u & (ks[m] & umask)) & 1) ? csub(o, v) : cadd(o, v);
                }
                o = cscale(d.inv_sqrt_s, o);
                cnt += keep(o, d.tau2) ? 1 : 0;
                if (u == 0 && g == 0 && readout && a.qls_readout && r.valid && r.jc == 0 &&
                    r.b1 == 0) {
                    double2 acc = a.qls_y[r.j];
                    acc.x += a.qls_coef * o.x;
                    acc.y += a.qls_coef * o.y;
                    a.qls_y[r.j] = acc;
                }
            }
        }
        int total;
        int pos = out + warp_excl_scan(cnt, total);
        if (head) {
            for (int u = 0; u < s; ++u) {
                double2 o = make_double2(0, 0);
                for (int m = i; m < gend; ++m) {
                    const double2 v = as[m];
                    o = (__popcll((uint64_t)u & (ks[m] & umask)) & 1) ? csub(o, v) : cadd(o, v);
                }
                o = cscale(d.inv_sqrt_s, o);
                if (keep(o, d.tau2)) {
                    if (pos < cap) { kd[pos] = (g << L) | (uint64_t)u; ad[pos] = o; }
                    pos++;
                }
            }
        }
        out += total;
    }
    __syncwarp();
    if (out > cap) {
        if (lane == 0) atomicOr(status, QW_ST_WARP_OVERFLOW);
        out = cap;
    }
    return out;
}

/* P of the walk (Eq. (impl)), in place on H-layout keys: the sign flips unless
 * b1, k, b2, jc and kc are all zero. */
__device__ void phase_op(const QwSimDev &d, const Row &r, const uint64_t *ks, double2 *as, int n)
{
    for (int i = lane_id(); i < n; i += 32) {
        const Regs x = decode_h(ks[i], d.nb, d.L);
        const bool zero = r.b1 == 0 && x.k == 0 && x.b2 == 0 && r.jc == 0 && x.kc == 0;
        if (!zero) as[i] = cneg(as[i]);
    }
    __syncwarp();
}

/* ---- buckets ---------------------------------------------------------------------- */

__device__ __forceinline__ uint32_t hash_rowkey(uint64_t x)
{
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return (uint32_t)x;
}

__device__ int64_t bucket_of(const QwSimDev &d, const QwBufDev &out, uint32_t inst, uint32_t jc,
                             uint32_t j, uint32_t b1, int32_t *status)
{
    if (jc == 0) {
        const int64_t lo = d.inst_bkt[inst], hi = d.inst_bkt[inst + 1];
        const int64_t b = lo + (((int64_t)j << 1) | (int64_t)b1);
        if (b < hi) return b;
        atomicOr(status, QW_ST_SPILL_FULL);
        return -1;
    }
    const uint64_t rk = qw_rowkey(inst, jc, j, b1);
    uint32_t h = hash_rowkey(rk) & (uint32_t)(d.spill_slots - 1);
    for (int t = 0; t < d.spill_slots; ++t) {
        const unsigned long long prev =
            atomicCAS(reinterpret_cast<unsigned long long *>(out.spill + h), QW_SPILL_EMPTY,
                      (unsigned long long)rk);
        if (prev == QW_SPILL_EMPTY || prev == rk) return d.dense_buckets + h;
        h = (h + 1) & (uint32_t)(d.spill_slots - 1);
    }
    atomicOr(status, QW_ST_SPILL_FULL);
    return -1;
}

__device__ bool row_of(const QwSimDev &d, const QwBufDev &in, int64_t b, Row &r)
{
    if (b < d.dense_buckets) {
        int lo = 0, hi = d.ninst;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (d.inst_bkt[mid] <= b) lo = mid;
            else hi = mid;
        }
        const int64_t idx = b - d.inst_bkt[lo];
        r.inst = (uint32_t)lo;
        r.jc = 0;
        r.j = (uint32_t)(idx >> 1);
        r.b1 = (uint32_t)(idx & 1);
    } else {
        const uint64_t rk = in.spill[b - d.dense_buckets];
        if (rk == QW_SPILL_EMPTY) return false;
        r.inst = (uint32_t)(rk >> 40);
        r.jc = (uint32_t)((rk >> 20) & 0xfffffu);
        r.j = (uint32_t)((rk >> 1) & 0x7ffffu);
        r.b1 = (uint32_t)(rk & 1);
    }
    r.n_inst = (uint32_t)d.inst_n[r.inst];
    r.img_base = d.inst_img[r.inst];
    r.valid = r.j < r.n_inst;
    return true;
}

/* Final register maps of T~ (O_s'^dag, O_A', O_s'), then S for a walk step,
 * and the append of each branch to the bucket of its row. */
template <typename AmpT>
__device__ double emit_row(const QwSimDev &d, const Row &r, const uint64_t *ks, const double2 *as,
                           int n, const QwBufDev &out, bool swap_rows, int32_t *status)
{
    double nrm = 0.0;
    for (int i = lane_id(); i < n; i += 32) {
        Regs x = decode_r(ks[i], d.nb);
        op_osdag(d, r, x);
        op_oa(d, r, x);
        op_os(d, r, x);
        if (x.A != 0) atomicOr(status, QW_ST_ANCILLA);
        uint32_t njc = r.jc, nj = r.j, nb1 = r.b1;
        Regs y = x;
        if (swap_rows) { /* S: (jc, j, b1) <-> (kc, k, b2) */
            njc = x.kc;
            nj = x.k;
            nb1 = x.b2;
            y.kc = r.jc;
            y.k = r.j;
            y.b2 = r.b1;
        }
        const int64_t b = bucket_of(d, out, r.inst, njc, nj, nb1, status);
        if (b < 0) continue;
        const int pos = atomicAdd(out.count + b, 1);
        if (pos >= d.cap_row) {
            atomicOr(status, QW_ST_ROW_OVERFLOW);
            continue;
        }
        const int64_t slot = b * (int64_t)d.cap_row + pos;
        out.key[slot] = encode_r(y, d.nb);
        nrm += store_amp<AmpT>(out.amp, slot, as[i]);
    }
    return nrm;
}

/* in-place register maps on a row buffer */
template <int CHAIN>
__device__ void chain(const QwSimDev &d, const Row &r, uint64_t *ks, int n)
{
    for (int i = lane_id(); i < n; i += 32) {
        if (CHAIN == 1) { /* start of T~^dag: O_s'^dag, O_A', O_s' (R layout) */
            Regs x = decode_r(ks[i], d.nb);
            op_osdag(d, r, x);
            op_oa(d, r, x);
            op_os(d, r, x);
            ks[i] = encode_r(x, d.nb);
        } else if (CHAIN == 2) { /* after R^dag: O_s'^dag, O_A' (R -> H layout) */
            Regs x = decode_r(ks[i], d.nb);
            op_osdag(d, r, x);
            op_oa(d, r, x);
            ks[i] = encode_h(x, d.nb, d.L);
        } else if (CHAIN == 3) { /* after H of T~: O_A', O_s' (H -> R layout) */
            Regs x = decode_h(ks[i], d.nb, d.L);
            op_oa(d, r, x);
            op_os(d, r, x);
            ks[i] = encode_r(x, d.nb);
        } else { /* R -> H layout, no map (start of T~) */
            Regs x = decode_r(ks[i], d.nb);
            ks[i] = encode_h(x, d.nb, d.L);
        }
    }
    __syncwarp();
}

template <typename AmpT, int MODE>
__global__ void __launch_bounds__(WARPS * 32) k_step(QwSimDev d, QwBufDev in, QwBufDev out,
                                                     QwBufDev clr, QwStepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double block_part[WARPS];
    __shared__ int is_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int C = d.warp_cap;
    const size_t per_warp = (size_t)C * 2 * (sizeof(double2) + sizeof(uint64_t)) +
                            (((size_t)d.s * sizeof(uint32_t) + 15) & ~(size_t)15);
    unsigned char *base = smem + per_warp * warp;
    double2 *aP = reinterpret_cast<double2 *>(base);
    double2 *aQ = aP + C;
    uint64_t *kP = reinterpret_cast<uint64_t *>(aQ + C);
    uint64_t *kQ = kP + C;
    uint32_t *simg = reinterpret_cast<uint32_t *>(kQ + C);

    /* A step issued after a failed one does nothing, so the state of the last
       clean step (its input buffer, never written) survives for the host. */
    const bool skip = *(volatile int32_t *)a.status != 0;
    if (MODE != QW_MODE_T && !skip) { /* clear X_{t+2} for the step after this one */
        const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
        for (int64_t b = tid; b < d.total_buckets; b += nthr) clr.count[b] = 0;
        for (int64_t t = tid; t < d.spill_slots; t += nthr) clr.spill[t] = QW_SPILL_EMPTY;
    }

    const double scale = a.scale_in ? *a.scale_in : 1.0;
    const int64_t blo = (MODE == QW_MODE_T) ? a.bucket_lo : 0;
    const int64_t bhi = skip ? blo : ((MODE == QW_MODE_T) ? a.bucket_hi : d.total_buckets);
    double nrm = 0.0;
    unsigned long long st_rows = 0, st_in = 0, st_rdag = 0, st_h1 = 0, st_hph = 0, st_out = 0;

    for (int64_t b = blo + (int64_t)blockIdx.x * WARPS + warp; b < bhi;
         b += (int64_t)gridDim.x * WARPS) {
        int n = in.count[b];
        if (n <= 0) continue;
        if (n > d.cap_row) n = d.cap_row;
        Row r;
        if (!row_of(d, in, b, r)) continue;
        if (n > C) {
            if (lane == 0) atomicOr(a.status, QW_ST_WARP_OVERFLOW);
            continue;
        }
        r.simg = simg;
        for (int t = lane; t < d.s; t += 32)
            simg[t] = r.valid ? __ldg(d.img + r.img_base + (int64_t)r.j * d.s + t) : 0u;
        const int64_t row0 = b * (int64_t)d.cap_row;
        for (int i = lane; i < n; i += 32) {
            kP[i] = in.key[row0 + i];
            double2 v = load_amp<AmpT>(in.amp, row0 + i);
            if (a.scale_in) v = cscale(scale, v);
            aP[i] = v;
        }
        __syncwarp();
        if (MODE == QW_MODE_T) {
            if (lane == 0) in.count[b] = 0; /* T~ rewrites the row in place */
            __syncwarp();
            chain<4>(d, r, kP, n);
            warp_sort(kP, aP, n, kQ, aQ);
            n = hadamard_op(d, r, kQ, aQ, n, kP, aP, C, a.status, a, false);
            chain<3>(d, r, kP, n);
            warp_sort(kP, aP, n, kQ, aQ);
            n = rot_op<false>(d, r, kQ, aQ, n, kP, aP, C, a.status);
            nrm += emit_row<AmpT>(d, r, kP, aP, n, in, false, a.status);
            continue;
        }
        st_rows++;
        st_in += n;
        /* T~^dag */
        chain<1>(d, r, kP, n);
        warp_sort(kP, aP, n, kQ, aQ);
        n = rot_op<true>(d, r, kQ, aQ, n, kP, aP, C, a.status);
        st_rdag += n;
        chain<2>(d, r, kP, n);
        warp_sort(kP, aP, n, kQ, aQ);
        if (MODE == QW_MODE_WALK_FUSED) {
            /* H (end of T~^dag), P, H (start of T~) */
            n = reflect_op(d, r, kQ, aQ, n, kP, aP, C, a.status, a);
        } else {
            n = hadamard_op(d, r, kQ, aQ, n, kP, aP, C, a.status, a, true);
            st_h1 += n;
            phase_op(d, r, kP, aP, n);
            n = hadamard_op(d, r, kP, aP, n, kQ, aQ, C, a.status, a, false);
            for (int i = lane; i < n; i += 32) {
                kP[i] = kQ[i];
                aP[i] = aQ[i];
            }
            __syncwarp();
        }
        st_hph += n;
        /* rest of T~, then S */
        chain<3>(d, r, kP, n);
        warp_sort(kP, aP, n, kQ, aQ);
        n = rot_op<false>(d, r, kQ, aQ, n, kP, aP, C, a.status);
        st_out += n;
        nrm += emit_row<AmpT>(d, r, kP, aP, n, out, true, a.status);
    }
    if (a.stats && lane == 0 && st_rows) {
        atomicAdd(a.stats + QW_STAT_ROWS, st_rows);
        atomicAdd(a.stats + QW_STAT_IN, st_in);
        atomicAdd(a.stats + QW_STAT_RDAG, st_rdag);
        if (st_h1) atomicAdd(a.stats + QW_STAT_H1, st_h1);
        atomicAdd(a.stats + QW_STAT_HPH, st_hph);
        atomicAdd(a.stats + QW_STAT_OUT, st_out);
    }

    /* ||output||^2: block partial sums, reduced in block order by the last block */
    nrm = warp_sum(nrm);
    if (lane == 0) block_part[warp] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < WARPS; ++w) s += block_part[w];
        a.partials[blockIdx.x] = s;
        __threadfence();
        const unsigned prev = atomicAdd(a.done_ctr, 1u);
        is_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last && threadIdx.x == 0) {
        __threadfence();
        double tot = 0.0;
        for (unsigned bb = 0; bb < gridDim.x; ++bb) tot += __ldcg(a.partials + bb);
        const bool clean = *(volatile int32_t *)a.status == 0;
        if (clean) {
            *a.norm_out = tot;
            if (a.scale_out)
                *a.scale_out = (a.renorm && tot > 0.0) ? sqrt(*a.renorm_target / tot) : 1.0;
            if (a.steps_done) *a.steps_done += 1;
            if (a.stats && MODE != QW_MODE_T) a.stats[QW_STAT_STEPS] += 1;
        }
        *a.done_ctr = 0u;
    }
}

/* ---- small kernels ------------------------------------------------------------ */

__global__ void k_clear(QwBufDev buf, int64_t lo, int64_t hi, int spill_slots, int clear_spill)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = lo + tid; b < hi; b += nthr) buf.count[b] = 0;
    if (clear_spill)
        for (int64_t t = tid; t < spill_slots; t += nthr) buf.spill[t] = QW_SPILL_EMPTY;
}

/* |b~>: branch (jc=0, j, b1=0, kc=0, k=0, b2=0) with amplitude b_j, stored in
 * the units of the pending renormalisation scale (amplitude / scale). */
template <typename AmpT>
__global__ void k_init_b(QwSimDev d, QwBufDev buf, int inst, const double2 *bvec, int n,
                         const double *scale)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double2 v = bvec[j];
    if (v.x == 0.0 && v.y == 0.0) return;
    if (scale) v = make_double2(v.x / *scale, v.y / *scale);
    const int64_t b = d.inst_bkt[inst] + ((int64_t)j << 1);
    const int64_t slot = b * (int64_t)d.cap_row;
    buf.key[slot] = 0ull;
    store_amp<AmpT>(buf.amp, slot, v);
    buf.count[b] = 1;
}

/* Every branch of instance inst (-1: all) to flat (row key, local key, amp). */
template <typename AmpT>
__global__ void k_export(QwSimDev d, QwBufDev buf, int inst, const double *scale, uint64_t *rowkey,
                         uint64_t *local, double2 *amp, unsigned long long *counter, int64_t cap)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    const double sc = scale ? *scale : 1.0;
    for (int64_t b = warp; b < d.total_buckets; b += nw) {
        int n = buf.count[b];
        if (n <= 0) continue;
        if (n > d.cap_row) n = d.cap_row;
        Row r;
        if (!row_of(d, buf, b, r)) continue;
        if (inst >= 0 && r.inst != (uint32_t)inst) continue;
        const uint64_t rk = qw_rowkey(r.inst, r.jc, r.j, r.b1);
        for (int i = lane; i < n; i += 32) {
            const int64_t slot = b * (int64_t)d.cap_row + i;
            const unsigned long long p = atomicAdd(counter, 1ull);
            if ((int64_t)p >= cap) continue;
            rowkey[p] = rk;
            local[p] = buf.key[slot];
            double2 v = load_amp<AmpT>(buf.amp, slot);
            if (scale) v = cscale(sc, v);
            amp[p] = v;
        }
    }
}

template <typename AmpT>
__global__ void k_measure(QwSimDev d, QwBufDev buf, int inst, const double *scale, int reg,
                          double *probs, int64_t len)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    const double sc = scale ? *scale : 1.0;
    for (int64_t b = warp; b < d.total_buckets; b += nw) {
        int n = buf.count[b];
        if (n <= 0) continue;
        if (n > d.cap_row) n = d.cap_row;
        Row r;
        if (!row_of(d, buf, b, r)) continue;
        if (r.inst != (uint32_t)inst) continue;
        for (int i = lane; i < n; i += 32) {
            const int64_t slot = b * (int64_t)d.cap_row + i;
            const Regs x = decode_r(buf.key[slot], d.nb);
            uint64_t v;
            switch (reg) {
            case 0: v = r.jc; break;
            case 1: v = r.j; break;
            case 2: v = r.b1; break;
            case 3: v = x.kc; break;
            case 4: v = x.k; break;
            default: v = x.b2; break;
            }
            if ((int64_t)v >= len) continue;
            double2 a = load_amp<AmpT>(buf.amp, slot);
            if (scale) a = cscale(sc, a);
            atomicAdd(probs + v, a.x * a.x + a.y * a.y);
        }
    }
}

__global__ void k_count(QwSimDev d, QwBufDev buf, int inst, unsigned long long *counter)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    unsigned long long c = 0;
    for (int64_t b = tid; b < d.total_buckets; b += nthr) {
        int n = buf.count[b];
        if (n <= 0) continue;
        if (n > d.cap_row) n = d.cap_row;
        if (inst >= 0) {
            Row r;
            if (!row_of(d, buf, b, r) || r.inst != (uint32_t)inst) continue;
        }
        c += (unsigned long long)n;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(counter, c);
}

__global__ void k_qls_norm(const double2 *y, int n, double *out)
{
    __shared__ double part[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += y[i].x * y[i].x + y[i].y * y[i].y;
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        *out = t;
    }
}

template <typename AmpT, int MODE> size_t step_smem(const QwSimDev &d)
{
    return (size_t)WARPS * ((size_t)d.warp_cap * 2 * (sizeof(double2) + sizeof(uint64_t)) +
                            (((size_t)d.s * sizeof(uint32_t) + 15) & ~(size_t)15));
}

template <typename AmpT, int MODE>
int step_grid_t(const QwSimDev &d)
{
    const size_t sm = step_smem<AmpT, MODE>(d);
    cudaFuncSetAttribute(k_step<AmpT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step<AmpT, MODE>, WARPS * 32, sm);
    if (per_sm < 1) per_sm = 1;
    int64_t want = (d.total_buckets + WARPS - 1) / WARPS;
    int64_t g = (int64_t)per_sm * qw_sm_count();
    if (want < g) g = want;
    return (int)(g < 1 ? 1 : g);
}

template <typename AmpT, int MODE>
cudaError_t launch_step_t(const QwSimDev &d, const QwBufDev &in, const QwBufDev &out,
                          const QwBufDev &clr, const QwStepArgs &a, int grid, cudaStream_t st)
{
    const size_t sm = step_smem<AmpT, MODE>(d);
    k_step<AmpT, MODE><<<grid, WARPS * 32, sm, st>>>(d, in, out, clr, a);
    return cudaGetLastError();
}

} // namespace

int qw_sm_count(void)
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n < 1) n = 1;
    }
    return n;
}

int qw_step_grid(const QwSimDev &d, int fp32, int mode)
{
    if (fp32) {
        if (mode == QW_MODE_WALK_FUSED) return step_grid_t<float2, QW_MODE_WALK_FUSED>(d);
        if (mode == QW_MODE_WALK_LITERAL) return step_grid_t<float2, QW_MODE_WALK_LITERAL>(d);
        return step_grid_t<float2, QW_MODE_T>(d);
    }
    if (mode == QW_MODE_WALK_FUSED) return step_grid_t<double2, QW_MODE_WALK_FUSED>(d);
    if (mode == QW_MODE_WALK_LITERAL) return step_grid_t<double2, QW_MODE_WALK_LITERAL>(d);
    return step_grid_t<double2, QW_MODE_T>(d);
}

cudaError_t qw_launch_step(const QwSimDev &d, const QwBufDev &in, const QwBufDev &out,
                           const QwBufDev &clr, const QwStepArgs &a, int fp32, int grid,
                           cudaStream_t st)
{
    if (fp32) {
        if (a.mode == QW_MODE_WALK_FUSED)
            return launch_step_t<float2, QW_MODE_WALK_FUSED>(d, in, out, clr, a, grid, st);
        if (a.mode == QW_MODE_WALK_LITERAL)
            return launch_step_t<float2, QW_MODE_WALK_LITERAL>(d, in, out, clr, a, grid, st);
        return launch_step_t<float2, QW_MODE_T>(d, in, out, clr, a, grid, st);
    }
    if (a.mode == QW_MODE_WALK_FUSED)
        return launch_step_t<double2, QW_MODE_WALK_FUSED>(d, in, out, clr, a, grid, st);
    if (a.mode == QW_MODE_WALK_LITERAL)
        return launch_step_t<double2, QW_MODE_WALK_LITERAL>(d, in, out, clr, a, grid, st);
    return launch_step_t<double2, QW_MODE_T>(d, in, out, clr, a, grid, st);
}

cudaError_t qw_launch_clear(const QwSimDev &d, const QwBufDev &buf, int64_t lo, int64_t hi,
                            int clear_spill, cudaStream_t st)
{
    int64_t work = hi - lo;
    if (clear_spill && d.spill_slots > work) work = d.spill_slots;
    int grid = (int)((work + 255) / 256);
    if (grid < 1) grid = 1;
    if (grid > 4 * qw_sm_count()) grid = 4 * qw_sm_count();
    k_clear<<<grid, 256, 0, st>>>(buf, lo, hi, d.spill_slots, clear_spill);
    return cudaGetLastError();
}

cudaError_t qw_launch_init_b(const QwSimDev &d, const QwBufDev &buf, int inst, const double2 *b,
                             int n, int fp32, const double *scale, cudaStream_t st)
{
    const int grid = (n + 255) / 256;
    if (fp32) k_init_b<float2><<<grid, 256, 0, st>>>(d, buf, inst, b, n, scale);
    else k_init_b<double2><<<grid, 256, 0, st>>>(d, buf, inst, b, n, scale);
    return cudaGetLastError();
}

cudaError_t qw_launch_export(const QwSimDev &d, const QwBufDev &buf, int inst, int fp32,
                             const double *scale, uint64_t *rowkey, uint64_t *local, double2 *amp,
                             unsigned long long *counter, int64_t cap, cudaStream_t st)
{
    const int grid = 4 * qw_sm_count();
    if (fp32)
        k_export<float2><<<grid, 256, 0, st>>>(d, buf, inst, scale, rowkey, local, amp, counter, cap);
    else
        k_export<double2><<<grid, 256, 0, st>>>(d, buf, inst, scale, rowkey, local, amp, counter, cap);
    return cudaGetLastError();
}

cudaError_t qw_launch_measure(const QwSimDev &d, const QwBufDev &buf, int inst, int fp32,
                              const double *scale, int reg, double *probs, int64_t len,
                              cudaStream_t st)
{
    const int grid = 4 * qw_sm_count();
    if (fp32) k_measure<float2><<<grid, 256, 0, st>>>(d, buf, inst, scale, reg, probs, len);
    else k_measure<double2><<<grid, 256, 0, st>>>(d, buf, inst, scale, reg, probs, len);
    return cudaGetLastError();
}

cudaError_t qw_launch_count(const QwSimDev &d, const QwBufDev &buf, int inst,
                            unsigned long long *counter, cudaStream_t st)
{
    const int grid = 4 * qw_sm_count();
    k_count<<<grid, 256, 0, st>>>(d, buf, inst, counter);
    return cudaGetLastError();
}

cudaError_t qw_launch_qls_norm(const double2 *y, int n, double *out, cudaStream_t st)
{
    k_qls_norm<<<1, 1024, 0, st>>>(y, n, out);
    return cudaGetLastError();
}
