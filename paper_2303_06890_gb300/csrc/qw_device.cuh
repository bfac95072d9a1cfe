/*
 * qw_device.cuh -- device primitives shared by the step kernels (qw_kernels.cu)
 * and the flat, globally sorted step (qw_flat.cu): the row descriptor and the
 * register layouts, complex helpers, the pruning rule, warp primitives, the
 * QRAM read, the quantum binary search (Def. 1), O_s', O_s'^dag and O_A'
 * (Sec. III-B), the rotation values, and the bucket lookup of a row.
 * Everything is internal to each translation unit that includes it.
 */
#ifndef QW_DEVICE_CUH
#define QW_DEVICE_CUH

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
    const void *sfg; /* rotation values of the row's s slots (fused kernel), or null */
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

/* Compaction for per-lane emit flags c0, c1 in {0, 1}, emitted in lane
 * order as (c0 item, c1 item): the lane's first output position among the
 * warp's outputs, and the warp total, from two ballots. */
__device__ __forceinline__ int warp_compact2(bool c0, bool c1, int &total)
{
    const unsigned lt = (1u << lane_id()) - 1u;
    const unsigned b0 = __ballot_sync(FULL, c0), b1 = __ballot_sync(FULL, c1);
    total = __popc(b0) + __popc(b1);
    return __popc(b0 & lt) + __popc(b1 & lt);
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

/* Quantum binary search (Def. 1): the net effect of the reversible loop of
 * Alg. 1 after its uncomputation, i(t) = in-row index of t, 0 if absent.
 * A row j < N holds a sorted list of distinct columns, where a branch-free
 * lower-bound search finds the same index as the fixed ceil(log2 s)+1-probe
 * search with a floor midpoint.  A row j >= N reads the all-zero list, where
 * that fixed-probe search stops at its first midpoint s/2 when t = 0 and
 * finds nothing otherwise. */
__device__ __forceinline__ uint32_t qbs(const QwSimDev &d, const Row &r, uint32_t target)
{
    if (!r.valid) return target == 0 ? (uint32_t)(d.s >> 1) : 0u;
    uint32_t i = 0, ci = r.simg[0] >> 16; /* ci: the column at i */
    for (int step = d.s >> 1; step > 0; step >>= 1) {
        const uint32_t c = r.simg[i + step] >> 16;
        const bool up = c <= target;
        i = up ? i + (uint32_t)step : i;
        ci = up ? c : ci;
    }
    return ci == target ? i : 0u;
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
        const int64_t lo = d.ninst == 1 ? 0 : d.inst_bkt[inst];
        const int64_t hi = d.ninst == 1 ? d.dense_buckets : d.inst_bkt[inst + 1];
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

/* S sends a branch to another partition: append to that partition's segment
 * of the outbox (FP64 amplitude); false and a status bit when it is full */
__device__ __forceinline__ void part_send(const QwSimDev &d, int dest, uint64_t rowkey, uint64_t local, double2 a,
                                          int32_t *status)
{
    const unsigned long long p = atomicAdd(d.outbox_count + dest, 1ull);
    if ((int64_t)p >= d.outbox_cap) {
        atomicOr(status, QW_ST_OUTBOX_FULL);
        return;
    }
    QwPartEntry e;
    e.rowkey = rowkey;
    e.local = local;
    e.re = a.x;
    e.im = a.y;
    d.outbox[(int64_t)dest * d.outbox_cap + (int64_t)p] = e;
}

__device__ bool row_of(const QwSimDev &d, const QwBufDev &in, int64_t b, Row &r)
{
    if (d.ninst == 1) { /* one instance: everything from the kernel parameters */
        if (b < d.dense_buckets) {
            r.inst = 0;
            r.jc = 0;
            r.j = (uint32_t)(b >> 1);
            r.b1 = (uint32_t)(b & 1);
        } else {
            const uint64_t rk = in.spill[b - d.dense_buckets];
            if (rk == QW_SPILL_EMPTY) return false;
            r.inst = (uint32_t)(rk >> 40);
            r.jc = (uint32_t)((rk >> 20) & 0xfffffu);
            r.j = (uint32_t)((rk >> 1) & 0x7ffffu);
            r.b1 = (uint32_t)(rk & 1);
        }
        r.n_inst = (uint32_t)d.n_single;
        r.img_base = 0;
        r.valid = r.j < r.n_inst;
        return true;
    }
    if (b < d.dense_buckets) {
        const int lo = d.unit_inst[b >> 1];
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

} // namespace

#endif /* QW_DEVICE_CUH */
