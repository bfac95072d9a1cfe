/*
 * qw_flat.cu -- the walk step as the paper's simulator runs it, on one flat
 * list of branches in global memory (Sec. V-A): every register map applied to
 * every branch, and every interference operation as
 *   (1) grouping: a stable LSD radix sort of the whole list by all
 *       registers, with the target's bits moved below the others, so that
 *       the branches equal on every idle register are contiguous (8-bit
 *       digits over the bits that vary between keys, one single-pass
 *       kernel per digit carrying a permutation, the entries moved once);
 *   (2) computing: the small dense operator on each group's zero-filled
 *       vector (a thread per output; for H the groups are counted first, so
 *       that s outputs are formed per group, not per list entry);
 *   (3) clearing: outputs with |a| <= tau dropped by a stream compaction.
 * T~^dag, H, P, H, T~ and S run in the order of Alg. "Quantum walk operator",
 * with the element register A allocated for the whole step.  Nothing here is
 * bounded by the row buckets or the on-chip buffers of the step kernels, only
 * by device memory: this is the path of a step whose rows outgrow them, and a
 * schedule that can be selected on its own.  Amplitudes are complex FP64
 * whatever the storage precision (converted when the state is gathered and
 * rounded when it is stored back).
 *
 * Packed key of a branch (two 64-bit words, bit 0 first), the layout of
 * qw_state_export:  b2 | k (nb) | kc (nb) | b1 | j (nb) | jc (nb) | A (16) |
 * inst (16), 4 nb + 34 bits.
 */
#include <vector>

#include "qw_device.cuh"
#include "qw_sort_chunks.h"

namespace {

/* a packed register key of NW 64-bit words (2: the qw_state_export layout;
   10: the register-faithful layout, the working registers above bit 128) */
template <int NW> struct FKeyN {
    uint64_t w[NW];
};
typedef FKeyN<2> FKey;
constexpr int NW_FAITH = 10;
typedef FKeyN<NW_FAITH> FKeyW;

struct FLayout {
    int nb, pk, pkc, pb1, pj, pjc, pA, pinst;
};

__host__ __device__ inline FLayout flayout(int nb)
{
    FLayout f;
    f.nb = nb;
    f.pk = 1;
    f.pkc = 1 + nb;
    f.pb1 = 1 + 2 * nb;
    f.pj = 2 + 2 * nb;
    f.pjc = 2 + 3 * nb;
    f.pA = 2 + 4 * nb;
    f.pinst = 18 + 4 * nb;
    return f;
}

/* word i of a key by selection over its words, so that the key stays in
   registers whatever i is (an indexed access moves it to local memory) */
template <int NW>
__device__ __forceinline__ uint64_t fword(const FKeyN<NW> &k, int i)
{
    uint64_t v = k.w[0];
#pragma unroll
    for (int t = 1; t < NW; ++t) v = t == i ? k.w[t] : v;
    return v;
}

template <int NW>
__device__ __forceinline__ uint64_t fget(const FKeyN<NW> &k, int pos, int w)
{
    const int i = pos >> 6, o = pos & 63;
    uint64_t v = fword(k, i) >> o;
    if (o + w > 64 && i + 1 < NW) v |= fword(k, i + 1) << (64 - o);
    return v & (w >= 64 ? ~0ull : ((1ull << w) - 1ull));
}

/* OR v into a field (the field must be 0) */
template <int NW>
__device__ __forceinline__ void fput(FKeyN<NW> &k, int pos, int w, uint64_t v)
{
    v &= (w >= 64 ? ~0ull : ((1ull << w) - 1ull));
    const int i = pos >> 6, o = pos & 63;
#pragma unroll
    for (int t = 0; t < NW; ++t) {
        if (t == i) k.w[t] |= v << o;
        if (t == i + 1 && o + w > 64) k.w[t] |= v >> (64 - o);
    }
}

struct FRegs {
    uint32_t inst, jc, j, b1;
    Regs x; /* k, kc, A, b2 */
};

/* the base registers (4 nb + 34 bits) lie in words 0 and 1 of any key
   width: they are decoded from and encoded into those two words */
template <int NW>
__device__ __forceinline__ FKeyN<2> fbase(const FKeyN<NW> &k)
{
    FKeyN<2> b;
    b.w[0] = k.w[0];
    b.w[1] = k.w[1];
    return b;
}

/* words 0 and 1 of a key in global memory, as one 16-byte load */
template <int NW>
__device__ __forceinline__ FKeyN<2> fbase_load(const FKeyN<NW> *k)
{
    const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(k);
    FKeyN<2> b;
    b.w[0] = v.x;
    b.w[1] = v.y;
    return b;
}

template <int NW>
__device__ __forceinline__ FRegs fdecode(const FKeyN<NW> &key, const FLayout &L)
{
    const FKeyN<2> k = fbase(key);
    FRegs r;
    r.x.b2 = fget(k, 0, 1);
    r.x.k = fget(k, L.pk, L.nb);
    r.x.kc = fget(k, L.pkc, L.nb);
    r.b1 = fget(k, L.pb1, 1);
    r.j = fget(k, L.pj, L.nb);
    r.jc = fget(k, L.pjc, L.nb);
    r.x.A = fget(k, L.pA, 16);
    r.inst = fget(k, L.pinst, 16);
    return r;
}

/* the base registers into k (their fields must be 0) */
template <int NW>
__device__ __forceinline__ void fencode_into(FKeyN<NW> &key, const FRegs &r, const FLayout &L)
{
    FKeyN<2> k = fbase(key);
    fput(k, 0, 1, r.x.b2);
    fput(k, L.pk, L.nb, r.x.k);
    fput(k, L.pkc, L.nb, r.x.kc);
    fput(k, L.pb1, 1, r.b1);
    fput(k, L.pj, L.nb, r.j);
    fput(k, L.pjc, L.nb, r.jc);
    fput(k, L.pA, 16, r.x.A);
    fput(k, L.pinst, 16, r.inst);
    key.w[0] = k.w[0];
    key.w[1] = k.w[1];
}

/* the base registers of a wider key rewritten, its other bits kept */
template <int NW>
__device__ __forceinline__ void frewrite(FKeyN<NW> &k, const FRegs &r, const FLayout &L)
{
    const int bits = L.pinst + 16;
    k.w[0] &= bits >= 64 ? 0ull : ~((1ull << bits) - 1ull);
    if (bits > 64) k.w[1] &= bits >= 128 ? 0ull : ~((1ull << (bits - 64)) - 1ull);
    fencode_into(k, r, L);
}

/* The row descriptor of a branch, reading its QRAM row straight from the
 * image in global memory. */
__device__ __forceinline__ Row frow(const QwSimDev &d, const FRegs &f)
{
    Row r;
    r.inst = f.inst;
    r.jc = f.jc;
    r.j = f.j;
    r.b1 = f.b1;
    r.n_inst = d.ninst == 1 ? (uint32_t)d.n_single : (uint32_t)d.inst_n[f.inst];
    r.img_base = d.ninst == 1 ? 0 : d.inst_img[f.inst];
    r.valid = f.j < r.n_inst;
    r.simg = r.valid ? d.img + r.img_base + (int64_t)f.j * d.s : nullptr;
    r.sfg = nullptr;
    return r;
}

/* grouping orders: ORDER_R groups b2-pairs (b2 is bit 0 already); ORDER_H
 * groups the Hadamard's 2^L values of the low L bits of k, which move below
 * b2 (the low L + 1 bits rotate by one) */
constexpr int ORDER_R = 0, ORDER_H = 1;

/* word 0 of the key with the target's bits moved below the others */
template <int ORDER>
__device__ __forceinline__ uint64_t permuted0(uint64_t w0, int L)
{
    if (ORDER == ORDER_H && L > 0) {
        const uint64_t m = (1ull << L) - 1ull;
        w0 = (w0 & ~((m << 1) | 1ull)) | ((w0 >> 1) & m) | ((w0 & 1ull) << L);
    }
    return w0;
}

template <int ORDER, int NW>
__device__ __forceinline__ bool same_group(const FKeyN<NW> &a, const FKeyN<NW> &b, int L)
{
    const uint64_t m = ORDER == ORDER_R ? 1ull : (((1ull << L) - 1ull) << 1);
    bool eq = (a.w[0] & ~m) == (b.w[0] & ~m);
#pragma unroll
    for (int i = 1; i < NW; ++i) eq = eq && a.w[i] == b.w[i];
    return eq;
}

/* ---- gather, maps, phase ------------------------------------------------------ */

template <typename AmpT, int NW>
__global__ void k_f_gather(QwSimDev d, QwBufDev buf, const double *scale, FKeyN<NW> *keys, double2 *amps,
                           unsigned long long *counter, int64_t cap)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    const double sc = scale ? *scale : 1.0;
    const FLayout L = flayout(d.nb);
    for (int64_t b = warp; b < d.total_buckets; b += nw) {
        int n = buf.count[b];
        if (n <= 0) continue;
        if (n > d.cap_row) n = d.cap_row;
        Row r;
        if (!row_of(d, buf, b, r)) continue;
        for (int i = lane; i < n; i += 32) {
            const int64_t slot = b * (int64_t)d.cap_row + i;
            const unsigned long long p = atomicAdd(counter, 1ull);
            if ((int64_t)p >= cap) continue;
            FRegs f;
            f.inst = r.inst;
            f.jc = r.jc;
            f.j = r.j;
            f.b1 = r.b1;
            f.x = decode_r(buf.key[slot], d.nb);
            FKeyN<NW> k;
#pragma unroll
            for (int t = 0; t < NW; ++t) k.w[t] = 0ull;
            fencode_into(k, f, L);
            keys[p] = k;
            amps[p] = cscale(sc, load_amp<AmpT>(buf.amp, slot));
        }
    }
}

/* op codes of k_f_map, applied from the lowest 4 bits up */
constexpr int F_OSDAG = 1, F_OA = 2, F_OS = 3, F_S = 4, F_A0 = 5;

template <int NW>
__global__ void k_f_map(QwSimDev d, FKeyN<NW> *keys, int64_t M, uint32_t ops, int32_t *status)
{
    const FLayout L = flayout(d.nb);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        /* the base registers are words 0 and 1 of any key width: only they
           are read and written */
        ulonglong2 *base = reinterpret_cast<ulonglong2 *>(keys + i);
        const ulonglong2 b01 = *base;
        FKey k;
        k.w[0] = b01.x;
        k.w[1] = b01.y;
        FRegs f = fdecode(k, L);
        for (uint32_t o = ops; o != 0; o >>= 4) {
            const uint32_t op = o & 15u;
            const Row r = frow(d, f);
            if (op == F_OSDAG) op_osdag(d, r, f.x);
            else if (op == F_OA) op_oa(d, r, f.x);
            else if (op == F_OS) op_os(d, r, f.x);
            else if (op == F_A0) {
                if (f.x.A != 0) atomicOr(status, QW_ST_ANCILLA);
            } else if (op == F_S) { /* (jc, j, b1) <-> (kc, k, b2) */
                const uint32_t jc = f.jc, j = f.j, b1 = f.b1;
                f.jc = f.x.kc;
                f.j = f.x.k;
                f.b1 = f.x.b2;
                f.x.kc = jc;
                f.x.k = j;
                f.x.b2 = b1;
            }
        }
        frewrite(k, f, L);
        *base = make_ulonglong2(k.w[0], k.w[1]);
    }
}

/* P = 2 Pi - 1 (Eq. (impl)): the sign flips unless b1, k, b2, jc, kc are 0 */
template <int NW>
__global__ void k_f_phase(QwSimDev d, const FKeyN<NW> *keys, double2 *amps, int64_t M)
{
    const FLayout L = flayout(d.nb);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const FRegs f = fdecode(fbase_load(keys + i), L);
        const bool zero = f.b1 == 0 && f.x.k == 0 && f.x.b2 == 0 && f.jc == 0 && f.x.kc == 0;
        if (!zero) amps[i] = cneg(amps[i]);
    }
}

/* ---- register-faithful sub-operations (10-word keys) -------------------------- */
/*
 * The working registers of O_s' (its QRAM address, computed out of place:
 * Eq. "Newprocess"), of O_A' and of the quantum binary search (Alg. 1: left,
 * right, mid, midval, the flag and the two comparison bits, and the push/pop
 * garbage stack of (mid, midval, cl, ce) frames, one per probe) held in each
 * branch's key between the sub-operations, above bit 128:
 *   addr, left, right, mid (aw bits each), midval (16), flag, cl, ce (1 each),
 *   then L + 1 frames of mid (aw), midval (16), cl, ce.
 * Addresses follow the QRAM of Fig. 1: the value segment [0, N s), the column
 * segment [N s, 2 N s), row j's slot l at j s + l; a read outside its segment
 * gives 0.
 */
struct FaithLayout {
    int aw;
    int p_addr, p_left, p_right, p_mid, p_midval, p_flag, p_cl, p_ce, p_stk, frame;
};

/* field access on a key held in shared memory (k_fq: one key per thread,
   indexed by the field's word) */
__device__ __forceinline__ uint64_t sget(const uint64_t *w, int pos, int n)
{
    const int i = pos >> 6, o = pos & 63;
    uint64_t v = w[i] >> o;
    if (o + n > 64 && i + 1 < NW_FAITH) v |= w[i + 1] << (64 - o);
    return v & (n >= 64 ? ~0ull : ((1ull << n) - 1ull));
}

__device__ __forceinline__ void sput(uint64_t *w, int pos, int n, uint64_t v)
{
    v &= (n >= 64 ? ~0ull : ((1ull << n) - 1ull));
    const int i = pos >> 6, o = pos & 63;
    w[i] |= v << o;
    if (o + n > 64 && i + 1 < NW_FAITH) w[i + 1] |= v >> (64 - o);
}

__device__ __forceinline__ void sclear(uint64_t *w, int pos, int n)
{
    const uint64_t m = (n >= 64 ? ~0ull : ((1ull << n) - 1ull));
    const int i = pos >> 6, o = pos & 63;
    w[i] &= ~(m << o);
    if (o + n > 64 && i + 1 < NW_FAITH) w[i + 1] &= ~(m >> (64 - o));
}

/* sub-operation codes (the same numbering as the oracle's) */
constexpr int FQ_ADDR_COL = 1, FQ_QRAM_COL = 2, FQ_QBS_FWD = 3, FQ_QBS_BWD = 4, FQ_SWAP = 5, FQ_ADDR_VAL = 6,
              FQ_QRAM_VAL = 7;

__device__ __forceinline__ uint64_t fq_qram(const QwSimDev &d, uint64_t addr, bool col_segment)
{
    const uint64_t ns = (uint64_t)d.n_single * (uint64_t)d.s;
    if (col_segment) {
        if (addr < ns || addr >= 2 * ns) return 0;
        return (uint64_t)(__ldg(d.img + (addr - ns)) >> 16);
    }
    if (addr >= ns) return 0;
    return (uint64_t)(__ldg(d.img + addr) & 0xffffu);
}

__global__ void __launch_bounds__(256) k_fq(QwSimDev d, FKeyW *keys, int64_t M, int op, FaithLayout F, int32_t *status)
{
    const FLayout L = flayout(d.nb);
    const int aw = F.aw;
    const uint64_t ns = (uint64_t)d.n_single * (uint64_t)d.s;
    __shared__ FKeyW sk[256];
    uint64_t *kw = sk[threadIdx.x].w;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        sk[threadIdx.x] = keys[i];
        FKey b = fbase(sk[threadIdx.x]);
        FRegs f = fdecode(b, L);
        uint64_t addr = sget(kw, F.p_addr, aw);
        const uint64_t offset = ns + (uint64_t)f.j * (uint64_t)d.s;
        if (op == FQ_ADDR_COL) {
            addr ^= offset + f.x.k;
        } else if (op == FQ_QRAM_COL) {
            f.x.kc ^= (uint32_t)fq_qram(d, addr, true);
        } else if (op == FQ_ADDR_VAL) {
            if (f.jc == 0 && f.x.kc == 0) addr ^= (uint64_t)f.j * (uint64_t)d.s + f.x.k;
        } else if (op == FQ_QRAM_VAL) {
            if (f.jc == 0 && f.x.kc == 0) f.x.A ^= (uint32_t)fq_qram(d, addr, false);
        } else if (op == FQ_SWAP) {
            const uint32_t t = f.x.k;
            f.x.k = f.x.kc;
            f.x.kc = t;
        } else if (op == FQ_QBS_FWD || op == FQ_QBS_BWD) {
            uint64_t left = sget(kw, F.p_left, aw), right = sget(kw, F.p_right, aw);
            uint64_t mid = sget(kw, F.p_mid, aw), midval = sget(kw, F.p_midval, 16);
            uint32_t flag = (uint32_t)sget(kw, F.p_flag, 1), cl = (uint32_t)sget(kw, F.p_cl, 1);
            uint32_t ce = (uint32_t)sget(kw, F.p_ce, 1);
            const uint64_t target = f.x.kc;
            if (op == FQ_QBS_FWD) { /* Alg. 1's loop, every probe's registers pushed */
                left ^= offset;
                right ^= left + (uint64_t)d.s;
                flag ^= 1u;
                for (int it = 0; it <= d.L; ++it) {
                    if (flag) mid ^= (left + right) / 2;
                    if (flag) midval ^= fq_qram(d, mid, true);
                    if (flag) {
                        cl ^= (midval < target) ? 1u : 0u;
                        ce ^= (midval == target) ? 1u : 0u;
                    }
                    if (ce) f.x.k ^= (uint32_t)(mid - offset);
                    if (ce) flag ^= 1u;
                    if (flag && cl) {
                        const uint64_t t = mid;
                        mid = left;
                        left = t;
                    }
                    if (flag) cl ^= 1u;
                    if (flag && cl) {
                        const uint64_t t = mid;
                        mid = right;
                        right = t;
                    }
                    const int pf = F.p_stk + it * F.frame; /* push: the frame takes them, zeros stay */
                    sput(kw, pf, aw, mid);
                    sput(kw, pf + aw, 16, midval);
                    sput(kw, pf + aw + 16, 1, cl);
                    sput(kw, pf + aw + 17, 1, ce);
                    mid = midval = 0;
                    cl = ce = 0u;
                }
            } else { /* the loop undone in reverse: pop, then every step inverted */
                for (int it = d.L; it >= 0; --it) {
                    const int pf = F.p_stk + it * F.frame;
                    mid = sget(kw, pf, aw);
                    midval = sget(kw, pf + aw, 16);
                    cl = (uint32_t)sget(kw, pf + aw + 16, 1);
                    ce = (uint32_t)sget(kw, pf + aw + 17, 1);
                    sclear(kw, pf, F.frame);
                    if (flag && cl) {
                        const uint64_t t = mid;
                        mid = right;
                        right = t;
                    }
                    if (flag) cl ^= 1u;
                    if (flag && cl) {
                        const uint64_t t = mid;
                        mid = left;
                        left = t;
                    }
                    if (ce) flag ^= 1u;
                    if (flag) {
                        cl ^= (midval < target) ? 1u : 0u;
                        ce ^= (midval == target) ? 1u : 0u;
                    }
                    if (flag) midval ^= fq_qram(d, mid, true);
                    if (flag) mid ^= (left + right) / 2;
                    if (mid != 0 || midval != 0 || cl != 0 || ce != 0) atomicOr(status, QW_ST_ANCILLA);
                    mid = midval = 0;
                    cl = ce = 0u;
                }
                flag ^= 1u;
                right ^= left + (uint64_t)d.s;
                left ^= offset;
                if (left != 0 || right != 0 || flag != 0) atomicOr(status, QW_ST_ANCILLA);
                left = right = 0;
                flag = 0u;
            }
            sclear(kw, F.p_left, aw);
            sclear(kw, F.p_right, aw);
            sclear(kw, F.p_mid, aw);
            sclear(kw, F.p_midval, 16);
            sclear(kw, F.p_flag, 3);
            sput(kw, F.p_left, aw, left);
            sput(kw, F.p_right, aw, right);
            sput(kw, F.p_mid, aw, mid);
            sput(kw, F.p_midval, 16, midval);
            sput(kw, F.p_flag, 1, flag);
            sput(kw, F.p_cl, 1, cl);
            sput(kw, F.p_ce, 1, ce);
        }
        sclear(kw, F.p_addr, aw);
        sput(kw, F.p_addr, aw, addr);
        frewrite(b, f, L);
        kw[0] = b.w[0];
        kw[1] = b.w[1];
        keys[i] = sk[threadIdx.x];
    }
}

/* The sub-operations that touch only the base registers and the address
 * register (ADDR_COL, QRAM_COL, SWAP, ADDR_VAL, QRAM_VAL), as k_fq runs them,
 * reading words 0..2 of the 80-byte key (the address lies at bits 128 ..
 * 128 + aw - 1, in word 2 for aw <= 64) and writing back only the words the
 * operation changes: the address word, or the base registers' two. */
__global__ void k_fq_light(QwSimDev d, FKeyW *keys, int64_t M, int op, int aw)
{
    const FLayout L = flayout(d.nb);
    const uint64_t ns = (uint64_t)d.n_single * (uint64_t)d.s;
    const uint64_t am = aw >= 64 ? ~0ull : (1ull << aw) - 1ull;
    const bool addr_op = op == FQ_ADDR_COL || op == FQ_ADDR_VAL;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        ulonglong2 *base = reinterpret_cast<ulonglong2 *>(keys + i);
        uint64_t *w2p = keys[i].w + 2;
        const ulonglong2 b01 = *base;
        FKey b;
        b.w[0] = b01.x;
        b.w[1] = b01.y;
        FRegs f = fdecode(b, L);
        const uint64_t w2 = op == FQ_SWAP ? 0ull : *w2p;
        uint64_t addr = w2 & am;
        if (addr_op) {
            if (op == FQ_ADDR_COL) addr ^= ns + (uint64_t)f.j * (uint64_t)d.s + f.x.k;
            else if (f.jc == 0 && f.x.kc == 0) addr ^= (uint64_t)f.j * (uint64_t)d.s + f.x.k;
            *w2p = (w2 & ~am) | (addr & am);
            continue;
        }
        if (op == FQ_QRAM_COL) {
            f.x.kc ^= (uint32_t)fq_qram(d, addr, true);
        } else if (op == FQ_QRAM_VAL) {
            if (f.jc == 0 && f.x.kc == 0) f.x.A ^= (uint32_t)fq_qram(d, addr, false);
        } else {
            const uint32_t t = f.x.k;
            f.x.k = f.x.kc;
            f.x.kc = t;
        }
        frewrite(b, f, L);
        *base = make_ulonglong2(b.w[0], b.w[1]);
    }
}

/* the working registers must be 0 (an interference op, P, S or the store) */
__global__ void k_fq_check_idle(const FKeyW *keys, int64_t M, int from_bit, int32_t *status)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const FKeyW k = keys[i];
        bool any = false;
        for (int t = from_bit >> 6; t < NW_FAITH; ++t) {
            uint64_t v = k.w[t];
            if (t == (from_bit >> 6)) v &= ~((1ull << (from_bit & 63)) - 1ull);
            any = any || v != 0ull;
        }
        if (any) atomicOr(status, QW_ST_ANCILLA);
    }
}

/* a list as a table of registers: QW_FQ_COLS values per branch in the order
   inst, jc, j, b1, kc, k, b2, A, addr, left, right, mid, midval, flag, cl,
   ce, then QW_FQ_FRAMES frames of (mid, midval, cl, ce) */
__global__ void k_fq_export(QwSimDev d, const FKeyW *keys, int64_t M, FaithLayout F, uint64_t *table)
{
    const FLayout L = flayout(d.nb);
    const int aw = F.aw;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const FKeyW k = keys[i];
        const FRegs f = fdecode(k, L);
        uint64_t *t = table + i * QW_FQ_COLS;
        t[0] = f.inst;
        t[1] = f.jc;
        t[2] = f.j;
        t[3] = f.b1;
        t[4] = f.x.kc;
        t[5] = f.x.k;
        t[6] = f.x.b2;
        t[7] = f.x.A;
        t[8] = fget(k, F.p_addr, aw);
        t[9] = fget(k, F.p_left, aw);
        t[10] = fget(k, F.p_right, aw);
        t[11] = fget(k, F.p_mid, aw);
        t[12] = fget(k, F.p_midval, 16);
        t[13] = fget(k, F.p_flag, 1);
        t[14] = fget(k, F.p_cl, 1);
        t[15] = fget(k, F.p_ce, 1);
        for (int it = 0; it < QW_FQ_FRAMES; ++it) {
            uint64_t *fr = t + 16 + 4 * it;
            if (it <= d.L) {
                const int pf = F.p_stk + it * F.frame;
                fr[0] = fget(k, pf, aw);
                fr[1] = fget(k, pf + aw, 16);
                fr[2] = fget(k, pf + aw + 16, 1);
                fr[3] = fget(k, pf + aw + 17, 1);
            } else {
                fr[0] = fr[1] = fr[2] = fr[3] = 0ull;
            }
        }
    }
}

/* ---- device-wide exclusive scan of 32-bit counts ------------------------------ */

constexpr int SCAN_TILE = 1024; /* elements per block: 256 threads x 4 */

__global__ void k_scan_reduce(const uint32_t *in, int64_t n, uint32_t *sums)
{
    __shared__ uint32_t ws[8];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    uint32_t v = 0;
    for (int t = 0; t < 4; ++t) {
        const int64_t i = base + threadIdx.x * 4 + t;
        if (i < n) v += in[i];
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < 8; ++w) t += ws[w];
        sums[blockIdx.x] = t;
    }
}

/* one block: exclusive scan of the block sums in place, total at sums[nb] */
__global__ void k_scan_blocks(uint32_t *sums, int64_t nb)
{
    __shared__ uint32_t ws[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = 0; base < nb; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const uint32_t v = i < nb ? sums[i] : 0u;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL, w, o);
                if (lane >= o) w += y;
            }
            ws[lane] = w;
        }
        __syncthreads();
        const uint32_t before = carry + (warp > 0 ? ws[warp - 1] : 0u) + x - v;
        if (i < nb) sums[i] = before;
        __syncthreads();
        if (threadIdx.x == 0) carry += ws[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void k_scan_apply(const uint32_t *in, int64_t n, const uint32_t *sums, uint32_t *out)
{
    __shared__ uint32_t ws[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * 4;
    uint32_t v[4], t = 0;
    for (int k = 0; k < 4; ++k) {
        v[k] = base + k < n ? in[base + k] : 0u;
        t += v[k];
    }
    uint32_t x = t;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += ws[w];
    uint32_t run = sums[blockIdx.x] + wpre + x - t;
    for (int k = 0; k < 4; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

/* ---- radix sort ------------------------------------------------------------------ */

/* OR and AND of every permuted key, word by word: the bits that differ
   between keys.  The key array is read as a flat array of 64-bit words; the
   grid's stride is a multiple of NW, so each thread always sees one word
   index. */
template <int ORDER, int NW>
__global__ void k_f_orand(const uint64_t *words, int64_t nwords, int L, unsigned long long *acc)
{
    __shared__ unsigned long long s_or[NW], s_and[NW];
    if (threadIdx.x < NW) {
        s_or[threadIdx.x] = 0ull;
        s_and[threadIdx.x] = ~0ull;
    }
    __syncthreads();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int wi = (int)(g % NW);
    uint64_t ov = 0ull, av = ~0ull;
    for (int64_t q = g; q < nwords; q += stride) {
        uint64_t v = words[q];
        if (wi == 0) v = permuted0<ORDER>(v, L);
        ov |= v;
        av &= v;
    }
    atomicOr(&s_or[wi], (unsigned long long)ov);
    atomicAnd(&s_and[wi], (unsigned long long)av);
    __syncthreads();
    if (threadIdx.x < NW) {
        atomicOr(acc + threadIdx.x, s_or[threadIdx.x]);
        atomicAnd(acc + NW + threadIdx.x, s_and[threadIdx.x]);
    }
}

/* The sort runs on a compacted key (the chunks of qw_sort_chunks.h).  LSD
 * order carries over chunks: chunk 0 is sorted first, chunk c + 1 is formed
 * from the keys in the order chunk c left. */
constexpr int OS_THREADS = 256, OS_IPT = 8, OS_TILE = OS_THREADS * OS_IPT;
constexpr int OS_SPIN_LIMIT = 1 << 22;

/* The chunk's compacted key of every entry -- the entry at position i of the
   current order, i.e. keys[perm[i]] (perm == nullptr: i) -- and the global
   count of every 8-bit digit of it for each of the chunk's passes
   (ghist[pass * 256 + digit], zeroed by the caller). */
template <int ORDER, int NW>
__global__ void __launch_bounds__(256) k_f_ckey(const FKeyN<NW> *keys, const uint32_t *perm, int64_t M, int L,
                                                CkRuns runs, uint64_t *ck, uint32_t *ghist)
{
    __shared__ uint32_t h[CK_MAXPASS * 256];
    for (int t = threadIdx.x; t < CK_MAXPASS * 256; t += blockDim.x) h[t] = 0u;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = perm ? (int64_t)perm[i] : i;
        if (j >= M) j = 0; /* only after a sort wait gave up */
        const FKeyN<NW> *k = keys + j;
        uint64_t c = 0ull, v = 0ull;
        int dst = 0, cw = -1;
        for (int r = 0; r < runs.n; ++r) {
            const int w = runs.word[r];
            if (w != cw) {
                v = k->w[w];
                if (w == 0) v = permuted0<ORDER>(v, L);
                cw = w;
            }
            const int ln = runs.len[r];
            const uint64_t m = ln >= 64 ? ~0ull : (1ull << ln) - 1ull;
            c |= ((v >> runs.shift[r]) & m) << dst;
            dst += ln;
        }
        ck[i] = c;
        for (int p = 0; p < runs.npass; ++p) atomicAdd(&h[p * 256 + (int)((c >> (8 * p)) & 255ull)], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < runs.npass * 256; t += blockDim.x)
        if (h[t]) atomicAdd(ghist + t, h[t]);
}

/* status of a tile in one pass, one 64-bit word per (tile, digit): the pass
   tag (bits 40..63; a word of another pass reads as not ready), 1 = the
   tile's own count / 2 = the inclusive prefix over tiles 0..vb (bits 38, 39),
   the count (bits 0..37) */
constexpr uint64_t OS_AGG = 1ull << 38, OS_INC = 2ull << 38, OS_CNT = (1ull << 38) - 1ull;

__device__ __forceinline__ uint64_t os_load(const uint64_t *p)
{
    return *reinterpret_cast<const volatile uint64_t *>(p);
}

__device__ __forceinline__ void os_store(uint64_t *p, uint64_t v)
{
    *reinterpret_cast<volatile uint64_t *>(p) = v;
}

/* One stable pass on the 8-bit digit at `shift` of the compacted key.  A
 * block takes tile vb in the order blocks start (a counter), so every tile
 * before it belongs to a block already running.  Warp w ranks items vb T +
 * 256 w + 32 r + lane (r = 0..7) by their digit in that order; the tile's
 * digit counts are published, then the counts of the tiles before it are
 * summed by looking back until a tile with its inclusive prefix (single-pass
 * "decoupled look-back" prefix sum); an item goes to the digit's global
 * start (the exclusive scan of ghist) + the tiles before + the warps before
 * + its rank.  A wait that outlasts OS_SPIN_LIMIT polls sets
 * QW_ST_SORT_WAIT and the block carries on (the sort's result is then
 * wrong, and the host reports the status). */
template <bool FIRST, bool WRITE_CK>
__global__ void __launch_bounds__(OS_THREADS, 4) k_f_onesweep(const uint64_t *ckin, const uint32_t *ixin, uint64_t *ckout,
                                                           uint32_t *ixout, int64_t M, int shift,
                                                           const uint32_t *ghist, uint64_t *stat, uint64_t tag,
                                                           unsigned int *ctr, int32_t *status)
{
    __shared__ uint32_t hw[8][256];
    __shared__ uint32_t sbase[256];
    __shared__ uint32_t wsum[8];
    __shared__ unsigned int svb;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (t == 0) svb = atomicAdd(ctr, 1u);
#pragma unroll
    for (int w = 0; w < 8; ++w) hw[w][t] = 0u;
    __syncthreads();
    const int64_t vb = svb;
    const int64_t base = vb * OS_TILE + warp * (32 * OS_IPT) + lane;
    uint64_t c[OS_IPT];
    uint32_t ix[OS_IPT], rk[OS_IPT];
    int dg[OS_IPT];
#pragma unroll
    for (int r = 0; r < OS_IPT; ++r) {
        const int64_t i = base + 32 * r;
        dg[r] = 256;
        c[r] = 0ull;
        ix[r] = 0u;
        if (i < M) {
            c[r] = ckin[i];
            ix[r] = FIRST ? (uint32_t)i : ixin[i];
            dg[r] = (int)((c[r] >> shift) & 255ull);
        }
    }
    const unsigned below = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < OS_IPT; ++r) {
        const unsigned m = __match_any_sync(FULL, dg[r]);
        const int d = dg[r];
        const uint32_t cnt = d < 256 ? hw[warp][d] : 0u;
        rk[r] = cnt + (uint32_t)__popc(m & below);
        __syncwarp();
        if (d < 256 && (m & below) == 0u) hw[warp][d] = cnt + (uint32_t)__popc(m);
        __syncwarp();
    }
    __syncthreads();
    /* thread t owns digit t: the warps' exclusive prefix, the tile's count */
    uint32_t run = 0u;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const uint32_t v = hw[w][t];
        hw[w][t] = run;
        run += v;
    }
    uint64_t *my = stat + vb * 256 + t;
    os_store(my, (tag << 40) | (vb == 0 ? OS_INC : OS_AGG) | run);
    /* global start of digit t: exclusive scan of this pass's digit counts */
    const uint32_t g = ghist[t];
    uint32_t x = g;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    /* look back over the tiles before */
    uint64_t excl = 0ull;
    if (vb > 0) {
        int64_t p = vb - 1;
        int spins = 0;
        while (p >= 0) {
            const uint64_t v = os_load(stat + p * 256 + t);
            if ((v >> 40) != tag) {
                if (++spins > OS_SPIN_LIMIT) {
                    atomicOr(status, QW_ST_SORT_WAIT);
                    break;
                }
                if (spins > 32) __nanosleep(64);
                continue;
            }
            excl += v & OS_CNT;
            if (v & OS_INC) break;
            --p;
        }
        os_store(my, (tag << 40) | OS_INC | (excl + run));
    }
    __syncthreads();
    uint32_t pre = 0u;
    for (int w = 0; w < warp; ++w) pre += wsum[w];
    sbase[t] = pre + x - g + (uint32_t)excl;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < OS_IPT; ++r) {
        const int d = dg[r];
        const uint32_t dest = d < 256 ? sbase[d] + hw[warp][d] + rk[r] : 0u;
        if (d < 256 && (int64_t)dest < M) { /* always, unless a wait gave up */
            if (WRITE_CK) ckout[dest] = c[r];
            ixout[dest] = ix[r];
        }
    }
}

/* the sorted list: entry i is the entry perm[i] of the input */
template <int NW>
__global__ void k_f_permute(const FKeyN<NW> *kin, const double2 *ain, const uint32_t *perm, FKeyN<NW> *kout,
                            double2 *aout, int64_t M)
{
    static_assert(NW % 2 == 0, "keys are copied as 16-byte words");
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = perm[i];
        if (j >= M) j = 0; /* only after a sort wait gave up */
        const ulonglong2 *s = reinterpret_cast<const ulonglong2 *>(kin + j);
        ulonglong2 *o = reinterpret_cast<ulonglong2 *>(kout + i);
#pragma unroll
        for (int q = 0; q < NW / 2; ++q) o[q] = s[q];
        aout[i] = ain[j];
    }
}

/* ---- per-group transforms (the "computing" step) -------------------------------- */

/* R (DAG = false) or R^dag on b2-pairs (sorted in ORDER_R): the head of each
 * pair writes both outputs at 2 i (b2 = 0) and 2 i + 1 (b2 = 1) with their
 * keep flags; R = [[f, -g], [g, conj f]] (Alg. T~ and the footnote of Sec. IV). */
template <bool DAG, int NW>
__global__ void k_f_rot(QwSimDev d, const FKeyN<NW> *keys, const double2 *amps, int64_t M, FKeyN<NW> *okeys,
                        double2 *oamps, uint32_t *flags)
{
    const FLayout L = flayout(d.nb);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const FKeyN<NW> k = keys[i];
        const bool head = i == 0 || !same_group<ORDER_R>(keys[i - 1], k, 0);
        flags[2 * i] = 0u;
        flags[2 * i + 1] = 0u;
        if (!head) continue;
        double2 a0 = make_double2(0, 0), a1 = make_double2(0, 0);
        if ((k.w[0] & 1ull) == 0) {
            a0 = amps[i];
            if (i + 1 < M && same_group<ORDER_R>(k, keys[i + 1], 0)) a1 = amps[i + 1];
        } else {
            a1 = amps[i];
        }
        const FRegs f = fdecode(k, L);
        double2 fv;
        double g;
        rot_fg(d, f.x.A, f.j, f.x.k, fv, g);
        double2 o0, o1;
        if (!DAG) {
            o0 = csub(cmul(fv, a0), cscale(g, a1));
            o1 = cadd(cscale(g, a0), cmul(cconj(fv), a1));
        } else {
            o0 = cadd(cmul(cconj(fv), a0), cscale(g, a1));
            o1 = csub(cmul(fv, a1), cscale(g, a0));
        }
        FKeyN<NW> k0 = k;
        k0.w[0] &= ~1ull;
        FKeyN<NW> k1 = k0;
        k1.w[0] |= 1ull;
        okeys[2 * i] = k0;
        okeys[2 * i + 1] = k1;
        oamps[2 * i] = o0;
        oamps[2 * i + 1] = o1;
        flags[2 * i] = keep(o0, d.tau2) ? 1u : 0u;
        flags[2 * i + 1] = keep(o1, d.tau2) ? 1u : 0u;
    }
}

/* H on the low L bits of k (sorted in ORDER_H): the head of each group
 * writes the s outputs (1/sqrt s) sum_v (-1)^(u.v) a_v at s i + u. */
template <int NW>
__global__ void k_f_heads(QwSimDev d, const FKeyN<NW> *keys, int64_t M, uint32_t *flags)
{
    const int L = d.L;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = (i == 0 || !same_group<ORDER_H>(keys[i - 1], keys[i], L)) ? 1u : 0u;
}

/* starts[g] = the first member of group g (gidx: the exclusive scan of the
   head flags), starts[G] = M */
__global__ void k_f_starts(const uint32_t *heads, const uint32_t *gidx, int64_t M, int64_t G, int64_t *starts)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        if (heads[i]) starts[gidx[i]] = i;
        if (i == 0) starts[G] = M;
    }
}

/* The s outputs of every Hadamard group (members equal but for the low L
 * bits of k, contiguous after the sort): one thread per (group, u), the
 * group's members read in list order, so each output is the same sum as a
 * dense s x s product on the zero-filled vector. */
/* H on each group's zero-filled vector of 2^L = s entries (the groups of
 * the list sorted in ORDER_H, starts[g] .. starts[g + 1]): output u of a group
 * is s^-1/2 sum_m (-1)^{|u & v_m|} a_m over its members m (v_m: their low L
 * bits of k).  A warp runs 32 / s groups (s < 32) or one group (s >= 32).
 * For s <= 128 lane t of a group holds entries t, t + 32, ... of the
 * zero-filled vector, and the L butterfly stages of the fast Walsh-Hadamard
 * transform (Sylvester order, (x, y) -> (x + y, x - y) on index bit h) run
 * over shuffles (bits below 32) and between the lane's registers (bits
 * above): s L additions per group instead of s^2; the FP64 pipe is the
 * limit.  Larger s: s / 32 rounds of 32 outputs, each the direct sum over
 * the members in list order (a lane loads one member per round and the
 * warp's shuffles hand them to every output).
 * COUNT: the kept outputs of each group into cnt[g]; otherwise the kept
 * outputs are written, in order of u, from gpos[g] (the exclusive scan of
 * cnt) -- the clearing step without a list of all G s outputs. */
template <int NW, bool COUNT, int FWHT_ROUNDS>
__global__ void __launch_bounds__(256) k_f_hgroups(QwSimDev d, const FKeyN<NW> *keys, const double2 *amps,
                                                   const int64_t *starts, int64_t G, uint32_t *cnt,
                                                   const uint32_t *gpos, FKeyN<NW> *okeys, double2 *oamps)
{
    const int s = d.s;
    const int sw = s < 32 ? s : 32, gpw = 32 / sw, rounds = s / sw;
    const int lane = threadIdx.x & 31, sub = lane / sw, ul = lane - sub * sw, first = sub * sw;
    const unsigned seg = sw == 32 ? FULL : ((1u << sw) - 1u) << first;
    const unsigned below = (1u << lane) - 1u;
    const uint64_t lowm = ((uint64_t)s - 1ull) << 1;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    constexpr int ZR = FWHT_ROUNDS > 0 ? FWHT_ROUNDS : 1;
    const bool fwht = FWHT_ROUNDS > 0;
    __shared__ double2 zv[8][32 * ZR];
    double2 *vec = zv[threadIdx.x >> 5];
    for (int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wg * gpw < G; wg += nwarps) {
        const int64_t g = wg * gpw + sub;
        const bool act = g < G;
        const int64_t b = act ? starts[g] : 0, nm = act ? starts[g + 1] - b : 0;
        /* fast transform: entry q sw + ul of the group's zero-filled vector
           in x[q], the butterflies of index bits below sw over shuffles, the
           ones above between the lane's registers; x[q] is then output
           u = q sw + ul */
        double2 x[ZR];
        if (fwht) {
#pragma unroll
            for (int q = 0; q < ZR; ++q)
                if (q < rounds) vec[first + q * sw + ul] = make_double2(0, 0);
            __syncwarp();
#pragma unroll
            for (int q = 0; q < ZR; ++q) {
                const int64_t mi = (int64_t)q * sw + ul;
                if (q < rounds && mi < nm)
                    vec[first + (int)((keys[b + mi].w[0] >> 1) & (uint64_t)(s - 1))] = amps[b + mi];
            }
            __syncwarp();
#pragma unroll
            for (int q = 0; q < ZR; ++q) x[q] = q < rounds ? vec[first + q * sw + ul] : make_double2(0, 0);
            __syncwarp();
            for (int h = 1; h < sw; h <<= 1) {
#pragma unroll
                for (int q = 0; q < ZR; ++q) {
                    if (q >= rounds) continue;
                    const double yx = __shfl_xor_sync(FULL, x[q].x, h), yy = __shfl_xor_sync(FULL, x[q].y, h);
                    x[q] = (ul & h) ? make_double2(yx - x[q].x, yy - x[q].y)
                                    : make_double2(x[q].x + yx, x[q].y + yy);
                }
            }
#pragma unroll
            for (int hq = 1; hq < ZR; hq <<= 1) {
#pragma unroll
                for (int q = 0; q < ZR; ++q) {
                    if ((q & hq) || (q | hq) >= rounds) continue;
                    const double2 lo = x[q], hi = x[q | hq];
                    x[q] = make_double2(lo.x + hi.x, lo.y + hi.y);
                    x[q | hq] = make_double2(lo.x - hi.x, lo.y - hi.y);
                }
            }
        }
        uint32_t run = 0u;
        for (int q = 0; q < rounds; ++q) {
            const uint32_t u = (uint32_t)(q * sw + ul);
            double2 o = make_double2(0, 0);
            if (fwht) {
#pragma unroll
                for (int t = 0; t < ZR; ++t)
                    if (t == q) o = x[t];
            }
            for (int q2 = 0; q2 < rounds && !fwht; ++q2) {
                const int64_t mi = (int64_t)q2 * sw + ul;
                uint32_t mv = 0u;
                double2 ma = make_double2(0, 0);
                if (mi < nm) {
                    mv = (uint32_t)((keys[b + mi].w[0] >> 1) & (uint64_t)(s - 1));
                    ma = amps[b + mi];
                }
                for (int j = 0; j < sw; ++j) {
                    const uint32_t v = __shfl_sync(FULL, mv, first + j);
                    const double ax = __shfl_sync(FULL, ma.x, first + j);
                    const double ay = __shfl_sync(FULL, ma.y, first + j);
                    if ((int64_t)q2 * sw + j < nm) {
                        const double2 a = make_double2(ax, ay);
                        o = (__popc(u & v) & 1) ? csub(o, a) : cadd(o, a);
                    }
                }
            }
            o = cscale(d.inv_sqrt_s, o);
            const bool kept = act && keep(o, d.tau2);
            const unsigned bal = __ballot_sync(FULL, kept) & seg;
            const uint32_t rank = run + (uint32_t)__popc(bal & below);
            if (!COUNT && kept && rank < cnt[g]) { /* the count pass made the same decisions */
                const int64_t dst = (int64_t)gpos[g] + rank;
                FKeyN<NW> ko = keys[b];
                ko.w[0] = (ko.w[0] & ~lowm) | ((uint64_t)u << 1);
                okeys[dst] = ko;
                oamps[dst] = o;
            }
            run += (uint32_t)__popc(bal);
        }
        if (COUNT && act && ul == 0) cnt[g] = run;
    }
}

/* the "clearing" step: kept entries to their scanned positions */
template <int NW>
__global__ void k_f_compact(const FKeyN<NW> *keys, const double2 *amps, const uint32_t *flags, const uint32_t *pos,
                            int64_t n, FKeyN<NW> *okeys, double2 *oamps)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!flags[i]) continue;
        okeys[pos[i]] = keys[i];
        oamps[pos[i]] = amps[i];
    }
}

/* QLS read-out after T~^dag's H: Y[j] += a_j * (the flag-0 amplitude of row j) */
template <int NW>
__global__ void k_f_readout(QwSimDev d, const FKeyN<NW> *keys, const double2 *amps, int64_t M, QwStepArgs a)
{
    const FLayout L = flayout(d.nb);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const FRegs f = fdecode(fbase_load(keys + i), L);
        if (f.jc != 0 || f.b1 != 0 || f.x.kc != 0 || f.x.k != 0 || f.x.b2 != 0 || f.x.A != 0) continue;
        if (f.j >= (uint32_t)d.n_single) continue;
        const double coef = a.qls_coefs[*a.qls_j];
        const double2 v = amps[i];
        atomicAdd(&a.qls_y[f.j].x, coef * v.x);
        atomicAdd(&a.qls_y[f.j].y, coef * v.y);
    }
}

/* the output into the row buckets, |stored a|^2 summed per block into *norm */
template <typename AmpT, int NW>
__global__ void k_f_scatter(QwSimDev d, QwBufDev out, const FKeyN<NW> *keys, const double2 *amps, int64_t M,
                            int32_t *status, unsigned int *maxrow, double *norm)
{
    __shared__ double ws[8];
    const FLayout L = flayout(d.nb);
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const FRegs f = fdecode(fbase_load(keys + i), L);
        if (f.x.A != 0) {
            atomicOr(status, QW_ST_ANCILLA);
            continue;
        }
        const int64_t b = bucket_of(d, out, f.inst, f.jc, f.j, f.b1, status);
        if (b < 0) continue;
        const int p = atomicAdd(out.count + b, 1);
        atomicMax(maxrow, (unsigned int)(p + 1));
        if (p >= d.cap_row) {
            atomicOr(status, QW_ST_ROW_OVERFLOW);
            continue;
        }
        const int64_t slot = b * (int64_t)d.cap_row + p;
        out.key[slot] = encode_r(f.x, d.nb);
        acc += store_amp<AmpT>(out.amp, slot, amps[i]);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        atomicAdd(norm, t);
    }
}

/* the step's bookkeeping, as the step kernels' last block does it */
__global__ void k_f_finish(QwStepArgs a, const double *norm, unsigned long long in, unsigned long long rdag,
                           unsigned long long h1, unsigned long long hph, unsigned long long out)
{
    const bool clean = *(volatile int32_t *)a.status == 0;
    if (!clean) return;
    const double tot = *norm;
    *a.norm_out = tot;
    if (a.scale_out) *a.scale_out = (a.renorm && tot > 0.0) ? sqrt(*a.renorm_target / tot) : 1.0;
    if (a.steps_done) *a.steps_done += 1;
    if (a.stats) {
        a.stats[QW_STAT_IN] += in;
        a.stats[QW_STAT_RDAG] += rdag;
        a.stats[QW_STAT_H1] += h1;
        a.stats[QW_STAT_HPH] += hph;
        a.stats[QW_STAT_OUT] += out;
        a.stats[QW_STAT_STEPS] += 1;
    }
}

int grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    const int cap = 16 * qw_sm_count();
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

template <int NW>
cudaError_t flat_sort_t(const QwSimDev &d, void *keys, double2 *amps, void *tmpk, double2 *tmpa, int64_t M, int order,
                        uint32_t *work, cudaStream_t st);

} // namespace

/* ---- launchers ------------------------------------------------------------------------ */
/* kw: the key words (2, the export layout; 10, the register-faithful layout) */

cudaError_t qw_flat_gather(const QwSimDev &d, const QwBufDev &buf, int fp32, const double *scale, void *keys,
                           double2 *amps, unsigned long long *counter, int64_t cap, cudaStream_t st, int kw)
{
    const int grid = 4 * qw_sm_count();
    if (kw == NW_FAITH) {
        if (fp32)
            k_f_gather<float2, NW_FAITH><<<grid, 256, 0, st>>>(d, buf, scale, static_cast<FKeyW *>(keys), amps,
                                                               counter, cap);
        else
            k_f_gather<double2, NW_FAITH><<<grid, 256, 0, st>>>(d, buf, scale, static_cast<FKeyW *>(keys), amps,
                                                                counter, cap);
    } else if (fp32) {
        k_f_gather<float2, 2><<<grid, 256, 0, st>>>(d, buf, scale, static_cast<FKey *>(keys), amps, counter, cap);
    } else {
        k_f_gather<double2, 2><<<grid, 256, 0, st>>>(d, buf, scale, static_cast<FKey *>(keys), amps, counter, cap);
    }
    return cudaGetLastError();
}

cudaError_t qw_flat_map(const QwSimDev &d, void *keys, int64_t M, uint32_t ops, int32_t *status, cudaStream_t st,
                        int kw)
{
    if (M <= 0) return cudaSuccess;
    if (kw == NW_FAITH) k_f_map<NW_FAITH><<<grid_for(M, 256), 256, 0, st>>>(d, static_cast<FKeyW *>(keys), M, ops, status);
    else k_f_map<2><<<grid_for(M, 256), 256, 0, st>>>(d, static_cast<FKey *>(keys), M, ops, status);
    return cudaGetLastError();
}

cudaError_t qw_flat_phase(const QwSimDev &d, const void *keys, double2 *amps, int64_t M, cudaStream_t st, int kw)
{
    if (M <= 0) return cudaSuccess;
    if (kw == NW_FAITH)
        k_f_phase<NW_FAITH><<<grid_for(M, 256), 256, 0, st>>>(d, static_cast<const FKeyW *>(keys), amps, M);
    else k_f_phase<2><<<grid_for(M, 256), 256, 0, st>>>(d, static_cast<const FKey *>(keys), amps, M);
    return cudaGetLastError();
}

size_t qw_flat_scan_words(int64_t n)
{
    return (size_t)((n + SCAN_TILE - 1) / SCAN_TILE) + 1;
}

cudaError_t qw_flat_scan(const uint32_t *in, int64_t n, uint32_t *sums, uint32_t *out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    k_scan_reduce<<<(unsigned)nb, 256, 0, st>>>(in, n, sums);
    k_scan_blocks<<<1, 1024, 0, st>>>(sums, nb);
    k_scan_apply<<<(unsigned)nb, 256, 0, st>>>(in, n, sums, out);
    return cudaGetLastError();
}

namespace {
/* work layout of qw_flat_sort, in bytes: the tiles' status words, the
   digit counts of every chunk, the block counters of every pass, two
   compacted-key and two permutation arrays */
struct SortWork {
    uint64_t *stat;
    uint32_t *ghist;
    unsigned int *ctr;
    unsigned long long *acc;
    uint64_t *ck[2];
    uint32_t *ix[2];
    size_t zero_bytes, total;
};

constexpr int SORT_MAXPASSES = 64 * NW_FAITH / 8;

size_t align256(size_t b)
{
    return (b + 255) & ~(size_t)255;
}

SortWork sort_work(void *base, int64_t M)
{
    const int64_t n = M < 1 ? 1 : M;
    const int64_t nblk = (n + OS_TILE - 1) / OS_TILE;
    char *p = static_cast<char *>(base);
    SortWork w;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *q = p ? p + off : nullptr;
        off += align256(bytes);
        return q;
    };
    w.stat = reinterpret_cast<uint64_t *>(take((size_t)nblk * 256 * 8));
    w.ghist = reinterpret_cast<uint32_t *>(take((size_t)NW_FAITH * CK_MAXPASS * 256 * 4));
    w.ctr = reinterpret_cast<unsigned int *>(take((size_t)SORT_MAXPASSES * 4));
    w.zero_bytes = off;
    w.acc = reinterpret_cast<unsigned long long *>(take(2 * NW_FAITH * 8));
    w.ck[0] = reinterpret_cast<uint64_t *>(take((size_t)n * 8));
    w.ck[1] = reinterpret_cast<uint64_t *>(take((size_t)n * 8));
    w.ix[0] = reinterpret_cast<uint32_t *>(take((size_t)n * 4));
    w.ix[1] = reinterpret_cast<uint32_t *>(take((size_t)n * 4));
    w.total = off;
    return w;
}

/* Stable sort of (keys, amps) by the permuted key of `order` (0: R, 1: H):
 * one synchronisation reads which bits vary; they are sorted in chunks of
 * 64, each by 8-bit passes carrying a permutation; the entries are moved
 * once at the end, into tmpk / tmpa (*in_tmp = 1).  A list whose keys are
 * all equal is already sorted (*in_tmp = 0). */
template <int NW>
cudaError_t flat_sort_t(const QwSimDev &d, void *keys, double2 *amps, void *tmpk, double2 *tmpa, int64_t M, int order,
                        void *work, int32_t *status, cudaStream_t st, int *in_tmp)
{
    *in_tmp = 0;
    if (M <= 1) return cudaSuccess;
    if (M > (int64_t)UINT32_MAX) return cudaErrorInvalidValue; /* 32-bit positions */
    const int L = d.L;
    const SortWork w = sort_work(work, M);
    unsigned long long init[2 * NW];
    for (int t = 0; t < NW; ++t) {
        init[t] = 0ull;
        init[NW + t] = ~0ull;
    }
    cudaError_t e = cudaMemcpyAsync(w.acc, init, sizeof init, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    const int othreads = 32 * NW;
    const int ogrid = grid_for(M * NW, othreads);
    const uint64_t *kwords = static_cast<const uint64_t *>(keys);
    if (order == ORDER_R) k_f_orand<ORDER_R, NW><<<ogrid, othreads, 0, st>>>(kwords, M * NW, L, w.acc);
    else k_f_orand<ORDER_H, NW><<<ogrid, othreads, 0, st>>>(kwords, M * NW, L, w.acc);
    if ((e = cudaMemsetAsync(w.stat, 0, w.zero_bytes, st)) != cudaSuccess) return e;
    unsigned long long h[2 * NW];
    if ((e = cudaMemcpyAsync(h, w.acc, sizeof h, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    /* the varying bits as runs, split into chunks of 64 */
    uint64_t var[NW];
    for (int wi = 0; wi < NW; ++wi) var[wi] = h[wi] ^ h[NW + wi];
    std::vector<CkRuns> chunks(NW);
    chunks.resize((size_t)qw_sort_chunks(var, NW, chunks.data()));
    if (chunks.empty()) return cudaSuccess;
    const int64_t nblk = (M + OS_TILE - 1) / OS_TILE;
    const int kgrid = grid_for(M, 256);
    const FKeyN<NW> *kin = static_cast<const FKeyN<NW> *>(keys);
    int curix = -1, curck = 0;
    uint64_t tag = 0;
    for (size_t c = 0; c < chunks.size(); ++c) {
        const CkRuns &r = chunks[c];
        uint32_t *gh = w.ghist + c * CK_MAXPASS * 256;
        const uint32_t *perm = curix < 0 ? nullptr : w.ix[curix];
        if (order == ORDER_R) k_f_ckey<ORDER_R, NW><<<kgrid, 256, 0, st>>>(kin, perm, M, L, r, w.ck[curck], gh);
        else k_f_ckey<ORDER_H, NW><<<kgrid, 256, 0, st>>>(kin, perm, M, L, r, w.ck[curck], gh);
        for (int p = 0; p < r.npass; ++p) {
            ++tag;
            const bool wck = p + 1 < r.npass;
            const int outix = curix == 0 ? 1 : 0;
            const uint64_t *ci = w.ck[curck];
            uint64_t *co = w.ck[curck ^ 1];
            uint32_t *xo = w.ix[outix];
            unsigned int *ctr = w.ctr + (tag - 1);
            const uint32_t *ghp = gh + p * 256;
            const unsigned grid = (unsigned)nblk;
            if (curix < 0) {
                if (wck) k_f_onesweep<true, true><<<grid, OS_THREADS, 0, st>>>(ci, nullptr, co, xo, M, 8 * p, ghp, w.stat, tag, ctr, status);
                else k_f_onesweep<true, false><<<grid, OS_THREADS, 0, st>>>(ci, nullptr, co, xo, M, 8 * p, ghp, w.stat, tag, ctr, status);
            } else {
                const uint32_t *xi = w.ix[curix];
                if (wck) k_f_onesweep<false, true><<<grid, OS_THREADS, 0, st>>>(ci, xi, co, xo, M, 8 * p, ghp, w.stat, tag, ctr, status);
                else k_f_onesweep<false, false><<<grid, OS_THREADS, 0, st>>>(ci, xi, co, xo, M, 8 * p, ghp, w.stat, tag, ctr, status);
            }
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            curix = outix;
            if (wck) curck ^= 1;
        }
    }
    k_f_permute<NW><<<kgrid, 256, 0, st>>>(kin, amps, w.ix[curix], static_cast<FKeyN<NW> *>(tmpk), tmpa, M);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *in_tmp = 1;
    return cudaSuccess;
}
} // namespace

size_t qw_flat_sort_bytes(int64_t M)
{
    return sort_work(nullptr, M).total;
}

cudaError_t qw_flat_sort(const QwSimDev &d, void *keys, double2 *amps, void *tmpk, double2 *tmpa, int64_t M,
                         int order, void *work, int32_t *status, cudaStream_t st, int kw, int *in_tmp)
{
    if (kw == NW_FAITH) return flat_sort_t<NW_FAITH>(d, keys, amps, tmpk, tmpa, M, order, work, status, st, in_tmp);
    return flat_sort_t<2>(d, keys, amps, tmpk, tmpa, M, order, work, status, st, in_tmp);
}

/* op: 0 = R^dag, 1 = R (2 outputs per entry), 2 = H (s outputs per entry) */
cudaError_t qw_flat_heads(const QwSimDev &d, const void *keys, int64_t M, uint32_t *flags, cudaStream_t st, int kw)
{
    if (M <= 0) return cudaSuccess;
    if (kw == NW_FAITH)
        k_f_heads<NW_FAITH><<<grid_for(M, 256), 256, 0, st>>>(d, static_cast<const FKeyW *>(keys), M, flags);
    else k_f_heads<2><<<grid_for(M, 256), 256, 0, st>>>(d, static_cast<const FKey *>(keys), M, flags);
    return cudaGetLastError();
}

cudaError_t qw_flat_starts(const uint32_t *heads, const uint32_t *gidx, int64_t M, int64_t G, int64_t *starts,
                           cudaStream_t st)
{
    if (M <= 0) return cudaSuccess;
    k_f_starts<<<grid_for(M, 256), 256, 0, st>>>(heads, gidx, M, G, starts);
    return cudaGetLastError();
}

cudaError_t qw_flat_group(const QwSimDev &d, int op, const void *keys, const double2 *amps, int64_t M, void *okeys,
                          double2 *oamps, uint32_t *flags, cudaStream_t st, int kw)
{
    if (M <= 0) return cudaSuccess;
    if (kw == NW_FAITH) {
        const FKeyW *k = static_cast<const FKeyW *>(keys);
        FKeyW *ok = static_cast<FKeyW *>(okeys);
        if (op == 0) k_f_rot<true, NW_FAITH><<<grid_for(M, 256), 256, 0, st>>>(d, k, amps, M, ok, oamps, flags);
        else k_f_rot<false, NW_FAITH><<<grid_for(M, 256), 256, 0, st>>>(d, k, amps, M, ok, oamps, flags);
    } else {
        const FKey *k = static_cast<const FKey *>(keys);
        FKey *ok = static_cast<FKey *>(okeys);
        if (op == 0) k_f_rot<true, 2><<<grid_for(M, 256), 256, 0, st>>>(d, k, amps, M, ok, oamps, flags);
        else k_f_rot<false, 2><<<grid_for(M, 256), 256, 0, st>>>(d, k, amps, M, ok, oamps, flags);
    }
    return cudaGetLastError();
}

namespace {
template <int NW, int R>
void launch_hgroups(const QwSimDev &d, const FKeyN<NW> *k, const double2 *amps, const int64_t *starts, int64_t G,
                    uint32_t *cnt, const uint32_t *gpos, FKeyN<NW> *ok, double2 *oamps, int grid, cudaStream_t st)
{
    if (gpos == nullptr) k_f_hgroups<NW, true, R><<<grid, 256, 0, st>>>(d, k, amps, starts, G, cnt, nullptr, nullptr, nullptr);
    else k_f_hgroups<NW, false, R><<<grid, 256, 0, st>>>(d, k, amps, starts, G, cnt, gpos, ok, oamps);
}

/* the fast transform's vector entries a lane: 1 (s <= 32), 2 (64), 4 (128);
   0: the direct sums (s > 128) */
template <int NW>
void launch_hgroups_s(const QwSimDev &d, const void *keys, const double2 *amps, const int64_t *starts, int64_t G,
                      uint32_t *cnt, const uint32_t *gpos, void *okeys, double2 *oamps, int grid, cudaStream_t st)
{
    const FKeyN<NW> *k = static_cast<const FKeyN<NW> *>(keys);
    FKeyN<NW> *ok = static_cast<FKeyN<NW> *>(okeys);
    if (d.s <= 32) launch_hgroups<NW, 1>(d, k, amps, starts, G, cnt, gpos, ok, oamps, grid, st);
    else if (d.s == 64) launch_hgroups<NW, 2>(d, k, amps, starts, G, cnt, gpos, ok, oamps, grid, st);
    else if (d.s == 128) launch_hgroups<NW, 4>(d, k, amps, starts, G, cnt, gpos, ok, oamps, grid, st);
    else launch_hgroups<NW, 0>(d, k, amps, starts, G, cnt, gpos, ok, oamps, grid, st);
}
} // namespace

cudaError_t qw_flat_hgroups(const QwSimDev &d, const void *keys, const double2 *amps, const int64_t *starts, int64_t G,
                            uint32_t *cnt, const uint32_t *gpos, void *okeys, double2 *oamps, cudaStream_t st, int kw)
{
    if (G <= 0) return cudaSuccess;
    const int gpw = d.s < 32 ? 32 / d.s : 1;
    const int grid = grid_for((G + gpw - 1) / gpw * 32, 256);
    if (kw == NW_FAITH) launch_hgroups_s<NW_FAITH>(d, keys, amps, starts, G, cnt, gpos, okeys, oamps, grid, st);
    else launch_hgroups_s<2>(d, keys, amps, starts, G, cnt, gpos, okeys, oamps, grid, st);
    return cudaGetLastError();
}

cudaError_t qw_flat_compact(const void *keys, const double2 *amps, const uint32_t *flags, const uint32_t *pos,
                            int64_t n, void *okeys, double2 *oamps, cudaStream_t st, int kw)
{
    if (n <= 0) return cudaSuccess;
    if (kw == NW_FAITH)
        k_f_compact<NW_FAITH><<<grid_for(n, 256), 256, 0, st>>>(static_cast<const FKeyW *>(keys), amps, flags, pos, n,
                                                                  static_cast<FKeyW *>(okeys), oamps);
    else
        k_f_compact<2><<<grid_for(n, 256), 256, 0, st>>>(static_cast<const FKey *>(keys), amps, flags, pos, n,
                                                           static_cast<FKey *>(okeys), oamps);
    return cudaGetLastError();
}

cudaError_t qw_flat_readout(const QwSimDev &d, const void *keys, const double2 *amps, int64_t M, const QwStepArgs &a,
                            cudaStream_t st, int kw)
{
    if (M <= 0) return cudaSuccess;
    if (kw == NW_FAITH)
        k_f_readout<NW_FAITH><<<grid_for(M, 256), 256, 0, st>>>(d, static_cast<const FKeyW *>(keys), amps, M, a);
    else k_f_readout<2><<<grid_for(M, 256), 256, 0, st>>>(d, static_cast<const FKey *>(keys), amps, M, a);
    return cudaGetLastError();
}

cudaError_t qw_flat_scatter(const QwSimDev &d, const QwBufDev &out, int fp32, const void *keys, const double2 *amps,
                            int64_t M, int32_t *status, unsigned int *maxrow, double *norm, cudaStream_t st, int kw)
{
    if (M <= 0) return cudaSuccess;
    if (kw == NW_FAITH) {
        const FKeyW *k = static_cast<const FKeyW *>(keys);
        if (fp32)
            k_f_scatter<float2, NW_FAITH><<<grid_for(M, 256), 256, 0, st>>>(d, out, k, amps, M, status, maxrow, norm);
        else
            k_f_scatter<double2, NW_FAITH><<<grid_for(M, 256), 256, 0, st>>>(d, out, k, amps, M, status, maxrow, norm);
    } else {
        const FKey *k = static_cast<const FKey *>(keys);
        if (fp32) k_f_scatter<float2, 2><<<grid_for(M, 256), 256, 0, st>>>(d, out, k, amps, M, status, maxrow, norm);
        else k_f_scatter<double2, 2><<<grid_for(M, 256), 256, 0, st>>>(d, out, k, amps, M, status, maxrow, norm);
    }
    return cudaGetLastError();
}

cudaError_t qw_flat_finish(const QwStepArgs &a, const double *norm, const int64_t *counts, cudaStream_t st)
{
    k_f_finish<<<1, 1, 0, st>>>(a, norm, (unsigned long long)counts[0], (unsigned long long)counts[1],
                                (unsigned long long)counts[2], (unsigned long long)counts[3],
                                (unsigned long long)counts[4]);
    return cudaGetLastError();
}

/* register-faithful layout of a simulator: address width and field positions */
static FaithLayout faith_layout(const QwSimDev &d)
{
    FaithLayout F;
    const uint64_t ns = (uint64_t)d.n_single * (uint64_t)d.s;
    const uint64_t top = ns + (((uint64_t)1 << d.nb) * (uint64_t)d.s) + ((uint64_t)1 << d.nb) + 1;
    int b = 0;
    while (((uint64_t)1 << b) < top) b++;
    F.aw = b;
    F.p_addr = 128;
    F.p_left = F.p_addr + b;
    F.p_right = F.p_left + b;
    F.p_mid = F.p_right + b;
    F.p_midval = F.p_mid + b;
    F.p_flag = F.p_midval + 16;
    F.p_cl = F.p_flag + 1;
    F.p_ce = F.p_cl + 1;
    F.p_stk = F.p_ce + 1;
    F.frame = b + 18;
    return F;
}

int qw_faithful_layout(const QwSimDev &d, int *addr_bits, int *layout_bits)
{
    const FaithLayout F = faith_layout(d);
    if (addr_bits) *addr_bits = F.aw;
    const int bits = F.p_stk + (d.L + 1) * F.frame;
    if (layout_bits) *layout_bits = bits;
    return bits <= 64 * NW_FAITH && d.L + 1 <= QW_FQ_FRAMES;
}

cudaError_t qw_faithful_op(const QwSimDev &d, void *keys, int64_t M, int op, int32_t *status, cudaStream_t st)
{
    if (M <= 0) return cudaSuccess;
    const FaithLayout F = faith_layout(d);
    const bool light = op == FQ_ADDR_COL || op == FQ_QRAM_COL || op == FQ_SWAP || op == FQ_ADDR_VAL ||
                       op == FQ_QRAM_VAL;
    if (light && F.p_addr == 128 && F.aw <= 64)
        k_fq_light<<<grid_for(M, 256), 256, 0, st>>>(d, static_cast<FKeyW *>(keys), M, op, F.aw);
    else k_fq<<<grid_for(M, 256), 256, 0, st>>>(d, static_cast<FKeyW *>(keys), M, op, F, status);
    return cudaGetLastError();
}

cudaError_t qw_faithful_export(const QwSimDev &d, const void *keys, int64_t M, uint64_t *table, cudaStream_t st)
{
    if (M <= 0) return cudaSuccess;
    k_fq_export<<<grid_for(M, 256), 256, 0, st>>>(d, static_cast<const FKeyW *>(keys), M, faith_layout(d), table);
    return cudaGetLastError();
}

cudaError_t qw_faithful_check_idle(const QwSimDev &d, const void *keys, int64_t M, int32_t *status, cudaStream_t st)
{
    if (M <= 0) return cudaSuccess;
    k_fq_check_idle<<<grid_for(M, 256), 256, 0, st>>>(static_cast<const FKeyW *>(keys), M, faith_layout(d).p_addr,
                                                       status);
    return cudaGetLastError();
}
