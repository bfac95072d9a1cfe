/*
 * qw_kernels.cu -- sm_103a kernels of the sparse-state quantum walk.
 *
 * The product's walk step W = S T~ P T~^dag (Alg. "Quantum walk operator") is
 * one launch of k_walk.  T~^dag, P and T~ never change the registers
 * (jc, j, b1) and every QRAM read they make (O_A', O_s', QBS) indexes row j,
 * so each (jc, j, b1) row of the state evolves independently until S.  One
 * warp takes the two rows (jc, j, b1 = 0 / 1) of a j: it loads their branches
 * with the row's s QRAM words, runs T~^dag P T~ on chip -- the register maps
 * (semi-quantum ops, Sec. V-A) and the interference ops R^dag, H P H and R
 * (the interference paragraph of Sec. V-A: grouping, per-group transform,
 * pruning), with b2-pairs found by warp matching instead of a sort and H P H
 * folded into R^dag's pass -- then applies S and appends every branch to the
 * bucket of its new row with one atomic per branch.  The HBM traffic of a
 * step is one read and one write of the state.  k_step runs the same step in
 * the paper's literal schedule (every map, H, P, H as three interference ops,
 * a rank sort before each); it is the plain reference schedule on the GPU.
 *
 * Arithmetic: register maps are exact integer work; the prune decision
 * |a|^2 <= tau^2 is taken with un-fused multiplies and adds.  complex128
 * amplitudes: FP64 throughout.  complex64 amplitudes: each rotation output
 * f a0 +- g a1 is formed from error-free products (the FMA-based TwoProduct)
 * and Knuth's error-free TwoSum on the FP32 pipe, with f and g held as float
 * pairs (~48 significant bits), and rounded to FP32 once; the zero-type
 * group sum of H P H is a float-pair accumulation by TwoSum; each lane's norm
 * share adds the FP32-rounded |a|^2 by TwoSum, and the block and grid
 * reductions of the norm, the renormalisation factor, the QLS read-out and
 * p_j are FP64.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/qwalk.h"
#include "qw_internal.h"
#include "qw_device.cuh"

/* Rotation controls carried in the key between a map and its rotation: the
 * element register A (its field of the R layout) and bit 63 = [j > k], the
 * sign sigma = -1 of the rotation for a negative element (sigma = +1 when
 * j <= k).  Both members of a b2-pair carry the same values. */
#define QW_SNEG_BIT 63
/* In the fused kernel a warp runs the rows (jc, j, b1 = 0) and (jc, j, b1 = 1)
 * together -- they read the same QRAM row and nothing before S reads or
 * changes b1 -- with b1 held in this bit of each branch's key. */
#define QW_B1_BIT 52

namespace {

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
                    const double coef = a.qls_coefs[*a.qls_j];
                    double2 acc = a.qls_y[r.j];
                    acc.x += coef * o.x;
                    acc.y += coef * o.y;
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

/* Sort-based step kernel: T~ alone (MODE_T, in place on a bucket range) or a
 * walk step with H, P and H as three interference ops (MODE_WALK_LITERAL). */
/* End of a step: the norm of the output from per-block partial sums.  Every
 * block stores its partial; the last block to finish sums them all -- each
 * thread a fixed strided subset, then a fixed-shape warp and block reduction,
 * so the result does not depend on the order blocks finish -- and publishes
 * the norm, the next step's renormalisation factor and the clean-step count.
 * nv: this warp's partial (any lane); block-uniform control flow. */
__device__ void finish_step(const QwStepArgs &a, double nv, double *block_part, int *is_last, bool count_step)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    nv = warp_sum(nv);
    if (lane == 0) block_part[warp] = nv;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < WARPS; ++w) sum += block_part[w];
        a.partials[blockIdx.x] = sum;
        __threadfence();
        const unsigned prev = atomicAdd(a.done_ctr, 1u);
        *is_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!*is_last) return;
    __threadfence();
    double v = 0.0;
    for (unsigned bb = threadIdx.x; bb < gridDim.x; bb += blockDim.x) v += __ldcg(a.partials + bb);
    v = warp_sum(v);
    if (lane == 0) block_part[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < WARPS; ++w) tot += block_part[w];
        const bool clean = *(volatile int32_t *)a.status == 0;
        if (clean) {
            *a.norm_out = tot;
            if (a.scale_out)
                *a.scale_out = (a.renorm && tot > 0.0) ? sqrt(*a.renorm_target / tot) : 1.0;
            if (a.steps_done) *a.steps_done += 1;
            if (a.stats && count_step) a.stats[QW_STAT_STEPS] += 1;
        }
        *a.done_ctr = 0u;
    }
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
        /* H (end of T~^dag), P, H (start of T~) as three interference ops */
        n = hadamard_op(d, r, kQ, aQ, n, kP, aP, C, a.status, a, true);
        st_h1 += n;
        phase_op(d, r, kP, aP, n);
        n = hadamard_op(d, r, kP, aP, n, kQ, aQ, C, a.status, a, false);
        for (int i = lane; i < n; i += 32) {
            kP[i] = kQ[i];
            aP[i] = aQ[i];
        }
        __syncwarp();
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

    /* ||output||^2 */
    finish_step(a, nrm, block_part, &is_last, MODE != QW_MODE_T);
}

/* per-warp shared memory of the fused kernels: keys x2, amps x2, zero-group
 * buffer, staged QRAM row, partner indices, then (16-byte aligned) the
 * staged rotation values of the row's s slots */
/* In-kernel key of the fused step: b2 (bit 0) | k (nb bits) | kc (nb bits),
 * and the row's b1 as a tag bit; the A register is never held in it (0
 * between steps; the maps return it beside the key).  32-bit keys whenever
 * 1 + 2 nb <= 29 (N <= 16384), which halves the key traffic on chip and keeps
 * the key arithmetic on 32-bit operations; 64-bit keys otherwise. */
template <typename KeyT> struct KeyB1;
template <> struct KeyB1<uint64_t> { static constexpr int bit = QW_B1_BIT; };
template <> struct KeyB1<uint32_t> { static constexpr int bit = 31; };

__host__ __device__ inline bool key32_fits(const QwSimDev &d) { return 1 + 2 * d.nb <= 29; }

/* per-warp shared memory of the fused kernels (byte offsets, 16-byte aligned):
 * keys x2, amplitudes x3 (a pair list holds two per key), the zero-type group (b2 = 0 values, b2 = 1 values,
 * presence), the staged QRAM row, pair-head indices, the row's rotation values */
struct WalkLayout {
    size_t kP, kQ, aP, aQ, aX, zbuf, z1buf, simg, pbuf, hidx, sfg, per_warp;
};

template <typename AmpT, typename KeyT>
__host__ __device__ inline WalkLayout walk_layout(const QwSimDev &d)
{
    WalkLayout o;
    size_t p = 0;
    const size_t C = (size_t)d.warp_cap, s = (size_t)d.s;
#define QW_TAKE(field, bytes)                                                                      \
    o.field = p;                                                                                   \
    p = (p + (bytes) + 15) & ~(size_t)15
    QW_TAKE(kP, C * sizeof(KeyT));
    QW_TAKE(kQ, C * sizeof(KeyT));
    QW_TAKE(aP, C * sizeof(AmpT));
    QW_TAKE(aQ, C * sizeof(AmpT));
    QW_TAKE(aX, C * sizeof(AmpT));
    QW_TAKE(zbuf, s * sizeof(AmpT));
    QW_TAKE(z1buf, s * sizeof(AmpT));
    QW_TAKE(simg, s * sizeof(uint32_t));
    QW_TAKE(pbuf, s * sizeof(int16_t));
    QW_TAKE(hidx, 64 * sizeof(int16_t));
    QW_TAKE(sfg, s * 16);
#undef QW_TAKE
    o.per_warp = p;
    return o;
}

/* ==== fused walk step: one sort per row, b2-pairs kept adjacent ============== */
/*
 * The register maps O_s', O_s'^dag and O_A' never read or write b2, so two
 * branches that differ only in b2 before a map still differ only in b2 after
 * it: b2-pairs are invariant.  The row is sorted once at load (R layout, b2 at
 * bit 0, so pairs become adjacent); every later op keeps pairs adjacent with
 * the b2 = 0 member first, and the rotations find their partner next to them.
 * H P H needs no grouping at all: a branch outside the zero-type groups is
 * only negated, and the zero-type groups are found by a predicate on the key.
 */

/* sign flips as integer operations on the sign bit (keeps FP64 negations
 * and selects off GB300's slow FP64 pipe) */
/* sign flip of an FP64 value as an integer XOR on its high word, kept opaque
   (inline PTX) so that it stays on the integer pipe: an FP64 negation would
   take a slot of GB300's 1/64-rate FP64 pipe */
__device__ __forceinline__ double flip_if(double x, bool neg)
{
    const int m = (int)((unsigned)neg << 31);
    int hi = __double2hiint(x);
    asm("xor.b32 %0, %0, %1;" : "+r"(hi) : "r"(m));
    return __hiloint2double(hi, __double2loint(x));
}
__device__ __forceinline__ float flip_if(float x, bool neg)
{
    return __int_as_float(__float_as_int(x) ^ ((int)neg << 31));
}

template <typename AmpT> struct Amp;

/* complex128 path: FP64 arithmetic throughout */
__device__ __noinline__ double2 scale_c128(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

/* the pruning decision inside the band around tau (rarely reached) */
__device__ __noinline__ bool keep_band(double x, double y, double tau2)
{
    return __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)) > tau2;
}

template <> struct Amp<double2> {
    typedef double2 T;
    static constexpr bool kHeadLanes = true; /* rotate with one lane per pair head */
    struct Norm {
        double v = 0.0;
        __device__ void add(T a) { v = fma(a.x, a.x, fma(a.y, a.y, v)); }
        __device__ double get() const { return v; }
        __device__ double warp_total() const
        {
            double t = v;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
            return t;
        }
    };
    /* sum of a zero-type Hadamard group (FP64) */
    struct Sum {
        double x = 0.0, y = 0.0;
        __device__ void add(T a) { x += a.x; y += a.y; }
        __device__ void set(T a) { x = a.x; y = a.y; } /* add() to an empty sum */
        /* lane t < min(s, 32) holds the partial sums of the values t, t + 32, ...
           (s a power of two); with width < 32 each aligned group of width
           lanes reduces its own values.  Butterfly over the w = min(s, 32) lanes, x on
           lanes t < w/2 and y on lanes t >= w/2 after the first level, so one
           FP64 add serves both components; the same pairs and order as a
           butterfly over each component alone (FP64 addition commutes). */
        __device__ void reduce(int s, int width = 32)
        {
            const int w = s < 32 ? s : 32, h = w >> 1;
            if (h > 0) {
                const bool hy = (lane_id() & h) != 0;
                const double recv = __shfl_xor_sync(FULL, hy ? x : y, h);
                double v = (hy ? y : x) + recv;
                for (int o = h >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
                x = v;
                y = v;
            }
            x = __shfl_sync(FULL, x, 0, width);
            y = __shfl_sync(FULL, y, h, width);
        }
        __device__ void scale_pow2(double f) { x *= f; y *= f; }
        __device__ T minus(T a) const { return make_double2(x - a.x, y - a.y); }
        /* scale_pow2(f) then minus(a) in one FMA per component: f is a power of
           two, so f x is exact and the result is the same rounding */
        __device__ T scaled_minus(double f, T a) const { return make_double2(fma(f, x, -a.x), fma(f, y, -a.y)); }
        __device__ double2 value() const { return make_double2(x, y); }
    };
    __device__ static T zero() { return make_double2(0.0, 0.0); }
    __device__ static T neg(T a) { return make_double2(flip_if(a.x, true), flip_if(a.y, true)); }
    __device__ static double2 to_d(T a) { return a; }
    __device__ static T from_d(double2 a) { return a; }
    /* |a|^2 > tau^2 exactly as the un-fused FP64 formula, decided from the
       exponent bits except in a narrow band around tau; the band's FP64
       arithmetic sits in a call of its own, so that it is not if-converted
       into every call (a predicated-off FP64 instruction still takes its
       slot of the 1/64-rate FP64 pipe) */
    __device__ static bool keep(const QwSimDev &d, T a)
    {
        const uint64_t ux = (uint64_t)__double_as_longlong(a.x) & 0x7fffffffffffffffull;
        const uint64_t uy = (uint64_t)__double_as_longlong(a.y) & 0x7fffffffffffffffull;
        const uint64_t um = ux > uy ? ux : uy;
        if (um > d.tau_hi_bits) return true;
        if (um <= d.tau_lo_bits) return false;
        return keep_band(a.x, a.y, d.tau2);
    }
    struct Scale { /* the renormalisation (off by default for complex128): out of
                      line, so its FP64 products are not if-converted into the
                      loads that do not rescale */
        double s;
        __device__ explicit Scale(double v) : s(v) {}
        __device__ T apply(T a) const { return scale_c128(a, s); }
        /* staged once per block (the factor in 8 bytes of shared memory) */
        __device__ static void to_shared(double v, double *buf) { buf[0] = v; }
        __device__ static Scale from_shared(const double *buf) { return Scale(buf[0]); }
    };
    typedef double2 RotVal; /* (sqrt|a|, sqrt(1-|a|)) */
    __device__ static RotVal rot_table(const QwSimDev &d, uint32_t A) { return __ldg(d.fg + A); }
    __device__ static RotVal rot_zero() { return make_double2(0.0, 1.0); }
    static constexpr bool kRotCode = false; /* FP64 square roots: read the table */
    __device__ static RotVal rot_code(uint32_t) { return rot_zero(); }
    __device__ static void rot(RotVal t, uint32_t A, bool dag, bool sneg, T a0, T a1, T &o0, T &o1);
    /* rot(t, A, true, sneg, a0, 0): R^dag of a pair whose b2 = 1 member is 0 */
    __device__ static void rot_dag_b2zero(RotVal t, uint32_t A, bool sneg, T a0, T &o0, T &o1);
    static constexpr bool kB2ZeroPath = true;
};

/* complex64 path: amplitudes are float; each rotation output f a0 +- g a1 is
   formed from error-free products and an error-free sum on the FP32 pipe
   (f, g held as float pairs with ~48 significant bits) and rounded once. */
template <> struct Amp<float2> {
    typedef float2 T;
    static constexpr bool kHeadLanes = false;
    struct Norm { /* |a|^2 rounded to FP32 once per branch (relative 2^-24), then
                     summed by TwoSum into a float pair, so the sum adds no
                     rounding error of note beyond those per-term roundings */
        float hi = 0.f, lo = 0.f;
        __device__ void add(T a)
        {
            const float v = __fadd_rn(__fmul_rn(a.x, a.x), __fmul_rn(a.y, a.y));
            const float s = __fadd_rn(hi, v);
            const float bp = __fsub_rn(s, hi);
            lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(v, bp)));
            hi = s;
        }
        __device__ double get() const { return (double)hi + (double)lo; }
        /* the warp's sum: a butterfly of float-pair additions, one conversion
           to FP64 on the lane that returns it (lane 0; the others return 0) */
        __device__ double warp_total() const;
    };
    /* float-pair (hi + lo) accumulator built from Knuth's TwoSum (the sum and
       its exact rounding error), ~48 significant bits */
    struct DF {
        float h = 0.f, l = 0.f;
        __device__ void add(float v)
        {
            const float s = __fadd_rn(h, v);
            const float bp = __fsub_rn(s, h);
            const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(v, bp));
            h = s;
            l = __fadd_rn(l, e);
        }
        __device__ void add(float vh, float vl)
        {
            add(vh);
            l = __fadd_rn(l, vl);
            const float s = __fadd_rn(h, l); /* renormalise: |l| small */
            l = __fsub_rn(l, __fsub_rn(s, h));
            h = s;
        }

        /* round(h + l - v) */
        __device__ float minus(float v) const
        {
            const float s = __fsub_rn(h, v);
            const float bp = __fsub_rn(s, h);
            const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(-v, bp));
            return __fadd_rn(s, __fadd_rn(e, l));
        }
    };
    /* sum of a zero-type Hadamard group of FP32 terms in a float pair: its
       error is of order 2^-46 times the sum of the terms' magnitudes */
    struct Sum {
        DF x, y;
        __device__ void add(T a) { x.add(a.x); y.add(a.y); }
        __device__ void set(T a) /* add() to an empty sum: the value, no error term */
        {
            x.h = a.x;
            x.l = 0.f;
            y.h = a.y;
            y.l = 0.f;
        }
        /* lane t < min(s, 32) holds the partial sums of the values t, t + 32, ...
           (s a power of two); with width < 32 each aligned group of width
           lanes reduces its own values.  Butterfly over the w = min(s, 32) lanes, x on
           lanes t < w/2 and y on lanes t >= w/2 after the first level (where a
           y lane adds its own pair to its partner's, the order the partner
           would use), so one float-pair add serves both components. */
        __device__ void reduce(int s, int width = 32)
        {
            const int w = s < 32 ? s : 32, h = w >> 1;
            if (h > 0) {
                const bool hy = (lane_id() & h) != 0;
                const float rh = __shfl_xor_sync(FULL, hy ? x.h : y.h, h);
                const float rl = __shfl_xor_sync(FULL, hy ? x.l : y.l, h);
                DF v;
                if (hy) { /* partner's y, then own y */
                    v.h = rh;
                    v.l = rl;
                    v.add(y.h, y.l);
                } else {
                    v = x;
                    v.add(rh, rl);
                }
                for (int o = h >> 1; o > 0; o >>= 1) {
                    const float oh = __shfl_xor_sync(FULL, v.h, o), ol = __shfl_xor_sync(FULL, v.l, o);
                    v.add(oh, ol);
                }
                x = v;
                y = v;
            }
            x.h = __shfl_sync(FULL, x.h, 0, width);
            x.l = __shfl_sync(FULL, x.l, 0, width);
            y.h = __shfl_sync(FULL, y.h, h, width);
            y.l = __shfl_sync(FULL, y.l, h, width);
        }
        __device__ void scale_pow2(double f)
        {
            const float g = (float)f; /* 2/s: a power of two, exact */
            x.h *= g; x.l *= g; y.h *= g; y.l *= g;
        }
        __device__ T minus(T a) const { return make_float2(x.minus(a.x), y.minus(a.y)); }
        __device__ T scaled_minus(double f, T a) const
        {
            Sum c = *this;
            c.scale_pow2(f);
            return c.minus(a);
        }
        __device__ double2 value() const
        {
            return make_double2((double)x.h + (double)x.l, (double)y.h + (double)y.l);
        }
    };
    __device__ static T zero() { return make_float2(0.f, 0.f); }
    __device__ static T neg(T a) { return make_float2(-a.x, -a.y); }
    __device__ static double2 to_d(T a) { return make_double2((double)a.x, (double)a.y); }
    __device__ static T from_d(double2 a) { return make_float2((float)a.x, (float)a.y); }
    __device__ static bool keep(const QwSimDev &d, T a)
    {
        return __fadd_rn(__fmul_rn(a.x, a.x), __fmul_rn(a.y, a.y)) > d.tau2f;
    }
    /* a * s with s = sh + sl, rounded once */
    __device__ static float mul_split(float a, float sh, float sl)
    {
        const float p = __fmul_rn(sh, a);
        float e = __fmaf_rn(sh, a, -p);
        e = __fmaf_rn(sl, a, e);
        return __fadd_rn(p, e);
    }
    struct Scale { /* the FP64 factor as a float pair, applied with one rounding */
        float sh, sl;
        __device__ explicit Scale(double v) : sh((float)v), sl((float)(v - (double)(float)v)) {}
        __device__ Scale(float h, float l) : sh(h), sl(l) {}
        __device__ T apply(T a) const { return make_float2(mul_split(a.x, sh, sl), mul_split(a.y, sh, sl)); }
        /* the split computed once per block (its FP64 conversions would
           otherwise take a slot of the 1/64-rate FP64 pipe in every thread) */
        __device__ static void to_shared(double v, double *buf)
        {
            float *f = reinterpret_cast<float *>(buf);
            f[0] = (float)v;
            f[1] = (float)(v - (double)(float)v);
        }
        __device__ static Scale from_shared(const double *buf)
        {
            const float *f = reinterpret_cast<const float *>(buf);
            return Scale(f[0], f[1]);
        }
    };
    /* round(A x + B y), A = ah + al, B = bh + bl: the products by the FMA-based
       TwoProduct (p = fl(a b), e = fma(a, b, -p) exact), their sum by Knuth's
       TwoSum, the low parts added to the error term, one final rounding */
    __device__ static float dot2(float ah, float al, float x, float bh, float bl, float y)
    {
        const float p1 = __fmul_rn(ah, x);
        float e1 = __fmaf_rn(ah, x, -p1);
        e1 = __fmaf_rn(al, x, e1);
        const float p2 = __fmul_rn(bh, y);
        float e2 = __fmaf_rn(bh, y, -p2);
        e2 = __fmaf_rn(bl, y, e2);
        const float s = __fadd_rn(p1, p2);
        const float bp = __fsub_rn(s, p1);
        const float t = __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bp)), __fsub_rn(p2, bp));
        return __fadd_rn(s, __fadd_rn(t, __fadd_rn(e1, e2)));
    }
    typedef float4 RotVal; /* (sqrt|a|, sqrt(1-|a|)) as float pairs */
    __device__ static RotVal rot_table(const QwSimDev &d, uint32_t A) { return __ldg(d.fg32 + A); }
    /* the table entry of code A (rot_bits = 0) computed in place: hi the
       correctly rounded square root, lo the Newton correction (x - hi^2) /
       (2 hi) with the residual exact by FMA -- the host builds the table the
       same way, so the bits agree */
    static constexpr bool kRotCode = true;
    __device__ static RotVal rot_code(uint32_t A)
    {
        const int q = (int)(int16_t)(uint16_t)A;
        const float x = (float)(q < 0 ? -q : q) * (1.0f / 32768.0f), y = 1.0f - x;
        const float fh = __fsqrt_rn(x), gh = __fsqrt_rn(y);
        const float fl = fh > 0.0f ? __fdiv_rn(__fmaf_rn(-fh, fh, x), 2.0f * fh) : 0.0f;
        const float gl = gh > 0.0f ? __fdiv_rn(__fmaf_rn(-gh, gh, y), 2.0f * gh) : 0.0f;
        return make_float4(fh, fl, gh, gl);
    }
    __device__ static RotVal rot_zero() { return make_float4(0.f, 0.f, 1.f, 0.f); }
    __device__ static void rot(RotVal t, uint32_t A, bool dag, bool sneg, T a0, T a1, T &o0, T &o1);
    __device__ static void rot_dag_b2zero(RotVal t, uint32_t A, bool sneg, T a0, T &o0, T &o1);
    static constexpr bool kB2ZeroPath = false;
    /* dot2 with y = 0: round(A x) -- the same bits (p1 + e1 rounded once) */
    __device__ static float dot1(float ah, float al, float x)
    {
        const float p1 = __fmul_rn(ah, x);
        float e1 = __fmaf_rn(ah, x, -p1);
        e1 = __fmaf_rn(al, x, e1);
        return __fadd_rn(p1, e1);
    }
};

__device__ double Amp<float2>::Norm::warp_total() const
{
    DF v;
    v.h = hi;
    v.l = lo;
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(FULL, v.h, o), ol = __shfl_xor_sync(FULL, v.l, o);
        v.add(oh, ol);
    }
    return lane_id() == 0 ? (double)v.h + (double)v.l : 0.0;
}

/* multiply by 1 (real f) or by i*sigma (imaginary f), sigma = sneg ? -1 : 1:
 * i sigma (x + i y) = -sigma y + i sigma x */
template <typename T>
__device__ __forceinline__ T rho(T a, bool imag, bool sneg)
{
    T r;
    r.x = imag ? flip_if(a.y, !sneg) : a.x;
    r.y = imag ? flip_if(a.x, sneg) : a.y;
    return r;
}

/* R:    o0 = f a0 - g a1,        o1 = g a0 + conj(f) a1
 * R^dag: o0 = conj(f) a0 + g a1, o1 = f a1 - g a0
 * with f = fm (a >= 0) or i sigma fm (a < 0): f x = fm rho(x, sigma),
 * conj(f) x = fm rho(x, -sigma). */
__device__ void Amp<double2>::rot(RotVal t, uint32_t A, bool dag, bool sneg, T a0, T a1, T &o0, T &o1)
{
    const double fm = t.x, g = t.y;
    const bool imag = (int16_t)(uint16_t)A < 0;
    const double2 x0 = rho(a0, imag, dag ? !sneg : sneg);
    const double2 x1 = rho(a1, imag, dag ? sneg : !sneg);
    if (!dag) {
        o0 = make_double2(fma(fm, x0.x, -g * a1.x), fma(fm, x0.y, -g * a1.y));
        o1 = make_double2(fma(g, a0.x, fm * x1.x), fma(g, a0.y, fm * x1.y));
    } else {
        o0 = make_double2(fma(fm, x0.x, g * a1.x), fma(fm, x0.y, g * a1.y));
        o1 = make_double2(fma(fm, x1.x, -g * a0.x), fma(fm, x1.y, -g * a0.y));
    }
}

/* R^dag (a0, 0): o0 = conj(f) a0, o1 = -g a0 -- the general formulas with
   a1 = 0, whose products by 0 change no rounding */
__device__ void Amp<double2>::rot_dag_b2zero(RotVal t, uint32_t A, bool sneg, T a0, T &o0, T &o1)
{
    const double fm = t.x, g = t.y;
    const bool imag = (int16_t)(uint16_t)A < 0;
    const double2 x0 = rho(a0, imag, !sneg);
    o0 = make_double2(fm * x0.x, fm * x0.y);
    o1 = make_double2(-g * a0.x, -g * a0.y);
}

__device__ void Amp<float2>::rot_dag_b2zero(RotVal t, uint32_t A, bool sneg, T a0, T &o0, T &o1)
{
    const bool imag = (int16_t)(uint16_t)A < 0;
    const float2 x0 = rho(a0, imag, !sneg);
    o0 = make_float2(dot1(t.x, t.y, x0.x), dot1(t.x, t.y, x0.y));
    o1 = make_float2(dot1(-t.z, -t.w, a0.x), dot1(-t.z, -t.w, a0.y));
}

__device__ void Amp<float2>::rot(RotVal t, uint32_t A, bool dag, bool sneg, T a0, T a1, T &o0, T &o1)
{
    /* t = (fh, fl, gh, gl) */
    const bool imag = (int16_t)(uint16_t)A < 0;
    const float2 x0 = rho(a0, imag, dag ? !sneg : sneg);
    const float2 x1 = rho(a1, imag, dag ? sneg : !sneg);
    if (!dag) {
        o0 = make_float2(dot2(t.x, t.y, x0.x, -t.z, -t.w, a1.x), dot2(t.x, t.y, x0.y, -t.z, -t.w, a1.y));
        o1 = make_float2(dot2(t.z, t.w, a0.x, t.x, t.y, x1.x), dot2(t.z, t.w, a0.y, t.x, t.y, x1.y));
    } else {
        o0 = make_float2(dot2(t.x, t.y, x0.x, t.z, t.w, a1.x), dot2(t.x, t.y, x0.y, t.z, t.w, a1.y));
        o1 = make_float2(dot2(t.x, t.y, x1.x, -t.z, -t.w, a0.x), dot2(t.x, t.y, x1.y, -t.z, -t.w, a0.y));
    }
}

/* Pair up to 32 branches held one per lane (valid lanes carry distinct keys):
 * b2-partners (keys equal but for bit 0) become adjacent, b2 = 0 first, in
 * kd/ad from position base on.  Returns the number of valid branches. */
template <typename AmpT, typename KeyT>
__device__ int pair32(KeyT k, AmpT a, bool valid, KeyT *kd, AmpT *ad, int base)
{
    const int lane = lane_id();
    /* inactive lanes get keys whose k >> 1 are distinct and above every real
       key (real keys stay below the b1 tag bit plus 2^(1 + 2 nb)) */
    if (!valid) k = (KeyT)~(KeyT)0 - (KeyT)(2 * lane);
    const unsigned m = __match_any_sync(FULL, (KeyT)(k >> 1));
    const unsigned other = m & ~(1u << lane);
    const bool head = valid && ((k & 1) == 0 || other == 0);
    const int cnt = head ? (other ? 2 : 1) : 0;
    int total;
    const int pos = base + warp_compact2(head, cnt == 2, total);
    const int src = other ? (__ffs(other) - 1) : lane;
    const KeyT pk = __shfl_sync(FULL, k, src);
    AmpT pa;
    pa.x = __shfl_sync(FULL, a.x, src);
    pa.y = __shfl_sync(FULL, a.y, src);
    if (head) {
        kd[pos] = k;
        ad[pos] = a;
        if (cnt == 2) {
            kd[pos + 1] = pk;
            ad[pos + 1] = pa;
        }
    }
    return total;
}

/* A stored branch (R layout, 64 bits) as an in-kernel key: b2 | k | kc plus
 * the b1 tag; A (bits ash..) must be 0 and is reported through anc if not. */
template <typename KeyT>
__device__ __forceinline__ KeyT in_key(uint64_t raw, int ash, KeyT tag, uint64_t &anc)
{
    anc |= raw >> ash;
    return (KeyT)(raw & ((1ull << ash) - 1)) | tag;
}

/* Load the nr branches of bucket b (b1 tag `tag`) and pair them into kd/ad
 * from position base on.  nr <= 32: one warp match.  nr <= 64 (and a scratch
 * of >= 64 entries): split the row in two halves of <= 32 by one key bit
 * above b2 (partners share every such bit), then one match per half.
 * Otherwise (or if no bit splits the row evenly enough) sort by key: the rank
 * of each key among the row's.  (have, hraw, ha): the row's first 32 stored
 * branches, loaded ahead. */
template <typename AmpT, typename KeyT>
__device__ void pair_row(const QwBufDev &in, int64_t b, int nr, KeyT tag, int cap_row, int ash, bool rescale,
                         const typename Amp<AmpT>::Scale &scale, KeyT *kd, AmpT *ad, int base, KeyT *ktmp,
                         AmpT *atmp, int cap, bool have, uint64_t hraw, AmpT ha, uint64_t &anc)
{
    const int lane = lane_id();
    const AmpT *amp = static_cast<const AmpT *>(in.amp);
    const int64_t row0 = b * (int64_t)cap_row;
    auto fetch = [&](int i, KeyT &k, AmpT &a) {
        k = in_key<KeyT>(in.key[row0 + i], ash, tag, anc);
        a = amp[row0 + i];
        if (rescale) a = scale.apply(a);
    };
    if (nr <= 32 || (nr <= 64 && cap >= 64)) {
        KeyT k0 = 0, k1 = 0;
        AmpT a0 = Amp<AmpT>::zero(), a1 = Amp<AmpT>::zero();
        const bool v0 = lane < nr, v1 = lane + 32 < nr;
        if (v0) {
            if (have) {
                k0 = in_key<KeyT>(hraw, ash, tag, anc);
                a0 = rescale ? scale.apply(ha) : ha;
            } else {
                fetch(lane, k0, a0);
            }
        }
        if (v1) fetch(lane + 32, k1, a1);
        if (nr <= 32) {
            pair32<AmpT, KeyT>(k0, a0, v0, kd, ad, base);
            __syncwarp();
            return;
        }
        constexpr int KB = 8 * (int)sizeof(KeyT);
        int t = 1;
        int c0 = 0;
        for (; t < KB - 1; ++t) {
            const bool z0 = v0 && ((k0 >> t) & 1) == 0;
            const bool z1 = v1 && ((k1 >> t) & 1) == 0;
            c0 = __popc(__ballot_sync(FULL, z0)) + __popc(__ballot_sync(FULL, z1));
            if (c0 <= 32 && nr - c0 <= 32) break;
        }
        if (t < KB - 1) {
            /* halves: bit t = 0 to ktmp[0, c0), bit t = 1 to ktmp[32, 32 + nr - c0) */
            const bool z0 = ((k0 >> t) & 1) == 0, z1 = ((k1 >> t) & 1) == 0;
            const unsigned lt = (1u << lane) - 1u;
            const unsigned bz0 = __ballot_sync(FULL, v0 && z0), bz1 = __ballot_sync(FULL, v1 && z1);
            const unsigned bo0 = __ballot_sync(FULL, v0 && !z0), bo1 = __ballot_sync(FULL, v1 && !z1);
            if (v0) {
                const int q = z0 ? __popc(bz0 & lt) : 32 + __popc(bo0 & lt);
                ktmp[q] = k0;
                atmp[q] = a0;
            }
            if (v1) {
                const int q = z1 ? __popc(bz0) + __popc(bz1 & lt) : 32 + __popc(bo0) + __popc(bo1 & lt);
                ktmp[q] = k1;
                atmp[q] = a1;
            }
            __syncwarp();
            const bool w0 = lane < c0, w1 = lane < nr - c0;
            const KeyT h0 = w0 ? ktmp[lane] : (KeyT)0, h1 = w1 ? ktmp[32 + lane] : (KeyT)0;
            const AmpT g0 = w0 ? atmp[lane] : Amp<AmpT>::zero();
            const AmpT g1 = w1 ? atmp[32 + lane] : Amp<AmpT>::zero();
            __syncwarp();
            const int m0 = pair32<AmpT, KeyT>(h0, g0, w0, kd, ad, base);
            pair32<AmpT, KeyT>(h1, g1, w1, kd, ad, base + m0);
            __syncwarp();
            return;
        }
        /* no balanced bit: fall through to the sort (the row reloads) */
    }
    for (int i = lane; i < nr; i += 32) {
        KeyT k;
        AmpT v;
        fetch(i, k, v);
        ktmp[i] = k;
        atmp[i] = v;
    }
    __syncwarp();
    for (int i = lane; i < nr; i += 32) {
        const KeyT ki = ktmp[i];
        int r = 0;
        for (int t = 0; t < nr; ++t) r += (ktmp[t] < ki);
        kd[base + r] = ki;
        ad[base + r] = atmp[i];
    }
    __syncwarp();
}

/* Load a segment -- the n0 branches of bucket A (b1 = tagA) and the n1 of
 * bucket B (b1 = 1) -- and group it: b2-pairs next to each other, b2 = 0
 * first.  Partners never straddle the two rows (they differ in b2 only), so a
 * segment that fits one warp is matched at once and a longer one row by row;
 * (have, hraw, ha) are the segment's first 32 stored branches (A's, then
 * B's), loaded ahead by the pipelined loop.  A stored key with A != 0 sets
 * the ancilla status bit. */
template <typename AmpT, typename KeyT>
__device__ void load_seg(const QwSimDev &d, const QwBufDev &in, int64_t bA, int n0, KeyT tagA, int64_t bB,
                         int n1, bool rescale, const typename Amp<AmpT>::Scale &scale, KeyT *kd, AmpT *ad,
                         KeyT *ktmp, AmpT *atmp, int cap, bool have, uint64_t hraw, AmpT ha, int32_t *status)
{
    const int lane = lane_id();
    const int ash = 1 + 2 * d.nb;
    const KeyT tagB = (KeyT)1 << KeyB1<KeyT>::bit;
    const int n = n0 + n1;
    uint64_t anc = 0;
    if (n <= 32) { /* both rows in one warp match (the b1 tag keeps them apart) */
        KeyT k = 0;
        AmpT a = Amp<AmpT>::zero();
        if (lane < n0) {
            const int64_t slot = bA * (int64_t)d.cap_row + lane;
            k = in_key<KeyT>(have ? hraw : in.key[slot], ash, tagA, anc);
            a = have ? ha : static_cast<const AmpT *>(in.amp)[slot];
        } else if (lane < n) {
            const int64_t slot = bB * (int64_t)d.cap_row + (lane - n0);
            k = in_key<KeyT>(have ? hraw : in.key[slot], ash, tagB, anc);
            a = have ? ha : static_cast<const AmpT *>(in.amp)[slot];
        }
        if (rescale && lane < n) a = scale.apply(a);
        pair32<AmpT, KeyT>(k, a, lane < n, kd, ad, 0);
        __syncwarp();
    } else {
        if (n0 > 0)
            pair_row<AmpT, KeyT>(in, bA, n0, tagA, d.cap_row, ash, rescale, scale, kd, ad, 0, ktmp, atmp, cap,
                                 have, hraw, ha, anc);
        if (n1 > 0)
            pair_row<AmpT, KeyT>(in, bB, n1, tagB, d.cap_row, ash, rescale, scale, kd, ad, n0, ktmp, atmp, cap,
                                 false, 0ull, Amp<AmpT>::zero(), anc);
    }
    if (__any_sync(FULL, anc != 0) && lane == 0) atomicOr(status, QW_ST_ANCILLA);
}


template <typename KeyT>
__device__ __forceinline__ KeyT map_tdag(const QwSimDev &d, const Row &r, KeyT key, uint32_t &slot, uint32_t &A,
                                         bool &sneg);
template <typename KeyT>
__device__ __forceinline__ KeyT map_t(const QwSimDev &d, const Row &r, KeyT key, uint32_t &slot, uint32_t &A,
                                      bool &sneg);

/* The pair headed by key k (b2 = 0 member amplitude a0, b2 = 1 member a1,
 * zero where absent): the register maps of one half-step on the key, then
 * R^dag (WHICH = 0, T~^dag) or R (WHICH = 1, T~).  The maps never read b2,
 * so the head maps the key once for both members; the rotation is controlled
 * by A and sigma, which the maps return beside the key.  Outputs o0 (b2 = 0)
 * and o1 (b2 = 1) under kb (b2 = 0, the b1 tag kept), and whether each is
 * kept by the pruning rule. */
template <int WHICH, typename AmpT, typename KeyT>
__device__ __forceinline__ void rot_head(const QwSimDev &d, const Row &r, KeyT k, AmpT a0, AmpT a1, AmpT &o0,
                                         AmpT &o1, bool &c0, bool &c1, KeyT &kb)
{
    const KeyT b1bit = k & ((KeyT)1 << KeyB1<KeyT>::bit);
    const KeyT key = k & ~((KeyT)1 | b1bit);
    uint32_t slot, A;
    bool sneg;
    const KeyT mk = (WHICH == 0) ? map_tdag<KeyT>(d, r, key, slot, A, sneg) : map_t<KeyT>(d, r, key, slot, A, sneg);
    /* A is 0 or the value of slot `slot` of row j: staged rotation values for
       a slot of this row, the per-code table otherwise */
    typename Amp<AmpT>::RotVal t;
    if (A == 0) t = Amp<AmpT>::rot_zero();
    else if (slot < (uint32_t)d.s && r.sfg) t = static_cast<const typename Amp<AmpT>::RotVal *>(r.sfg)[slot];
    else t = Amp<AmpT>::rot_table(d, A);
    Amp<AmpT>::rot(t, A, WHICH == 0, sneg, a0, a1, o0, o1);
    c0 = Amp<AmpT>::keep(d, o0);
    c1 = Amp<AmpT>::keep(d, o1);
    kb = mk | b1bit;
}

/* Appends rotated pairs to a warp buffer, pair-adjacent (b2 = 0 first), kept
 * outputs only.  REFL: H P H folded in -- k_high | kc | b1 all zero in a row
 * with jc = 0 marks the zero-type Hadamard group (b2 = 0: set aside in zbuf
 * for the reflection; b2 = 1: negated, set aside beside it); every other
 * output is negated here.  Called by all lanes of the warp together. */
template <typename AmpT, typename KeyT, bool REFL>
struct PairSink {
    KeyT *kd;
    AmpT *ad;
    int cap, out, div;
    KeyT zm;
    bool rowzero;
    int smask;
    AmpT *zbuf, *z1buf;
    int16_t *pbuf;
    __device__ PairSink(const QwSimDev &d, const Row &r, KeyT *kd_, AmpT *ad_, int cap_, AmpT *zb, AmpT *z1b,
                        int16_t *pb)
        : kd(kd_), ad(ad_), cap(cap_), out(0), div(0), smask(d.s - 1), zbuf(zb), z1buf(z1b), pbuf(pb)
    {
        const int ash = 1 + 2 * d.nb;
        zm = ((((KeyT)1 << ash) - 1) & ~(((KeyT)1 << (d.L + 1)) - 1)) | ((KeyT)1 << KeyB1<KeyT>::bit);
        rowzero = REFL && r.jc == 0;
    }
    __device__ __forceinline__ void put(bool head, KeyT kb, AmpT o0, AmpT o1, bool c0, bool c1)
    {
        if (REFL) {
            const bool zt = head && rowzero && (kb & zm) == 0;
            div += __popc(__ballot_sync(FULL, zt && c0)) + __popc(__ballot_sync(FULL, zt && c1));
            if (zt) {
                const int u = (int)((kb >> 1) & (KeyT)smask);
                if (c0) zbuf[u] = o0;
                if (c1) {
                    z1buf[u] = Amp<AmpT>::neg(o1);
                    pbuf[u] = 1;
                }
                c0 = c1 = false;
            } else {
                o0 = Amp<AmpT>::neg(o0);
                o1 = Amp<AmpT>::neg(o1);
            }
        }
        int total;
        int pos = out + warp_compact2(c0, c1, total);
        if (c0) {
            if (pos < cap) { kd[pos] = kb; ad[pos] = o0; }
            pos++;
        }
        if (c1) {
            if (pos < cap) { kd[pos] = kb | (KeyT)1; ad[pos] = o1; }
        }
        out += total;
    }
};

/* The same outputs as PairSink, as a pair list: one entry per pair with a
 * kept member -- key kb (b2 = 0), the b2 = 0 and b2 = 1 amplitudes, zero for a
 * member that is absent (a kept amplitude is never zero: it exceeds tau).
 * elems counts the kept branches. */
template <typename AmpT, typename KeyT, bool REFL>
struct PairListSink {
    KeyT *kd;
    AmpT *a0d, *a1d;
    int cap, out, div, elems;
    KeyT zm;
    bool rowzero;
    int smask;
    AmpT *zbuf, *z1buf;
    int16_t *pbuf;
    __device__ PairListSink(const QwSimDev &d, const Row &r, KeyT *kd_, AmpT *a0_, AmpT *a1_, int cap_, AmpT *zb,
                            AmpT *z1b, int16_t *pb)
        : kd(kd_), a0d(a0_), a1d(a1_), cap(cap_), out(0), div(0), elems(0), smask(d.s - 1), zbuf(zb), z1buf(z1b),
          pbuf(pb)
    {
        const int ash = 1 + 2 * d.nb;
        zm = ((((KeyT)1 << ash) - 1) & ~(((KeyT)1 << (d.L + 1)) - 1)) | ((KeyT)1 << KeyB1<KeyT>::bit);
        rowzero = REFL && r.jc == 0;
    }
    __device__ __forceinline__ void put(bool head, KeyT kb, AmpT o0, AmpT o1, bool c0, bool c1)
    {
        if (REFL) {
            const bool zt = head && rowzero && (kb & zm) == 0;
            div += __popc(__ballot_sync(FULL, zt && c0)) + __popc(__ballot_sync(FULL, zt && c1));
            if (zt) {
                const int u = (int)((kb >> 1) & (KeyT)smask);
                if (c0) zbuf[u] = o0;
                if (c1) {
                    z1buf[u] = Amp<AmpT>::neg(o1);
                    pbuf[u] = 1;
                }
                c0 = c1 = false;
            } else {
                o0 = Amp<AmpT>::neg(o0);
                o1 = Amp<AmpT>::neg(o1);
            }
        }
        const bool any = c0 || c1;
        const unsigned m = __ballot_sync(FULL, any);
        elems += __popc(__ballot_sync(FULL, c0)) + __popc(__ballot_sync(FULL, c1));
        if (any) {
            const int pos = out + __popc(m & ((1u << lane_id()) - 1u));
            if (pos < cap) {
                kd[pos] = kb;
                a0d[pos] = c0 ? o0 : Amp<AmpT>::zero();
                a1d[pos] = c1 ? o1 : Amp<AmpT>::zero();
            }
        }
        out += __popc(m);
    }
};

/* One half-step over a pair list of np entries: one lane per pair. */
template <int WHICH, typename AmpT, typename KeyT, typename Sink>
__device__ void map_rot_list(const QwSimDev &d, const Row &r, const KeyT *ks, const AmpT *a0s, const AmpT *a1s,
                             int np, Sink &sink)
{
    for (int base = 0; base < np; base += 32) {
        const int p = base + lane_id();
        const bool head = p < np;
        AmpT o0 = Amp<AmpT>::zero(), o1 = Amp<AmpT>::zero();
        bool c0 = false, c1 = false;
        KeyT kb = 0;
        if (head) rot_head<WHICH, AmpT, KeyT>(d, r, ks[p], a0s[p], a1s[p], o0, o1, c0, c1, kb);
        sink.put(head, kb, o0, o1, c0, c1);
    }
    __syncwarp();
}

/* One half-step (maps + rotation) over a warp buffer of n branches with
 * b2-pairs adjacent: each pair head (a b2 = 0 branch, or a b2 = 1 one
 * without its partner) rotates both members; the outputs go to the sink. */
template <int WHICH, typename AmpT, typename KeyT, typename Sink>
__device__ void map_rot_pairs(const QwSimDev &d, const Row &r, const KeyT *ks, const AmpT *as, int n, Sink &sink,
                              int16_t *hidx)
{
    const int lane = lane_id();
    auto pair_at = [&](int i, bool head) {
        AmpT o0 = Amp<AmpT>::zero(), o1 = Amp<AmpT>::zero();
        bool c0 = false, c1 = false;
        KeyT kb = 0;
        if (head) {
            const KeyT k = ks[i];
            AmpT a0 = Amp<AmpT>::zero(), a1 = Amp<AmpT>::zero();
            if ((k & (KeyT)1) == 0) {
                a0 = as[i];
                if (i + 1 < n && ks[i + 1] == (k | (KeyT)1)) a1 = as[i + 1];
            } else {
                a1 = as[i];
            }
            rot_head<WHICH, AmpT, KeyT>(d, r, k, a0, a1, o0, o1, c0, c1, kb);
        }
        sink.put(head, kb, o0, o1, c0, c1);
    };
    auto is_head = [&](int i) {
        return i < n && !(i > 0 && ks[i - 1] == (ks[i] ^ (KeyT)1));
    };
    if (Amp<AmpT>::kHeadLanes) {
        /* blocks of 64 branches: list the heads, then one lane per head, so no
           lane idles through the (FP64) rotation for a pair's second member */
        const unsigned lt = (1u << lane) - 1u;
        for (int base = 0; base < n; base += 64) {
            int nh = 0;
            for (int half = 0; half < 64; half += 32) {
                const int i = base + half + lane;
                const bool head = is_head(i);
                const unsigned hm = __ballot_sync(FULL, head);
                if (head) hidx[nh + __popc(hm & lt)] = (int16_t)i;
                nh += __popc(hm);
            }
            __syncwarp();
            for (int hb = 0; hb < nh; hb += 32) {
                const bool head = hb + lane < nh;
                pair_at(head ? hidx[hb + lane] : 0, head);
            }
            __syncwarp();
        }
    } else {
        for (int base = 0; base < n; base += 32) pair_at(base + lane, is_head(base + lane));
        __syncwarp();
    }
}

/* T~^dag on up to 32 loaded branches held one per lane (valid lanes carry
 * distinct keys): b2-partners found by a warp match on key >> 1, the head of
 * each pair takes its partner's amplitude by a shuffle and rotates both. */
template <typename AmpT, typename KeyT, typename Sink>
__device__ __forceinline__ void rot0_chunk(const QwSimDev &d, const Row &r, KeyT k, AmpT a, bool valid, Sink &sink)
{
    const int lane = lane_id();
    if (!valid) k = (KeyT)~(KeyT)0 - (KeyT)(2 * lane); /* distinct k >> 1 above every real key */
    const unsigned m = __match_any_sync(FULL, (KeyT)(k >> 1));
    const unsigned other = m & ~(1u << lane);
    const bool b2one = (k & (KeyT)1) != 0;
    const bool head = valid && (!b2one || other == 0);
    const int src = other ? (__ffs(other) - 1) : lane;
    AmpT pa;
    pa.x = __shfl_sync(FULL, a.x, src);
    pa.y = __shfl_sync(FULL, a.y, src);
    AmpT o0 = Amp<AmpT>::zero(), o1 = Amp<AmpT>::zero();
    bool c0 = false, c1 = false;
    KeyT kb = 0;
    if (head) {
        const AmpT a0 = b2one ? Amp<AmpT>::zero() : a;
        const AmpT a1 = b2one ? a : (other ? pa : Amp<AmpT>::zero());
        rot_head<0, AmpT, KeyT>(d, r, k, a0, a1, o0, o1, c0, c1, kb);
    }
    sink.put(head, kb, o0, o1, c0, c1);
}

/* Close a sink: its branch count, capped at the buffer (overflow flagged). */
template <typename Sink>
__device__ int sink_count(Sink &sink, int32_t *status)
{
    __syncwarp();
    if (sink.out > sink.cap) {
        if (lane_id() == 0) atomicOr(status, QW_ST_WARP_OVERFLOW);
        return sink.cap;
    }
    return sink.out;
}


/* The zero-type Hadamard group of H P H, after T~^dag's rotation has negated
 * every other branch and set the group aside (PairListSink with REFL): in a
 * row with jc = b1 = 0, the group (kc = k_high = b2 = 0) maps a_u ->
 * (2/s) sum_v a_v - a_u for all s values of u (H P H = 2|+><+| - 1 there).
 * Appends the s pairs (u: the reflected b2 = 0 value, and the set-aside
 * negated b2 = 1 partner) to the np entries of the pair list; elems receives
 * the number of branches appended.  The sum is taken by u in a fixed order
 * (FP64 for complex128, a float pair for complex64); with readout,
 * (1/sqrt s) sum_v a_v -- the flag-0 amplitude of T~^dag's output -- goes into
 * the QLS accumulator. */
template <typename AmpT, typename KeyT>
__device__ int reflect_zero_list(const QwSimDev &d, const Row &r, KeyT *kd, AmpT *a0d, AmpT *a1d, int np, int cap,
                                 int32_t *status, const QwStepArgs &a, const AmpT *zbuf, const AmpT *z1buf,
                                 const int16_t *pbuf, int &elems)
{
    elems = 0;
    if (r.jc != 0) return np;
    const int lane = lane_id();
    const int s = d.s;
    typename Amp<AmpT>::Sum sum;
    for (int t = lane; t < s; t += 32) sum.add(zbuf[t]);
    sum.reduce(s);
    if (a.qls_readout && r.valid && lane == 0) {
        const double2 sv = sum.value();
        const double coef = a.qls_coefs[*a.qls_j];
        double2 acc = a.qls_y[r.j];
        acc.x += coef * (d.inv_sqrt_s * sv.x);
        acc.y += coef * (d.inv_sqrt_s * sv.y);
        a.qls_y[r.j] = acc;
    }
    sum.scale_pow2(d.two_over_s);
    int out = np;
    for (int ub = 0; ub < s; ub += 32) {
        const int u = ub + lane;
        const bool vu = u < s;
        AmpT o0 = Amp<AmpT>::zero();
        bool c1 = false;
        if (vu) {
            o0 = sum.minus(zbuf[u]);
            c1 = pbuf[u] > 0;
        }
        const bool c0 = vu && Amp<AmpT>::keep(d, o0);
        const bool any = c0 || c1;
        const unsigned m = __ballot_sync(FULL, any);
        elems += __popc(__ballot_sync(FULL, c0)) + __popc(__ballot_sync(FULL, c1));
        if (any) {
            const int pos = out + __popc(m & ((1u << lane) - 1u));
            if (pos < cap) {
                kd[pos] = (KeyT)u << 1;
                a0d[pos] = c0 ? o0 : Amp<AmpT>::zero();
                a1d[pos] = c1 ? z1buf[u] : Amp<AmpT>::zero();
            }
        }
        out += __popc(m);
    }
    __syncwarp();
    if (out > cap) {
        if (lane == 0) atomicOr(status, QW_ST_WARP_OVERFLOW);
        out = cap;
    }
    return out;
}

/* Register maps of T~^dag before R^dag.  T~^dag applies O_s'^dag, O_A', O_s',
 * R^dag, O_s'^dag, O_A': O_s' R^dag O_s'^dag is R^dag in the coordinates
 * (l, z) = O_s'^dag(k, kc), controlled by A and by the input column k, and the
 * second O_A' undoes the first.  So each branch moves to (l, z) and carries
 * A = [jc = 0, z = 0] a_{j,l} and sigma(j, k) for the rotation; after R^dag the
 * controls are dropped (A = 0).  Input A is 0 (T~ and T~^dag return it to 0
 * at the end of every step; the loader checks it). */
template <typename KeyT>
__device__ __forceinline__ KeyT map_tdag(const QwSimDev &d, const Row &r, KeyT key, uint32_t &slot, uint32_t &A,
                                         bool &sneg)
{
    const uint32_t m = (1u << d.nb) - 1u;
    const uint32_t k = (uint32_t)(key >> 1) & m, kc = (uint32_t)(key >> (1 + d.nb)) & m;
    const uint32_t l = kc ^ qbs(d, r, k);
    const uint32_t w = qword(d, r, l);
    const uint32_t z = k ^ (w >> 16);
    A = (r.jc == 0 && z == 0) ? (w & 0xffffu) : 0u;
    slot = r.valid ? l : 0xffffffffu;
    sneg = r.j > k;
    return (key & (KeyT)1) | ((KeyT)l << 1) | ((KeyT)z << (1 + d.nb));
}

/* Register maps of T~ after H: O_A', O_s', R, O_s'^dag, O_A', O_s'.  From
 * (l, z): A = [jc = 0, z = 0] a_{j,l}, then O_s' gives (k, kc) =
 * (z ^ K(j,l), l ^ I(j, k)); R is controlled by A and sigma(j, k); the last
 * three maps only return A to 0. */
template <typename KeyT>
__device__ __forceinline__ KeyT map_t(const QwSimDev &d, const Row &r, KeyT key, uint32_t &slot, uint32_t &A,
                                      bool &sneg)
{
    const uint32_t m = (1u << d.nb) - 1u;
    const uint32_t l = (uint32_t)(key >> 1) & m, z = (uint32_t)(key >> (1 + d.nb)) & m;
    const uint32_t w = qword(d, r, l);
    slot = r.valid ? l : 0xffffffffu;
    A = (r.jc == 0 && z == 0) ? (w & 0xffffu) : 0u;
    const uint32_t k = z ^ (w >> 16);
    /* z = 0 and l a slot of a row j < N: k is the column of slot l, whose
       in-row index in the unique sorted list is l itself, so kc = l ^ l = 0
       without the search */
    const uint32_t kc = (z == 0 && l < (uint32_t)d.s && r.valid) ? 0u : l ^ qbs(d, r, k);
    sneg = r.j > k;
    return (key & (KeyT)1) | ((KeyT)k << 1) | ((KeyT)kc << (1 + d.nb));
}

/* S, and the append of every branch to the bucket of its new row. */
template <typename AmpT, typename KeyT>
__device__ void emit_pairs(const QwSimDev &d, const Row &r, const KeyT *ks, const AmpT *as, int n,
                           const QwBufDev &out, int32_t *status, typename Amp<AmpT>::Norm &nrm)
{
    const uint32_t m = (1u << d.nb) - 1u;
    const int64_t blo = d.ninst == 1 ? 0 : d.inst_bkt[r.inst];
    const int64_t bhi = d.ninst == 1 ? d.dense_buckets : d.inst_bkt[r.inst + 1];
    Regs y;
    y.kc = r.jc;
    y.k = r.j;
    y.b2 = 0;
    y.A = 0;
    const uint64_t local0 = encode_r(y, d.nb);
    /* destination bucket of branch i (-1: dropped with a status bit, or sent
       to the partition owning its new row) */
    auto dest = [&](int i) -> int64_t {
        const KeyT key = ks[i];
        const uint32_t b2 = (uint32_t)(key & (KeyT)1), k = (uint32_t)(key >> 1) & m;
        const uint32_t kc = (uint32_t)(key >> (1 + d.nb)) & m;
        if (d.nparts > 1) {
            const int own = qw_part_owner_of(d, kc, k);
            if (own != d.part) {
                part_send(d, own, qw_rowkey(r.inst, kc, k, b2),
                          local0 | (uint64_t)((key >> KeyB1<KeyT>::bit) & (KeyT)1), Amp<AmpT>::to_d(as[i]), status);
                nrm.add(as[i]);
                return -1;
            }
        }
        if (kc == 0) {
            const int64_t b = blo + (((int64_t)k << 1) | (int64_t)b2);
            if (b < bhi) return b;
            atomicOr(status, QW_ST_SPILL_FULL);
            return -1;
        }
        return bucket_of(d, out, r.inst, kc, k, b2, status);
    };
    auto put = [&](int i, int64_t b, int pos) {
        if (pos >= d.cap_row) {
            atomicOr(status, QW_ST_ROW_OVERFLOW);
            return;
        }
        const int64_t slot = b * (int64_t)d.cap_row + pos;
        out.key[slot] = local0 | (uint64_t)((ks[i] >> KeyB1<KeyT>::bit) & (KeyT)1); /* new b2 = old b1 */
        static_cast<AmpT *>(out.amp)[slot] = as[i];
        nrm.add(as[i]);
    };
    /* two branches per lane per pass: both slot claims are in flight before
       either store waits on its claim */
    for (int i0 = lane_id(); i0 < n; i0 += 64) {
        const int i1 = i0 + 32;
        const int64_t b0 = dest(i0);
        const int64_t b1 = i1 < n ? dest(i1) : -1;
        const int p0 = b0 >= 0 ? atomicAdd(out.count + b0, 1) : 0;
        const int p1 = b1 >= 0 ? atomicAdd(out.count + b1, 1) : 0;
        if (b0 >= 0) put(i0, b0, p0);
        if (b1 >= 0) put(i1, b1, p1);
    }
}

/* Per-warp shared buffers of the row pipeline (offsets from walk_layout). */
template <typename AmpT, typename KeyT> struct WalkBufs {
    KeyT *kP, *kQ;
    AmpT *aP, *aQ, *aX, *zbuf, *z1buf;
    uint32_t *simg;
    int16_t *pbuf, *hidx;
    typename Amp<AmpT>::RotVal *sfg;
    __device__ WalkBufs(unsigned char *b, const WalkLayout &lay)
        : kP(reinterpret_cast<KeyT *>(b + lay.kP)), kQ(reinterpret_cast<KeyT *>(b + lay.kQ)),
          aP(reinterpret_cast<AmpT *>(b + lay.aP)), aQ(reinterpret_cast<AmpT *>(b + lay.aQ)),
          aX(reinterpret_cast<AmpT *>(b + lay.aX)), zbuf(reinterpret_cast<AmpT *>(b + lay.zbuf)),
          z1buf(reinterpret_cast<AmpT *>(b + lay.z1buf)), simg(reinterpret_cast<uint32_t *>(b + lay.simg)),
          pbuf(reinterpret_cast<int16_t *>(b + lay.pbuf)), hidx(reinterpret_cast<int16_t *>(b + lay.hidx)),
          sfg(reinterpret_cast<typename Amp<AmpT>::RotVal *>(b + lay.sfg))
    {
    }
};

/* What one pass of the row pipeline runs: one row (bucket bA, n0 branches,
 * b1 tag tagA) or the two rows of a j as one segment (buckets bA, bB). */
template <typename KeyT> struct WalkItem {
    int64_t bA, bB;
    int n0, n1;
    KeyT tagA;
    bool valid;
};

/* Branch counters of one warp (QW_STAT_*), added to the step's at its end
 * (32 bits per warp: a warp sees far fewer than 2^32 branches in a step). */
struct WalkStats {
    unsigned int rows = 0, in = 0, rdag = 0, hph = 0, out = 0;
    __device__ void flush(const QwStepArgs &a) const
    {
        if (a.stats && lane_id() == 0 && rows) {
            atomicAdd(a.stats + QW_STAT_ROWS, (unsigned long long)rows);
            atomicAdd(a.stats + QW_STAT_IN, (unsigned long long)in);
            atomicAdd(a.stats + QW_STAT_RDAG, (unsigned long long)rdag);
            atomicAdd(a.stats + QW_STAT_HPH, (unsigned long long)hph);
            atomicAdd(a.stats + QW_STAT_OUT, (unsigned long long)out);
        }
    }
};

/* One item through T~^dag, H P H, T~ and S (the row pipeline).  (have, hk,
 * ha): the item's first 32 stored branches, loaded ahead by a pipelined
 * caller; prefetch() runs once the item's input has been read (a pipelined
 * caller loads the next item's first branches there).  staged: (inst, j) of
 * the QRAM row held in B.simg. */
template <typename AmpT, typename KeyT, typename Prefetch>
__device__ __forceinline__ void walk_item(const QwSimDev &d, const QwBufDev &in, const QwBufDev &out,
                                          const QwStepArgs &a, const WalkItem<KeyT> &it, bool have_cur, uint64_t hk,
                                          AmpT ha, bool rescale, const typename Amp<AmpT>::Scale &scale,
                                          const WalkBufs<AmpT, KeyT> &B, int64_t &staged,
                                          typename Amp<AmpT>::Norm &nrm, WalkStats &st, Prefetch &&prefetch)
{
    typedef typename Amp<AmpT>::RotVal RotVal;
    constexpr int B1 = KeyB1<KeyT>::bit;
    const int lane = lane_id();
    const int C = d.warp_cap;
    int n = it.n0 + it.n1;
    if (n <= 0) return;
    Row r;
    if (!row_of(d, in, it.bA, r)) return;
    if (n > C) {
        if (lane == 0) atomicOr(a.status, QW_ST_WARP_OVERFLOW);
        return;
    }
    r.simg = B.simg;
    r.sfg = B.sfg;
    const int64_t want = ((int64_t)r.inst << 32) | (int64_t)r.j;
    if (r.valid && want != staged) {
        const int64_t w0 = r.img_base + (int64_t)r.j * d.s;
        for (int t = lane; t < d.s; t += 32) {
            B.simg[t] = __ldg(d.img + w0 + t);
            B.sfg[t] = __ldg(static_cast<const RotVal *>(d.slot_rot) + w0 + t);
        }
        staged = want;
    }
    st.rows++;
    st.in += n;
    if (r.jc == 0) { /* the zero-type group's slots, filled by T~^dag */
        for (int t = lane; t < d.s; t += 32) {
            B.zbuf[t] = Amp<AmpT>::zero();
            B.pbuf[t] = -1;
        }
        __syncwarp();
    }
    PairListSink<AmpT, KeyT, true> s0(d, r, B.kQ, B.aQ, B.aX, C, B.zbuf, B.z1buf, B.pbuf);
    if (!Amp<AmpT>::kHeadLanes && it.n0 <= 32 && it.n1 <= 32) {
        /* rows of <= 32: T~^dag straight from the loaded registers, the
           pairs found by one warp match per chunk of <= 32 */
        const int ash = 1 + 2 * d.nb;
        const KeyT tagB = (KeyT)1 << B1;
        uint64_t anc = 0;
        const AmpT *amp = static_cast<const AmpT *>(in.amp);
        auto get = [&](int64_t slot, bool pre, uint64_t praw, AmpT pamp, KeyT tag, KeyT &k, AmpT &v) {
            k = in_key<KeyT>(pre ? praw : in.key[slot], ash, tag, anc);
            v = pre ? pamp : amp[slot];
            if (rescale) v = scale.apply(v);
        };
        if (n <= 32) {
            KeyT k = 0;
            AmpT v = Amp<AmpT>::zero();
            if (lane < it.n0) get(it.bA * (int64_t)d.cap_row + lane, have_cur, hk, ha, it.tagA, k, v);
            else if (lane < n) get(it.bB * (int64_t)d.cap_row + (lane - it.n0), have_cur, hk, ha, tagB, k, v);
            rot0_chunk<AmpT, KeyT>(d, r, k, v, lane < n, s0);
        } else {
            KeyT k = 0;
            AmpT v = Amp<AmpT>::zero();
            if (lane < it.n0) get(it.bA * (int64_t)d.cap_row + lane, have_cur, hk, ha, it.tagA, k, v);
            rot0_chunk<AmpT, KeyT>(d, r, k, v, lane < it.n0, s0);
            /* row B: its first 32 - n0 branches were loaded ahead into lanes n0.. */
            const int src = (it.n0 + lane) & 31;
            const uint64_t bh = __shfl_sync(FULL, hk, src);
            AmpT ba;
            ba.x = __shfl_sync(FULL, ha.x, src);
            ba.y = __shfl_sync(FULL, ha.y, src);
            KeyT kB = 0;
            AmpT vB = Amp<AmpT>::zero();
            if (lane < it.n1)
                get(it.bB * (int64_t)d.cap_row + lane, have_cur && it.n0 + lane < 32, bh, ba, tagB, kB, vB);
            rot0_chunk<AmpT, KeyT>(d, r, kB, vB, lane < it.n1, s0);
        }
        if (__any_sync(FULL, anc != 0) && lane == 0) atomicOr(a.status, QW_ST_ANCILLA);
    } else {
        load_seg<AmpT, KeyT>(d, in, it.bA, it.n0, it.tagA, it.bB, it.n1, rescale, scale, B.kP, B.aP, B.kQ, B.aQ, C,
                             have_cur, hk, ha, a.status);
        map_rot_pairs<0, AmpT, KeyT>(d, r, B.kP, B.aP, n, s0, B.hidx);
    }
    prefetch();
    int np = sink_count(s0, a.status); /* T~^dag, H P H signs */
    st.rdag += s0.elems + s0.div;
    int ez = 0;
    np = reflect_zero_list<AmpT, KeyT>(d, r, B.kQ, B.aQ, B.aX, np, C, a.status, a, B.zbuf, B.z1buf, B.pbuf,
                                       ez); /* H P H */
    st.hph += s0.elems + ez;
    PairSink<AmpT, KeyT, false> s1(d, r, B.kP, B.aP, C, nullptr, nullptr, nullptr);
    map_rot_list<1, AmpT, KeyT>(d, r, B.kQ, B.aQ, B.aX, np, s1);
    n = sink_count(s1, a.status); /* T~ */
    st.out += n;
    emit_pairs<AmpT, KeyT>(d, r, B.kP, B.aP, n, out, a.status, nrm); /* S */
    __syncwarp();
}

/* The row pipeline for one item, out of line: the slot kernel's path for
 * what its lanes do not cover (so the fast path keeps its registers and its
 * accumulators stay out of memory).  Returns the item's norm share and adds
 * its counters to *st. */
template <typename AmpT, typename KeyT>
__device__ __noinline__ double walk_item_ool(const QwSimDev &d, const QwBufDev &in, const QwBufDev &out,
                                             const QwStepArgs &a, WalkItem<KeyT> it, bool rescale, double scale_v,
                                             unsigned char *base, WalkLayout lay, WalkStats *st)
{
    const WalkBufs<AmpT, KeyT> B(base, lay);
    const typename Amp<AmpT>::Scale scale(scale_v);
    int64_t staged = -1;
    typename Amp<AmpT>::Norm nrm;
    WalkStats sti;
    walk_item<AmpT, KeyT>(d, in, out, a, it, false, 0ull, Amp<AmpT>::zero(), rescale, scale, B, staged, nrm, sti,
                          [] {});
    st->rows += sti.rows;
    st->in += sti.in;
    st->rdag += sti.rdag;
    st->hph += sti.hph;
    st->out += sti.out;
    return nrm.get();
}

/* Start of a step: a step issued after a failed one does nothing, so the
 * state of the last clean step (its input buffer, never written) survives for
 * the host; otherwise clear X_{t+2} for the step after this one. */
__device__ __forceinline__ bool step_begin(const QwSimDev &d, const QwBufDev &clr, const QwStepArgs &a)
{
    const bool skip = *(volatile int32_t *)a.status != 0;
    if (!skip) {
        const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
        for (int64_t b = tid; b < d.total_buckets; b += nthr) clr.count[b] = 0;
        for (int64_t t = tid; t < d.spill_slots; t += nthr) clr.spill[t] = QW_SPILL_EMPTY;
    }
    return skip;
}

/* One walk step.  SEG = false: the two rows (jc = 0, j, b1 = 0 / 1) of a j
 * are processed one after the other by the same warp; SEG = true: together,
 * as one segment.  PF = false: 4 blocks per SM, each item loaded when its
 * turn comes; PF = true: 3 blocks per SM (more registers), the item loop
 * software-pipelined -- the next item's counts read at the start of the
 * current one, its first 32 branches loaded while the current one runs. */
template <typename AmpT, bool PF, bool SEG, typename KeyT>
__global__ void __launch_bounds__(WARPS * 32, PF ? 3 : 4) k_walk(QwSimDev d, QwBufDev in, QwBufDev out,
                                                                 QwBufDev clr, QwStepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double block_part[WARPS];
    __shared__ int is_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const WalkLayout lay = walk_layout<AmpT, KeyT>(d);
    const WalkBufs<AmpT, KeyT> B(smem + lay.per_warp * warp, lay);

    const bool skip = step_begin(d, clr, a);
    const bool rescale = a.scale_in != nullptr;
    const typename Amp<AmpT>::Scale scale(rescale ? *a.scale_in : 1.0);
    typename Amp<AmpT>::Norm nrm;
    WalkStats st;

    /* Units: a dense unit u holds the rows (jc = 0, j) with b1 = 0 and 1
       (buckets 2u and 2u + 1); a garbage-row bucket (jc != 0) is a unit of
       its own.  Warps stride over units (a b1 = 0 row is about twice a b1 = 1
       row, so keeping both rows of a j on one warp balances the warps).  An
       item is what one pass of the row pipeline runs: a whole dense unit
       (SEG) or one of its rows. */
    const int64_t nwarps = (int64_t)gridDim.x * WARPS;
    const int64_t d2 = d.dense_buckets >> 1;
    const int64_t units = skip ? 0 : d2 + d.spill_slots;
    constexpr int B1 = KeyB1<KeyT>::bit;
    auto item_of = [&](int64_t uu, int part, WalkItem<KeyT> &it) {
        it.valid = uu < units;
        it.n0 = it.n1 = 0;
        it.tagA = 0;
        it.bB = -1;
        if (!it.valid) return;
        if (uu < d2) {
            if (SEG) {
                it.bA = 2 * uu;
                it.bB = it.bA + 1;
                it.n1 = min(in.count[it.bB], d.cap_row);
            } else {
                it.bA = 2 * uu + part;
                it.tagA = (KeyT)part << B1;
            }
            it.n0 = min(in.count[it.bA], d.cap_row);
        } else {
            it.bA = d.dense_buckets + (uu - d2);
            it.n0 = min(in.count[it.bA], d.cap_row);
            if (it.n0 > 0) it.tagA = (KeyT)(in.spill[uu - d2] & 1ull) << B1;
        }
    };
    auto advance = [&](int64_t &uu, int &part) {
        if (!SEG && uu < d2 && part == 0) {
            part = 1;
        } else {
            part = 0;
            uu += nwarps;
        }
    };
    int64_t u = (int64_t)blockIdx.x * WARPS + warp;
    int part = 0;
    WalkItem<KeyT> cur, nxt;
    item_of(u, part, cur);
    bool have = false;
    uint64_t pk = 0;
    AmpT pa = Amp<AmpT>::zero();
    int64_t staged = -1; /* (inst, j) of the QRAM row held in simg */
    while (cur.valid) {
        int64_t un = u;
        int pn = part;
        advance(un, pn);
        const bool have_cur = have;
        const uint64_t hk = pk;
        const AmpT ha = pa;
        have = false;
        if (PF) item_of(un, pn, nxt);
        const WalkItem<KeyT> it = cur;
        u = un;
        part = pn;
        if (!PF) item_of(u, part, cur);
        else cur = nxt;
        walk_item<AmpT, KeyT>(d, in, out, a, it, have_cur, hk, ha, rescale, scale, B, staged, nrm, st, [&] {
            if (PF && cur.valid) { /* the next item's first 32 branches (row A, then row B) */
                const int nn = cur.n0 + cur.n1;
                have = nn > 0;
                if (lane < nn) {
                    const int64_t slot = lane < cur.n0 ? cur.bA * (int64_t)d.cap_row + lane
                                                       : cur.bB * (int64_t)d.cap_row + (lane - cur.n0);
                    pk = in.key[slot];
                    pa = static_cast<const AmpT *>(in.amp)[slot];
                }
            }
        });
    }
    st.flush(a);
    finish_step(a, nrm.get(), block_part, &is_last, true);
}

/* ==== slot kernel: one lane per QRAM slot ==================================== */
/*
 * A branch (kc, k, b2) of a row (jc = 0, j < N, b1) whose T~^dag coordinates
 * (l, z) = O_s'^dag(k, kc) = (kc ^ I(j, k), k ^ K(j, l)) have z = 0 sits on
 * slot l < s of the row, and its b2 partner on the same slot.  In the states
 * the walk reaches from T~|b~> every branch of a b1 = 0 row is of that kind
 * and so are most of a b1 = 1 row (the others come from rows whose padding
 * names j without j's row naming them).  The kernel takes RPP = 32 / s
 * consecutive j (a group) per warp pass, lane t = u s + l on slot l of the
 * group's u-th j:
 *   - load: every branch of the group's 2 RPP buckets is read once, mapped by
 *     T~^dag's first O_s'^dag (one QBS and one QRAM word on the staged rows)
 *     and scattered into the slot table of its row, where its partner lands
 *     beside it: no matching and no sort; the rest ("extras") are listed;
 *   - pass A, the b1 = 0 rows: R^dag on each slot's pair; the zero-type group
 *     of H P H (kc = z = 0, l < s, b2 = 0, jc = b1 = 0) is exactly the row's s
 *     slots, summed over the unit's s lanes; the reflected pair goes through
 *     T~ (O_A' reads slot l, O_s' maps (l, 0) to (K(j, l), 0) with no search)
 *     and R, then S;
 *   - pass B, the b1 = 1 rows' slots and the extras, one lane per pair:
 *     R^dag, the sign of H P H (-1 outside the zero-type groups), the maps and
 *     R of T~, S.
 * The operations, their order, the pruning points and the counters are those
 * of k_walk, and so are the results (bit for bit up to the norm's summation
 * order).  Groups holding anything the lanes do not cover (a row j >= N with
 * branches, more extras than the list holds) and the garbage rows (jc != 0)
 * go through the row pipeline. */
constexpr int kSlotExtras = 32; /* extras list of a group */
constexpr int kSlotItems = 64;  /* pass B items: 32 slots + 32 extra pairs */
constexpr int kSlotStage = 128; /* a group's first branches, copied to shared memory ahead */

/* Asynchronous copies global -> shared (cp.async, sm_80 and later): the
 * branch loads of a group are all in flight together, and land without
 * passing through registers. */
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
template <typename AmpT> __device__ __forceinline__ void cp_async_amp(AmpT *dst, const AmpT *src);
template <> __device__ __forceinline__ void cp_async_amp<float2>(float2 *dst, const float2 *src) { cp_async8(dst, src); }
template <> __device__ __forceinline__ void cp_async_amp<double2>(double2 *dst, const double2 *src)
{
    cp_async16(dst, src);
}

struct SlotUnit {
    uint32_t j, inst, n;
    int32_t valid;
    int64_t img, blo, bhi; /* image offset of the instance, its dense bucket range */
};

struct SlotLayout {
    size_t ws, rot, ta, tb, ek, ea, im, ia, unit, sk, sa, per_warp;
};

template <typename AmpT>
__host__ __device__ inline SlotLayout slot_layout()
{
    SlotLayout o;
    size_t p = 0;
#define QW_TAKE(field, bytes)                                                                      \
    o.field = p;                                                                                   \
    p = (p + (bytes) + 15) & ~(size_t)15
    QW_TAKE(ws, 32 * sizeof(uint32_t));
    QW_TAKE(rot, 32 * 16);
    QW_TAKE(ta, 64 * sizeof(AmpT));
    QW_TAKE(tb, 64 * sizeof(AmpT));
    QW_TAKE(ek, kSlotExtras * sizeof(uint64_t));
    QW_TAKE(ea, kSlotExtras * sizeof(AmpT));
    QW_TAKE(im, kSlotItems * sizeof(uint16_t));
    QW_TAKE(ia, 2 * kSlotItems * sizeof(AmpT));
    QW_TAKE(unit, 8 * sizeof(SlotUnit));
    QW_TAKE(sk, kSlotStage * sizeof(uint64_t));
    QW_TAKE(sa, kSlotStage * sizeof(AmpT));
#undef QW_TAKE
    o.per_warp = p;
    return o;
}

template <typename AmpT, typename KeyT>
__host__ __device__ inline size_t slot_per_warp(const QwSimDev &d)
{
    const size_t a = walk_layout<AmpT, KeyT>(d).per_warp, b = slot_layout<AmpT>().per_warp;
    return a > b ? a : b;
}

/* Def. 1 on a staged row of S sorted distinct columns (the branch-free lower
 * bound of qbs() with S known at compile time). */
template <int S>
__device__ __forceinline__ uint32_t qbs_row(const uint32_t *row, uint32_t target)
{
    uint32_t i = 0, ci = row[0] >> 16;
#pragma unroll
    for (int step = S >> 1; step > 0; step >>= 1) {
        const uint32_t c = row[i + step] >> 16;
        const bool up = c <= target;
        i = up ? i + (uint32_t)step : i;
        ci = up ? c : ci;
    }
    return ci == target ? i : 0u;
}

__device__ __forceinline__ Row slot_row(const SlotUnit &U, const uint32_t *ws, const void *rot)
{
    Row r;
    r.inst = U.inst;
    r.jc = 0;
    r.j = U.j;
    r.b1 = 0;
    r.n_inst = U.n;
    r.img_base = U.img;
    r.valid = U.valid != 0;
    r.simg = ws;
    r.sfg = rot;
    return r;
}

template <typename AmpT>
__device__ __forceinline__ bool amp_nonzero(AmpT a)
{
    return a.x != 0 || a.y != 0;
}

/* S for up to two kept outputs of a lane, in two halves so that a caller
 * can have the slot claims of several lanes' outputs in flight together:
 * slot_route finds the buckets of (kc_out, k_out, b2 = 0 / 1), the new rows
 * of row (jc = 0, j, b1)'s outputs (-1: nothing to store here; a branch whose
 * new row another partition owns is sent to it), slot_put stores a branch
 * with local registers (kc, k, b2) = (0, j, b1) at the claimed position. */
template <typename AmpT>
__device__ __forceinline__ void slot_route(const QwSimDev &d, const QwBufDev &out, const SlotUnit &U, uint32_t k_out,
                                           uint32_t kc_out, uint32_t b1, AmpT r0, AmpT r1, bool e0, bool e1,
                                           int32_t *status, typename Amp<AmpT>::Norm &nrm, int64_t &b0, int64_t &bb1)
{
    b0 = -1;
    bb1 = -1;
    if (!e0 && !e1) return;
    if (d.nparts > 1) { /* the new row (kc_out, k_out) is another partition's */
        const int own = qw_part_owner_of(d, kc_out, k_out);
        if (own != d.part) {
            const uint64_t local = (uint64_t)b1 | ((uint64_t)U.j << 1);
            if (e0) {
                part_send(d, own, qw_rowkey(U.inst, kc_out, k_out, 0), local, Amp<AmpT>::to_d(r0), status);
                nrm.add(r0);
            }
            if (e1) {
                part_send(d, own, qw_rowkey(U.inst, kc_out, k_out, 1), local, Amp<AmpT>::to_d(r1), status);
                nrm.add(r1);
            }
            return;
        }
    }
    if (kc_out == 0) {
        const int64_t b = U.blo + ((int64_t)k_out << 1);
        if (e0) {
            if (b < U.bhi) b0 = b;
            else atomicOr(status, QW_ST_SPILL_FULL);
        }
        if (e1) {
            if (b + 1 < U.bhi) bb1 = b + 1;
            else atomicOr(status, QW_ST_SPILL_FULL);
        }
    } else {
        if (e0) b0 = bucket_of(d, out, U.inst, kc_out, k_out, 0, status);
        if (e1) bb1 = bucket_of(d, out, U.inst, kc_out, k_out, 1, status);
    }
}

template <typename AmpT>
__device__ __forceinline__ void slot_put(const QwSimDev &d, const QwBufDev &out, int64_t b, int p, uint64_t local,
                                         AmpT r, int32_t *status, typename Amp<AmpT>::Norm &nrm)
{
    if (b < 0) return;
    if (p < d.cap_row) {
        const int64_t sl = b * (int64_t)d.cap_row + p;
        out.key[sl] = local;
        static_cast<AmpT *>(out.amp)[sl] = r;
        nrm.add(r);
    } else {
        atomicOr(status, QW_ST_ROW_OVERFLOW);
    }
}

/* One lane's kept outputs waiting for S: the buckets of their new rows, the
 * local key and the amplitudes. */
template <typename AmpT> struct SlotOut {
    int64_t b0, b1;
    uint64_t local;
    AmpT r0, r1;
};

template <typename AmpT>
__device__ __forceinline__ void slot_out(const QwSimDev &d, const QwBufDev &out, const SlotUnit &U, uint32_t k_out,
                                         uint32_t kc_out, uint32_t b1, AmpT r0, AmpT r1, bool e0, bool e1,
                                         int32_t *status, typename Amp<AmpT>::Norm &nrm, SlotOut<AmpT> &o)
{
    slot_route<AmpT>(d, out, U, k_out, kc_out, b1, r0, r1, e0, e1, status, nrm, o.b0, o.b1);
    o.local = (uint64_t)b1 | ((uint64_t)U.j << 1);
    o.r0 = r0;
    o.r1 = r1;
}

/* claims of two lanes' worth of outputs in flight together, then the stores */
template <typename AmpT>
__device__ __forceinline__ void slot_store2(const QwSimDev &d, const QwBufDev &out, const SlotOut<AmpT> &x,
                                            const SlotOut<AmpT> &y, int32_t *status, typename Amp<AmpT>::Norm &nrm)
{
    const int px0 = x.b0 >= 0 ? atomicAdd(out.count + x.b0, 1) : 0;
    const int px1 = x.b1 >= 0 ? atomicAdd(out.count + x.b1, 1) : 0;
    const int py0 = y.b0 >= 0 ? atomicAdd(out.count + y.b0, 1) : 0;
    const int py1 = y.b1 >= 0 ? atomicAdd(out.count + y.b1, 1) : 0;
    slot_put<AmpT>(d, out, x.b0, px0, x.local, x.r0, status, nrm);
    slot_put<AmpT>(d, out, x.b1, px1, x.local, x.r1, status, nrm);
    slot_put<AmpT>(d, out, y.b0, py0, y.local, y.r0, status, nrm);
    slot_put<AmpT>(d, out, y.b1, py1, y.local, y.r1, status, nrm);
}

template <typename AmpT, int S, typename KeyT>
__global__ void __launch_bounds__(WARPS * 32, 4) k_walk_slot(QwSimDev d, QwBufDev in, QwBufDev out, QwBufDev clr,
                                                             QwStepArgs a)
{
    typedef typename Amp<AmpT>::RotVal RotVal;
    constexpr int RPP = 32 / S, NBK = 2 * RPP;
    constexpr int B1 = KeyB1<KeyT>::bit;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double block_part[WARPS];
    __shared__ int is_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const WalkLayout lay = walk_layout<AmpT, KeyT>(d);
    const SlotLayout sl = slot_layout<AmpT>();
    unsigned char *base = smem + slot_per_warp<AmpT, KeyT>(d) * warp;
    uint32_t *ws = reinterpret_cast<uint32_t *>(base + sl.ws);
    RotVal *rotv = reinterpret_cast<RotVal *>(base + sl.rot);
    AmpT *ta = reinterpret_cast<AmpT *>(base + sl.ta);
    AmpT *tb = reinterpret_cast<AmpT *>(base + sl.tb);
    uint64_t *ek = reinterpret_cast<uint64_t *>(base + sl.ek);
    AmpT *ea = reinterpret_cast<AmpT *>(base + sl.ea);
    uint16_t *im = reinterpret_cast<uint16_t *>(base + sl.im);
    AmpT *ia = reinterpret_cast<AmpT *>(base + sl.ia);
    SlotUnit *units = reinterpret_cast<SlotUnit *>(base + sl.unit);
    uint64_t *sk = reinterpret_cast<uint64_t *>(base + sl.sk);
    AmpT *sa = reinterpret_cast<AmpT *>(base + sl.sa);

    const bool skip = step_begin(d, clr, a);
    const bool rescale = a.scale_in != nullptr;
    const double scale_v = rescale ? *a.scale_in : 1.0;
    const typename Amp<AmpT>::Scale scale(scale_v);
    typename Amp<AmpT>::Norm nrm;
    WalkStats st;
    const AmpT zero = Amp<AmpT>::zero();
    const AmpT *amp_in = static_cast<const AmpT *>(in.amp);
    const uint32_t msk = (1u << d.nb) - 1u;
    const int ash = 1 + 2 * d.nb;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t d2 = d.dense_buckets >> 1;
    const int64_t ngroups = skip ? 0 : (d2 + RPP - 1) / RPP;
    const int64_t nwarps = (int64_t)gridDim.x * WARPS;
    const int64_t gw = (int64_t)blockIdx.x * WARPS + warp;

    /* units the lanes do not cover go to the row pipeline, run by the last
       block once every other block is done (the hot loop holds no call) */
    auto defer = [&](int32_t entry) {
        if (lane == 0) {
            a.deferred[atomicAdd(a.deferred_ctr, 1u)] = entry;
            __threadfence(); /* visible before this block counts itself done */
        }
    };

    /* groups: each warp's first is its own index.  One instance: then every
       nwarps-th group (the groups are alike), the next group's counts read
       one group ahead.  Several instances (groups of very different sizes,
       empty ones past each N): the rest are claimed from a counter, the claim
       issued a group ahead so that its latency hides behind the work */
    const bool dyn = d.ninst > 1;
    unsigned claim_raw = 0;
    auto claim = [&]() {
        if (dyn && lane == 0) claim_raw = atomicAdd(a.work_ctr, 1u);
    };
    auto group_counts = [&](int64_t gg) {
        const int64_t uu0 = gg * RPP;
        return (gg < ngroups && lane < NBK && uu0 + (lane >> 1) < d2) ? min(in.count[2 * uu0 + lane], d.cap_row) : 0;
    };
    int64_t g = gw;
    int cnt_next = group_counts(g);
    if (g < ngroups) claim();
    for (; g < ngroups; g = dyn ? nwarps + (int64_t)__shfl_sync(FULL, claim_raw, 0) : g + nwarps, claim()) {
        const int64_t u0 = g * RPP;
        /* counts of the group's buckets 2 u0 .. 2 u0 + NBK - 1 and their
           exclusive offsets in the group's branch order */
        const int cnt = dyn ? group_counts(g) : cnt_next;
        if (!dyn) cnt_next = group_counts(g + nwarps);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < NBK; o <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(FULL, incl, NBK - 1);
        if (total == 0) continue;
        const int excl = incl - cnt;
        if (lane < RPP) {
            SlotUnit U;
            const int64_t uu = u0 + lane;
            U.valid = 0;
            U.j = 0;
            U.inst = 0;
            U.n = 0;
            U.img = 0;
            U.blo = 0;
            U.bhi = d.dense_buckets;
            if (uu < d2) {
                if (d.ninst == 1) {
                    U.j = (uint32_t)uu;
                    U.n = (uint32_t)d.n_single;
                } else {
                    const int i = d.unit_inst[uu];
                    U.inst = (uint32_t)i;
                    U.blo = d.inst_bkt[i];
                    U.bhi = d.inst_bkt[i + 1];
                    U.j = (uint32_t)((2 * uu - U.blo) >> 1);
                    U.n = (uint32_t)d.inst_n[i];
                    U.img = d.inst_img[i];
                }
                U.valid = U.j < U.n;
            }
            units[lane] = U;
        }
        __syncwarp();
        /* a row j >= N holding branches: the row pipeline */
        const bool bad = lane < NBK && cnt > 0 && !units[lane >> 1].valid;
        if (__any_sync(FULL, bad)) {
            for (int q = 0; q < RPP; ++q) {
                const int c0 = __shfl_sync(FULL, cnt, 2 * q), c1 = __shfl_sync(FULL, cnt, 2 * q + 1);
                if (c0 + c1 > 0) defer((int32_t)(u0 + q));
            }
            continue;
        }
        int ex[NBK];
#pragma unroll
        for (int q = 0; q < NBK; ++q) ex[q] = __shfl_sync(FULL, excl, q);
        /* bucket of the group's t-th branch and its position there */
        auto locate = [&](int t, int &bi, int64_t &at) {
            int start = 0;
            bi = 0;
#pragma unroll
            for (int q = 1; q < NBK; ++q) {
                const bool ge = t >= ex[q];
                bi += ge ? 1 : 0;
                start = ge ? ex[q] : start;
            }
            at = (2 * u0 + bi) * (int64_t)d.cap_row + (t - start);
        };
        /* the group's first kSlotStage branches to shared memory, all in flight
           while the QRAM rows are staged */
        for (int t = lane; t < total && t < kSlotStage; t += 32) {
            int bi;
            int64_t at;
            locate(t, bi, at);
            cp_async8(sk + t, in.key + at);
            cp_async_amp<AmpT>(sa + t, amp_in + at);
        }
        cp_async_commit();
        /* stage the group's QRAM rows (contiguous in the image for one
           instance): lane t holds slot l = t % S of the row of unit t / S;
           a slot whose element is 0 rotates by R(0) */
        {
            const SlotUnit &U = units[lane / S];
            uint32_t w = 0;
            RotVal rv = Amp<AmpT>::rot_zero();
            if (U.valid) {
                const int64_t at = U.img + (int64_t)U.j * S + (lane % S);
                w = __ldg(d.img + at);
                if ((w & 0xffffu) != 0) rv = __ldg(static_cast<const RotVal *>(d.slot_rot) + at);
            }
            ws[lane] = w;
            rotv[lane] = rv;
            ta[lane] = zero;
            ta[lane + 32] = zero;
            tb[lane] = zero;
            tb[lane + 32] = zero;
        }
        cp_async_wait_all();
        __syncwarp();
        /* load: O_s'^dag of each branch, scattered to its slot or listed */
        uint64_t anc = 0;
        int ne = 0;
        for (int b0 = 0; b0 < total; b0 += 32) {
            const int t = b0 + lane;
            const bool act = t < total;
            int bi;
            int64_t at;
            locate(t, bi, at);
            const int ut = bi >> 1, b1 = bi & 1;
            uint64_t raw = 0;
            AmpT v = zero;
            if (act) {
                if (t < kSlotStage) {
                    raw = sk[t];
                    v = sa[t];
                } else {
                    raw = in.key[at];
                    v = amp_in[at];
                }
                if (rescale) v = scale.apply(v);
                anc |= raw >> ash;
            }
            const uint32_t b2 = (uint32_t)(raw & 1u), k = (uint32_t)(raw >> 1) & msk;
            const uint32_t kc = (uint32_t)(raw >> (1 + d.nb)) & msk;
            const uint32_t *row = ws + ut * S;
            const uint32_t l = kc ^ qbs_row<S>(row, k);
            bool isslot = false;
            if (act && l < (uint32_t)S) isslot = (k ^ (row[l] >> 16)) == 0;
            if (isslot) (b1 ? tb : ta)[(ut * S + (int)l) * 2 + (int)b2] = v;
            const bool isext = act && !isslot;
            const unsigned xm = __ballot_sync(FULL, isext);
            if (isext) {
                const int e = ne + __popc(xm & lt);
                if (e < kSlotExtras) {
                    ek[e] = (uint64_t)in_key<KeyT>(raw, ash, (KeyT)b1 << B1, anc) | ((uint64_t)ut << 56);
                    ea[e] = v;
                }
            }
            ne += __popc(xm);
        }
        if (__any_sync(FULL, anc != 0) && lane == 0) atomicOr(a.status, QW_ST_ANCILLA);
        if (ne > kSlotExtras) { /* more extras than the list holds: the row pipeline */
            for (int q = 0; q < RPP; ++q) {
                const int c0 = __shfl_sync(FULL, cnt, 2 * q), c1 = __shfl_sync(FULL, cnt, 2 * q + 1);
                if (c0 + c1 > 0) defer((int32_t)(u0 + q));
            }
            continue;
        }
        {
            unsigned int nu = 0;
#pragma unroll
            for (int q = 0; q < RPP; ++q) nu += (ex[2 * q] != (2 * q + 2 < NBK ? ex[2 * q + 2] : total)) ? 1u : 0u;
            st.rows += nu;
            st.in += (unsigned int)total;
        }
        __syncwarp();

        /* ---- pass A: the b1 = 0 rows, lane t on slot l = t % S of unit t / S ---- */
        {
            const SlotUnit &U = units[lane / S];
            const uint32_t w = ws[lane], col = w >> 16, val = w & 0xffffu;
            const RotVal rv = rotv[lane];
            const bool sneg = U.j > col;
            AmpT o0, o1;
            Amp<AmpT>::rot(rv, val, true, sneg, ta[2 * lane], ta[2 * lane + 1], o0, o1); /* R^dag */
            const bool c0 = Amp<AmpT>::keep(d, o0), c1 = Amp<AmpT>::keep(d, o1);
            st.rdag += __popc(__ballot_sync(FULL, c0)) + __popc(__ballot_sync(FULL, c1));
            /* H P H on the zero-type group: a_l -> (2/s) sum_v a_v - a_l; the
               b2 = 1 member, outside every zero-type group, is negated */
            const AmpT z0 = c0 ? o0 : zero;
            typename Amp<AmpT>::Sum sum;
            sum.set(z0);
            sum.reduce(S, S);
            if (a.qls_readout && U.valid && (lane % S) == 0) {
                const double2 sv = sum.value();
                const double coef = a.qls_coefs[*a.qls_j];
                double2 acc = a.qls_y[U.j];
                acc.x += coef * (d.inv_sqrt_s * sv.x);
                acc.y += coef * (d.inv_sqrt_s * sv.y);
                a.qls_y[U.j] = acc;
            }
            const AmpT h0 = sum.scaled_minus(d.two_over_s, z0);
            const bool d0 = Amp<AmpT>::keep(d, h0);
            st.hph += __popc(__ballot_sync(FULL, d0)) + __popc(__ballot_sync(FULL, c1));
            /* T~: O_A' reads slot l (A = a_{j,l}), O_s' takes (l, 0) to (K(j, l), 0);
               R; the rest of T~ returns A to 0 */
            AmpT r0, r1;
            Amp<AmpT>::rot(rv, val, false, sneg, d0 ? h0 : zero, c1 ? Amp<AmpT>::neg(o1) : zero, r0, r1);
            const bool e0 = Amp<AmpT>::keep(d, r0), e1 = Amp<AmpT>::keep(d, r1);
            st.out += __popc(__ballot_sync(FULL, e0)) + __popc(__ballot_sync(FULL, e1));
            SlotOut<AmpT> outA, none; /* S */
            slot_out<AmpT>(d, out, U, col, 0u, 0u, r0, r1, e0, e1, a.status, nrm, outA);
            none.b0 = none.b1 = -1;
            slot_store2<AmpT>(d, out, outA, none, a.status, nrm);
        }

        /* ---- pass B: list the b1 = 1 slots and the extras' pairs ---- */
        int ni;
        {
            const AmpT p0 = tb[2 * lane], p1 = tb[2 * lane + 1];
            const bool pres = amp_nonzero(p0) || amp_nonzero(p1);
            const unsigned pm = __ballot_sync(FULL, pres);
            if (pres) {
                const int q = __popc(pm & lt);
                im[q] = (uint16_t)lane;
                ia[2 * q] = p0;
                ia[2 * q + 1] = p1;
            }
            ni = __popc(pm);
            if (ne > 0) {
                /* pairs among the extras: keys equal but for b2, in one unit */
                const bool v = lane < ne;
                uint64_t kk = v ? ek[lane] : ~0ull - (uint64_t)(2 * lane);
                const AmpT va = v ? ea[lane] : zero;
                const unsigned mm = __match_any_sync(FULL, kk >> 1);
                const unsigned other = mm & ~(1u << lane);
                const bool one = (kk & 1ull) != 0;
                const bool head = v && (!one || other == 0);
                const int src = other ? (__ffs(other) - 1) : lane;
                AmpT pa;
                pa.x = __shfl_sync(FULL, va.x, src);
                pa.y = __shfl_sync(FULL, va.y, src);
                const unsigned hm = __ballot_sync(FULL, head);
                if (head) {
                    const int q = ni + __popc(hm & lt);
                    im[q] = (uint16_t)(0x8000u | (unsigned)lane);
                    ia[2 * q] = one ? zero : va;
                    ia[2 * q + 1] = one ? va : (other ? pa : zero);
                }
                ni += __popc(hm);
            }
        }
        __syncwarp();
        /* ---- pass B: one lane per pair ---- */
        for (int c = 0; c < ni; c += 32) {
            const int q = c + lane;
            const bool act = q < ni;
            const unsigned meta = act ? im[q] : 0u;
            const bool isext = (meta & 0x8000u) != 0;
            const AmpT a0 = act ? ia[2 * q] : zero, a1 = act ? ia[2 * q + 1] : zero;
            int ut;
            uint32_t b1, Adag, At, k_out = 0, kc_out = 0;
            bool sdag, st_neg;
            RotVal rdag, rt;
            KeyT key = 0;
            if (!isext) { /* slot t of a b1 = 1 row: (l, 0) both ways */
                const int t = (int)(meta & 63u);
                ut = t / S;
                b1 = 1;
                const uint32_t w = ws[t];
                k_out = w >> 16;
                Adag = At = w & 0xffffu;
                rdag = rt = rotv[t];
                sdag = st_neg = units[ut].j > k_out;
            } else { /* an extra: the general maps of rot_head */
                const uint64_t e = ek[meta & 0x7fffu];
                ut = (int)(e >> 56);
                key = (KeyT)(e & ~(0xffull << 56));
                b1 = (uint32_t)((key >> B1) & (KeyT)1);
                key &= ~(((KeyT)1) | ((KeyT)1 << B1));
                const Row r = slot_row(units[ut], ws + ut * S, rotv + ut * S);
                uint32_t slot;
                key = map_tdag<KeyT>(d, r, key, slot, Adag, sdag);
                rdag = Adag == 0 ? Amp<AmpT>::rot_zero()
                                 : (slot < (uint32_t)S ? rotv[ut * S + slot] : Amp<AmpT>::rot_table(d, Adag));
            }
            AmpT o0, o1;
            Amp<AmpT>::rot(rdag, Adag, true, sdag, a0, a1, o0, o1); /* R^dag */
            const bool c0 = act && Amp<AmpT>::keep(d, o0), c1 = act && Amp<AmpT>::keep(d, o1);
            const int kept = __popc(__ballot_sync(FULL, c0)) + __popc(__ballot_sync(FULL, c1));
            st.rdag += kept;
            st.hph += kept; /* H P H: -1 here */
            if (isext && act) {
                const Row r = slot_row(units[ut], ws + ut * S, rotv + ut * S);
                uint32_t slot;
                const KeyT kt = map_t<KeyT>(d, r, key, slot, At, st_neg);
                k_out = (uint32_t)(kt >> 1) & msk;
                kc_out = (uint32_t)(kt >> (1 + d.nb)) & msk;
                rt = At == 0 ? Amp<AmpT>::rot_zero()
                             : (slot < (uint32_t)S ? rotv[ut * S + slot] : Amp<AmpT>::rot_table(d, At));
            }
            AmpT r0, r1;
            Amp<AmpT>::rot(rt, At, false, st_neg, c0 ? Amp<AmpT>::neg(o0) : zero, c1 ? Amp<AmpT>::neg(o1) : zero,
                           r0, r1); /* R */
            const bool e0 = act && Amp<AmpT>::keep(d, r0), e1 = act && Amp<AmpT>::keep(d, r1);
            st.out += __popc(__ballot_sync(FULL, e0)) + __popc(__ballot_sync(FULL, e1));
            SlotOut<AmpT> outB, none;
            slot_out<AmpT>(d, out, units[ut], k_out, kc_out, b1, r0, r1, e0, e1, a.status, nrm, outB); /* S */
            none.b0 = none.b1 = -1;
            slot_store2<AmpT>(d, out, outB, none, a.status, nrm);
        }
        __syncwarp();
    }
    /* the garbage rows (jc != 0) */
    if (!skip) {
        for (int64_t su = gw; su < d.spill_slots; su += nwarps)
            if (in.count[d.dense_buckets + su] > 0) defer((int32_t)(0x80000000u | (uint32_t)su));
    }
    st.flush(a);

    /* end of the step: block partial of the norm; the last block to finish
       runs the deferred units through the row pipeline, then reduces */
    double nv = warp_sum(nrm.get());
    if (lane == 0) block_part[warp] = nv;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < WARPS; ++w) sum += block_part[w];
        a.partials[blockIdx.x] = sum;
        __threadfence();
        const unsigned prev = atomicAdd(a.done_ctr, 1u);
        is_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    const unsigned nd = *(volatile unsigned int *)a.deferred_ctr;
    double nd_nrm = 0.0;
    WalkStats st_ool;
    for (unsigned e = (unsigned)warp; e < nd; e += WARPS) {
        const uint32_t ent = (uint32_t)__ldcg(a.deferred + e);
        WalkItem<KeyT> it;
        it.valid = true;
        if (ent & 0x80000000u) { /* a garbage row: one row on its own */
            const int64_t su = (int64_t)(ent & 0x7fffffffu);
            it.bA = d.dense_buckets + su;
            it.bB = -1;
            it.n0 = min(__ldcg(in.count + it.bA), d.cap_row);
            it.n1 = 0;
            it.tagA = (KeyT)(__ldcg(in.spill + su) & 1ull) << B1;
        } else { /* a dense unit: its two rows as one segment */
            it.bA = 2 * (int64_t)ent;
            it.bB = it.bA + 1;
            it.n0 = min(__ldcg(in.count + it.bA), d.cap_row);
            it.n1 = min(__ldcg(in.count + it.bB), d.cap_row);
            it.tagA = 0;
        }
        nd_nrm += walk_item_ool<AmpT, KeyT>(d, in, out, a, it, rescale, scale_v, base, lay, &st_ool);
    }
    st_ool.flush(a);
    nd_nrm = warp_sum(nd_nrm);
    __syncthreads();
    if (lane == 0) block_part[warp] = nd_nrm;
    __syncthreads();
    double v = 0.0;
    for (unsigned bb = threadIdx.x; bb < gridDim.x; bb += blockDim.x) v += __ldcg(a.partials + bb);
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) block_part[warp] += v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < WARPS; ++w) tot += block_part[w];
        const bool clean = *(volatile int32_t *)a.status == 0;
        if (clean) {
            *a.norm_out = tot;
            if (a.scale_out) *a.scale_out = (a.renorm && tot > 0.0) ? sqrt(*a.renorm_target / tot) : 1.0;
            if (a.steps_done) *a.steps_done += 1;
            if (a.stats) a.stats[QW_STAT_STEPS] += 1;
        }
        *a.deferred_ctr = 0u;
        *a.work_ctr = 0u;
        *a.done_ctr = 0u;
    }
}

/* ==== positional walk step (walk_variant 7) ==================================== */
/*
 * The state of a one-instance walk held by position instead of by key.  At a
 * step boundary every branch that the walk reaches from T~|b~> sits in a row
 * (jc = 0, j < N, b1) with kc = A = 0, and its k is either a column of row j
 * (W = S (2 T~ Pi T~^dag - 1): the branches of T~ Pi's range are those of
 * T~'s rows, the swapped ones have k = a row whose padded column list holds j)
 * -- position 2 l + b2 for the column in slot l -- or one of the E_j rows x
 * whose slot l_x holds column j while row j holds no column x (a padded, so
 * unpaired, entry) -- position 2 s + 2 e + b2.  Row (j, b1) is pos_R = 2 s +
 * 2 pos_E amplitudes at (2 j + b1) pos_R; an absent branch is 0, so the
 * position is the key.
 *
 * The lane of slot (j, l) runs the slot kernel's arithmetic on the pairs of
 * both rows of j at positions 2 l, 2 l + 1 (T~^dag's maps take them to (l, 0),
 * T~'s back to k = col): R^dag, H P H (the zero-type sum over the unit's
 * lanes for b1 = 0, -1 for b1 = 1), R; S sends its b2 = 0 / 1 outputs to rows
 * (col, 0) / (col, 1) at position tp(j, l) + b1, where tp is the position of
 * k = j in row col.  An extra (j, b1, e) is outside every zero-type group and
 * its maps leave A = 0 (kc = x ^ col(j, 0) != 0 after O_s'^dag, so O_A' does
 * not fire): R(0) (-1) R(0)^dag = -1 on its pair, sent to positions 2 l_x + b1
 * of rows (x, 0 / 1).  Every position of the output has exactly
 * one writer, and pruned outputs are written as 0: no counts, atomics,
 * searches or keys, and nothing to clear between steps.
 */
/* launch shape of k_walk_pos per amplitude type (measured on GB300 at
   N = 16384, s = 16): complex64 runs fastest with 16 warps per SM and up to
   128 registers a thread (the next group's inputs held in registers while
   the current one computes), complex128 -- bound by the FP64 pipe -- with
   blocks of 4 warps, 5 per SM */
template <typename AmpT> struct PosCfg;
template <> struct PosCfg<float2> {
    static constexpr int warps = 8, blocks = 2;
    static constexpr bool even = true; /* grid: as many groups for every warp */
};
template <> struct PosCfg<double2> {
    static constexpr int warps = 4, blocks = 4;
    static constexpr bool even = false; /* grid: every resident block (FP64-pipe bound) */
};

template <typename AmpT> struct PosPair;
template <> struct PosPair<float2> {
    __device__ static void load(const float2 *p, float2 &a0, float2 &a1)
    {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        a0 = make_float2(v.x, v.y);
        a1 = make_float2(v.z, v.w);
    }
    __device__ static void store(float2 *p, float2 a0, float2 a1)
    {
        *reinterpret_cast<float4 *>(p) = make_float4(a0.x, a0.y, a1.x, a1.y);
    }
};
template <> struct PosPair<double2> {
    __device__ static void load(const double2 *p, double2 &a0, double2 &a1)
    {
        a0 = __ldg(p);
        a1 = __ldg(p + 1);
    }
    __device__ static void store(double2 *p, double2 a0, double2 a1)
    {
        p[0] = a0;
        p[1] = a1;
    }
};

/* per-lane branch counters of the positional step, summed over the warp at
   the end (the same quantities as WalkStats) */
struct PosStats {
    unsigned int rows = 0, in = 0, rdag = 0, hph = 0, out = 0;
    __device__ void flush(const QwStepArgs &a)
    {
        unsigned int v[5] = {rows, in, rdag, hph, out};
#pragma unroll
        for (int i = 0; i < 5; ++i)
            for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(FULL, v[i], o);
        if (a.stats && lane_id() == 0 && v[1]) {
            atomicAdd(a.stats + QW_STAT_ROWS, (unsigned long long)v[0]);
            atomicAdd(a.stats + QW_STAT_IN, (unsigned long long)v[1]);
            atomicAdd(a.stats + QW_STAT_RDAG, (unsigned long long)v[2]);
            atomicAdd(a.stats + QW_STAT_HPH, (unsigned long long)v[3]);
            atomicAdd(a.stats + QW_STAT_OUT, (unsigned long long)v[4]);
        }
    }
};

/* 1 for a non-zero amplitude (+-0 is zero), tested on the bits: an FP64
   comparison would take a slot of the FP64 pipe */
__device__ __forceinline__ unsigned int nz(float2 a)
{
    return ((__float_as_uint(a.x) | __float_as_uint(a.y)) << 1) != 0u ? 1u : 0u;
}
__device__ __forceinline__ unsigned int nz(double2 a)
{
    return (((uint64_t)__double_as_longlong(a.x) | (uint64_t)__double_as_longlong(a.y)) << 1) != 0ull ? 1u : 0u;
}

template <typename AmpT, int S, int PW>
__global__ void __launch_bounds__(PW * 32, PosCfg<AmpT>::blocks / (S > 32 ? 2 : 1))
    k_walk_pos(QwSimDev d, const AmpT *__restrict__ pin, AmpT *__restrict__ pout, QwStepArgs a)
{
    typedef typename Amp<AmpT>::RotVal RotVal;
    /* a unit (one j) on SW lanes, each lane holding SPL of its slots (l = lb
       + 32 k); RPP units per warp */
    constexpr int SW = S > 32 ? 32 : S, SPL = S / SW, RPP = 32 / SW;
    __shared__ double block_part[PW];
    __shared__ double scale_sm;
    __shared__ int is_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool skip = *(volatile int32_t *)a.status != 0;
    const bool rescale = a.scale_in != nullptr;
    const bool rot_in_place = Amp<AmpT>::kRotCode && d.rot_calc;
    typename Amp<AmpT>::Norm nrm;
    PosStats st;
    const AmpT zero = Amp<AmpT>::zero();
    /* 32-bit indices: the host keeps 2 N pos_R below 2^31 */
    const uint32_t R = (uint32_t)d.pos_R;
    const int E = d.pos_E;
    const uint32_t n = (uint32_t)d.pos_rows; /* rows of all instances */
    const uint32_t nall = (n + RPP - 1) / RPP, ngroups = skip ? 0u : nall;
    const uint32_t nwarps = gridDim.x * PW;
    const int ul = lane / SW, lb = lane % SW;
    const int nx = RPP * 2 * E; /* extra items of a group: (unit, b1, e) */
    /* the lane's first extra item is the same in every group */
    int x_u = 0, x_b1 = 0, x_e = 0;
    if (lane < nx) {
        x_u = lane / (2 * E);
        const int rem = lane - x_u * 2 * E;
        x_b1 = rem / E;
        x_e = rem - x_b1 * E;
    }
    /* a group's inputs, loaded one group ahead: the next group's loads are in
       flight while the current one computes */
    struct In {
        uint32_t rb;       /* first row of the row's instance */
        uint32_t w[SPL];   /* QRAM words */
        RotVal t[SPL];
        int tp[SPL];
        AmpT a0[SPL], a1[SPL], q0[SPL], q1[SPL];
        uint32_t xe; /* the lane's first extra item: x << 8 | l_x, 0xffffffff if none */
        AmpT x0, x1;
    };
    /* extra item (u, b1, e) of group gg: its entry and pair (none past the
       row's extras count) */
    auto fetch_extra = [&](uint32_t gg, int u, int b1, int e, uint32_t &xe, AmpT &x0, AmpT &x1) {
        const uint32_t jx = gg * RPP + u;
        xe = 0xffffffffu;
        x0 = x1 = zero;
        if (gg < nall && jx < n && e < (int)__ldg(d.pos_xcnt + jx)) {
            xe = __ldg(d.pos_xin + jx * (uint32_t)E + e);
            PosPair<AmpT>::load(pin + (2 * jx + b1) * R + 2 * S + 2 * e, x0, x1);
        }
    };
    auto fetch = [&](uint32_t gg, In &x) {
        const uint32_t jj = gg * RPP + ul;
        const bool have = gg < nall && jj < n;
        x.rb = 0;
        if (have && d.pos_rowbase) x.rb = __ldg(d.pos_rowbase + jj);
#pragma unroll
        for (int k = 0; k < SPL; ++k) {
            const uint32_t l = lb + 32 * k;
            x.w[k] = 0;
            x.t[k] = Amp<AmpT>::rot_zero();
            x.tp[k] = 0;
            x.a0[k] = x.a1[k] = x.q0[k] = x.q1[k] = zero;
            if (have) {
                const uint32_t at = jj * S + l;
                x.w[k] = __ldg(d.img + at);
                if (!rot_in_place) x.t[k] = __ldg(static_cast<const RotVal *>(d.slot_rot) + at);
                x.tp[k] = __ldg(d.pos_tp + at);
                PosPair<AmpT>::load(pin + 2 * jj * R + 2 * l, x.a0[k], x.a1[k]);
                PosPair<AmpT>::load(pin + (2 * jj + 1) * R + 2 * l, x.q0[k], x.q1[k]);
            }
        }
        x.xe = 0xffffffffu;
        x.x0 = x.x1 = zero;
        if (lane < nx) fetch_extra(gg, x_u, x_b1, x_e, x.xe, x.x0, x.x1);
    };
    In nxt;
    fetch(blockIdx.x * PW + warp, nxt);
    /* the renormalisation factor, staged once per block while the first
       group's loads are in flight */
    if (threadIdx.x == 0) Amp<AmpT>::Scale::to_shared(rescale ? *a.scale_in : 1.0, &scale_sm);
    __syncthreads();
    const typename Amp<AmpT>::Scale scale = Amp<AmpT>::Scale::from_shared(&scale_sm);
    for (uint32_t g = blockIdx.x * PW + warp; g < ngroups; g += nwarps) {
        const In cur = nxt;
        fetch(g + nwarps, nxt);
        const uint32_t j = g * RPP + ul;
        const bool valid = j < n;
        RotVal rv[SPL];
        uint32_t val[SPL], gc[SPL];
        bool sneg[SPL];
        AmpT a0[SPL], a1[SPL], q0[SPL], q1[SPL];
        unsigned int nin = 0;
#pragma unroll
        for (int k = 0; k < SPL; ++k) {
            const uint32_t w = cur.w[k];
            val[k] = w & 0xffffu;
            /* a 0 element rotates by R(0); complex64 derives the float pairs
               from the value word (4 MB less read per step than the per-slot
               table at N = 16384, s = 16) */
            rv[k] = val[k] == 0 ? Amp<AmpT>::rot_zero() : (rot_in_place ? Amp<AmpT>::rot_code(val[k]) : cur.t[k]);
            gc[k] = cur.rb + (w >> 16); /* the column's row among all instances' rows */
            sneg[k] = j > gc[k];        /* j > col within the instance */
            a0[k] = cur.a0[k];
            a1[k] = cur.a1[k];
            q0[k] = cur.q0[k];
            q1[k] = cur.q1[k];
            if (valid && rescale) {
                a0[k] = scale.apply(a0[k]);
                a1[k] = scale.apply(a1[k]);
                q0[k] = scale.apply(q0[k]);
                q1[k] = scale.apply(q1[k]);
            }
            nin += nz(a0[k]) + nz(a1[k]) + nz(q0[k]) + nz(q1[k]);
        }
        st.in += nin;
        {
            const unsigned m = __ballot_sync(FULL, nin != 0);
            const unsigned um = SW == 32 ? m : (m >> (ul * SW)) & ((1u << (SW & 31)) - 1u);
            if (lb == 0 && um != 0) st.rows += 1; /* units holding branches */
        }

        /* b1 = 0: R^dag, H P H on the zero-type group (the unit's slots), R */
        AmpT rA0[SPL], rA1[SPL];
        bool eA0[SPL], eA1[SPL];
        {
            AmpT o1[SPL], z0[SPL];
            bool c1[SPL];
#pragma unroll
            for (int k = 0; k < SPL; ++k) {
                AmpT o0;
                Amp<AmpT>::rot(rv[k], val[k], true, sneg[k], a0[k], a1[k], o0, o1[k]);
                const bool c0 = Amp<AmpT>::keep(d, o0);
                c1[k] = Amp<AmpT>::keep(d, o1[k]);
                st.rdag += (c0 ? 1u : 0u) + (c1[k] ? 1u : 0u);
                z0[k] = c0 ? o0 : zero;
            }
            typename Amp<AmpT>::Sum sum;
            sum.set(z0[0]);
#pragma unroll
            for (int k = 1; k < SPL; ++k) sum.add(z0[k]);
            sum.reduce(SW, SW);
            if (a.qls_readout && valid && lb == 0) {
                const double2 sv = sum.value();
                const double coef = a.qls_coefs[*a.qls_j];
                double2 acc = a.qls_y[j];
                acc.x += coef * (d.inv_sqrt_s * sv.x);
                acc.y += coef * (d.inv_sqrt_s * sv.y);
                a.qls_y[j] = acc;
            }
#pragma unroll
            for (int k = 0; k < SPL; ++k) {
                const AmpT h0 = sum.scaled_minus(d.two_over_s, z0[k]);
                const bool d0 = Amp<AmpT>::keep(d, h0);
                st.hph += (d0 ? 1u : 0u) + (c1[k] ? 1u : 0u);
                Amp<AmpT>::rot(rv[k], val[k], false, sneg[k], d0 ? h0 : zero, c1[k] ? Amp<AmpT>::neg(o1[k]) : zero,
                               rA0[k], rA1[k]);
                eA0[k] = Amp<AmpT>::keep(d, rA0[k]);
                eA1[k] = Amp<AmpT>::keep(d, rA1[k]);
            }
        }
        /* b1 = 1: R^dag, -1, R, then S: rows (col, 0) and (col, 1), positions
           tp (from b1 = 0) and tp + 1 (from b1 = 1) */
#pragma unroll
        for (int k = 0; k < SPL; ++k) {
            AmpT rB0, rB1;
            AmpT o0, o1;
            /* in the walk's reachable states the b2 = 1 member of a b1 = 1 pair
               is 0: then R^dag takes half the products (same results).  Taken
               on the FP64-pipe-bound complex128 path only: on complex64 the
               vote and the second code path cost more than the products */
            if (Amp<AmpT>::kB2ZeroPath && __all_sync(FULL, nz(q1[k]) == 0u))
                Amp<AmpT>::rot_dag_b2zero(rv[k], val[k], sneg[k], q0[k], o0, o1);
            else
                Amp<AmpT>::rot(rv[k], val[k], true, sneg[k], q0[k], q1[k], o0, o1);
            const bool c0 = Amp<AmpT>::keep(d, o0), c1 = Amp<AmpT>::keep(d, o1);
            const unsigned int kept = (c0 ? 1u : 0u) + (c1 ? 1u : 0u);
            st.rdag += kept;
            st.hph += kept;
            Amp<AmpT>::rot(rv[k], val[k], false, sneg[k], c0 ? Amp<AmpT>::neg(o0) : zero,
                           c1 ? Amp<AmpT>::neg(o1) : zero, rB0, rB1);
            const bool eB0 = Amp<AmpT>::keep(d, rB0), eB1 = Amp<AmpT>::keep(d, rB1);
            if (valid) {
                const AmpT s0 = eA0[k] ? rA0[k] : zero, s1 = eB0 ? rB0 : zero;
                const AmpT s2 = eA1[k] ? rA1[k] : zero, s3 = eB1 ? rB1 : zero;
                if (eA0[k]) nrm.add(rA0[k]);
                if (eB0) nrm.add(rB0);
                if (eA1[k]) nrm.add(rA1[k]);
                if (eB1) nrm.add(rB1);
                st.out += (eA0[k] ? 1u : 0u) + (eB0 ? 1u : 0u) + (eA1[k] ? 1u : 0u) + (eB1 ? 1u : 0u);
                const uint32_t tp = (uint32_t)cur.tp[k];
                PosPair<AmpT>::store(pout + 2 * gc[k] * R + tp, s0, s1);
                PosPair<AmpT>::store(pout + (2 * gc[k] + 1) * R + tp, s2, s3);
            }
        }

        /* the extras of the group's rows: the lane's first item prefetched, any
           further ones (more than 32 per group) loaded here */
        for (int it = lane; it < nx; it += 32) {
            int xb1 = x_b1;
            uint32_t xe = cur.xe;
            AmpT x0 = cur.x0, x1 = cur.x1;
            if (it != lane) {
                const int uu = it / (2 * E), rem = it - uu * 2 * E;
                xb1 = rem / E;
                fetch_extra(g, uu, xb1, rem - xb1 * E, xe, x0, x1);
            }
            if (xe == 0xffffffffu) continue;
            if (rescale) {
                x0 = scale.apply(x0);
                x1 = scale.apply(x1);
            }
            st.in += nz(x0) + nz(x1);
            /* R(0) (-1) R(0)^dag with R(0) = [[0, -1], [1, 0]]: R(0)^dag gives
               (x1, -x0), -1 and R(0) give (-x0, -x1) -- each output the
               negated input, kept where the input is (every product is by
               0 or 1, so this is the general rotation's result exactly) */
            const bool k0 = Amp<AmpT>::keep(d, x0), k1 = Amp<AmpT>::keep(d, x1);
            const unsigned int kept = (k0 ? 1u : 0u) + (k1 ? 1u : 0u);
            st.rdag += kept;
            st.hph += kept;
            st.out += kept;
            const AmpT r0 = Amp<AmpT>::neg(x0), r1 = Amp<AmpT>::neg(x1);
            if (k0) nrm.add(r0);
            if (k1) nrm.add(r1);
            const uint32_t x = xe >> 8, px = 2 * (xe & 0xffu) + (uint32_t)xb1;
            pout[2 * x * R + px] = k0 ? r0 : zero;
            pout[(2 * x + 1) * R + px] = k1 ? r1 : zero;
        }
    }
    st.flush(a);

    /* end of the step: block partial of the norm, the last block reduces */
    const double nv = nrm.warp_total();
    if (lane == 0) block_part[warp] = nv;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < PW; ++w) sum += block_part[w];
        a.partials[blockIdx.x] = sum;
        __threadfence();
        const unsigned prev = atomicAdd(a.done_ctr, 1u);
        is_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double v = 0.0;
    for (unsigned bb = threadIdx.x; bb < gridDim.x; bb += blockDim.x) v += __ldcg(a.partials + bb);
    v = warp_sum(v);
    if (lane == 0) block_part[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < PW; ++w) tot += block_part[w];
        const bool clean = *(volatile int32_t *)a.status == 0;
        if (clean) {
            *a.norm_out = tot;
            if (a.scale_out) *a.scale_out = (a.renorm && tot > 0.0) ? sqrt(*a.renorm_target / tot) : 1.0;
            if (a.steps_done) *a.steps_done += 1;
            if (a.stats) a.stats[QW_STAT_STEPS] += 1;
        }
        *a.done_ctr = 0u;
    }
}

/* T~|b~> written straight into the positional layout for rows g0 .. g0 + n
 * of pbuf (one instance): |b~> holds one branch per row, a = b_j (divided by
 * the pending renormalisation factor when other instances share the state);
 * T~'s Hadamard gives (l, z = 0) with a / sqrt(s) for every slot l, its maps
 * take slot l to k = col(j, l), and R(A_jl) on (a / sqrt(s), 0) gives the
 * pair at positions 2 l, 2 l + 1 of row (j, b1 = 0) -- the arithmetic of
 * k_tinit.  Every other position of both rows is written 0.  One thread per
 * position. */
template <typename AmpT>
__global__ void k_tinit_pos(QwSimDev d, AmpT *pbuf, int64_t g0, int64_t n, const double *b_re, const double *b_im,
                            const double *scale)
{
    typedef typename Amp<AmpT>::RotVal RotVal;
    const int S = d.s;
    const int64_t R = d.pos_R, total = 2 * n * R;
    const AmpT zero = Amp<AmpT>::zero();
    const bool rot_in_place = Amp<AmpT>::kRotCode && d.rot_calc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / R, j = r >> 1;
        const int q = (int)(i - r * R);
        AmpT out = zero;
        if ((r & 1) == 0 && q < 2 * S) {
            double2 v = make_double2(b_re[j], b_im ? b_im[j] : 0.0);
            if (scale) v = make_double2(v.x / *scale, v.y / *scale);
            const double2 a = Amp<AmpT>::to_d(Amp<AmpT>::from_d(v)); /* as stored by |b~> */
            const AmpT h = Amp<AmpT>::from_d(make_double2(d.inv_sqrt_s * a.x, d.inv_sqrt_s * a.y));
            if ((v.x != 0.0 || v.y != 0.0) && Amp<AmpT>::keep(d, h)) {
                const int64_t at = (g0 + j) * S + (q >> 1);
                const uint32_t w = __ldg(d.img + at), val = w & 0xffffu;
                const RotVal rv = val == 0 ? Amp<AmpT>::rot_zero()
                                           : (rot_in_place ? Amp<AmpT>::rot_code(val)
                                                           : __ldg(static_cast<const RotVal *>(d.slot_rot) + at));
                AmpT o0, o1;
                Amp<AmpT>::rot(rv, val, false, (uint32_t)j > (w >> 16), h, zero, o0, o1); /* R */
                const AmpT o = (q & 1) ? o1 : o0;
                if (Amp<AmpT>::keep(d, o)) out = o;
            }
        }
        pbuf[2 * g0 * R + i] = out;
    }
}

/* Marginal of one register over instance rows g0 .. g0 + n of the
 * positional layout (the key of a position: jc = kc = 0, j = its row, b1, k
 * = the slot's column or the extra's row, b2 = position & 1).  A warp per j
 * reads both rows whole (positions past a row's extras are 0), all loads in
 * flight together; the row registers (jc, j, b1) add their sums once. */
template <typename AmpT>
__global__ void k_measure_pos(QwSimDev d, const AmpT *pbuf, int64_t g0, int64_t n, const double *scale, int reg,
                              double *probs, int64_t len)
{
    const int S = d.s, E = d.pos_E;
    const int R = d.pos_R;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double sc = scale ? *scale : 1.0;
    for (int64_t j = warp; j < n; j += nw) {
        const int64_t g = g0 + j;
        const AmpT *rows = pbuf + 2 * g * R; /* rows (j, 0) and (j, 1) */
        double acc[2] = {0.0, 0.0};
        for (int q2 = lane; q2 < 2 * R; q2 += 32) {
            double2 a = Amp<AmpT>::to_d(rows[q2]);
            if (a.x == 0.0 && a.y == 0.0) continue;
            if (scale) a = make_double2(sc * a.x, sc * a.y);
            const double p = a.x * a.x + a.y * a.y;
            const int b1 = q2 >= R ? 1 : 0, q = q2 - b1 * R;
            if (reg <= 2) {
                acc[reg == 2 ? b1 : 0] += p;
                continue;
            }
            uint64_t v = 0; /* kc = 0 */
            if (reg == 4) v = q < 2 * S ? (d.img[g * S + (q >> 1)] >> 16)
                                        : (uint64_t)((d.pos_xin[g * E + ((q - 2 * S) >> 1)] >> 8) - (uint32_t)g0);
            else if (reg == 5) v = (uint64_t)(q & 1);
            if ((int64_t)v < len) atomicAdd(probs + v, p);
        }
        if (reg <= 2) {
            for (int t = 0; t < 2; ++t)
                for (int o = 16; o > 0; o >>= 1) acc[t] += __shfl_xor_sync(FULL, acc[t], o);
            if (lane == 0) {
                if (reg == 1) {
                    if (j < len && acc[0] != 0.0) atomicAdd(probs + j, acc[0]);
                } else {
                    for (int t = 0; t < 2; ++t) {
                        const int64_t v = reg == 2 ? t : 0;
                        if (v < len && acc[t] != 0.0) atomicAdd(probs + v, acc[t]);
                    }
                }
            }
        }
    }
}

/* the row buckets into the positional layout (pbuf zeroed by the caller):
   one thread per bucket slot */
template <typename AmpT>
__global__ void k_pos_pack(QwSimDev d, QwBufDev buf, AmpT *pbuf, int32_t *status)
{
    const int S = d.s, E = d.pos_E;
    const int64_t total = d.total_buckets * (int64_t)d.cap_row;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / d.cap_row;
        const int p = (int)(i - b * d.cap_row);
        if (p >= buf.count[b]) continue;
        if (b >= d.dense_buckets) { /* a row with jc != 0 */
            atomicOr(status, QW_ST_POS_UNREP);
            continue;
        }
        int64_t j = b >> 1, n = d.n_single, g0 = 0;
        if (d.ninst > 1) {
            const int inst = d.unit_inst[b >> 1];
            j = (b - d.inst_bkt[inst]) >> 1;
            n = d.inst_n[inst];
            g0 = d.inst_img[inst] / S;
        }
        if (j >= n) { /* a row j >= N */
            atomicOr(status, QW_ST_POS_UNREP);
            continue;
        }
        const int64_t gr = g0 + j; /* the row among all instances' rows */
        const Regs x = decode_r(buf.key[i], d.nb);
        int pos = -1;
        if (x.kc == 0 && x.A == 0) {
            const uint32_t *row = d.img + gr * S;
            int lo = 0, hi = S; /* lower bound of k among the row's sorted columns */
            while (lo < hi) {
                const int m = (lo + hi) >> 1;
                if ((row[m] >> 16) < x.k) lo = m + 1;
                else hi = m;
            }
            if (lo < S && (row[lo] >> 16) == x.k) {
                pos = 2 * lo + (int)x.b2;
            } else {
                const int ne = d.pos_xcnt[gr];
                for (int e = 0; e < ne; ++e)
                    if ((d.pos_xin[gr * E + e] >> 8) - g0 == x.k) {
                        pos = 2 * S + 2 * e + (int)x.b2;
                        break;
                    }
            }
        }
        if (pos < 0) {
            atomicOr(status, QW_ST_POS_UNREP);
            continue;
        }
        pbuf[(2 * gr + (b & 1)) * d.pos_R + pos] = static_cast<const AmpT *>(buf.amp)[i];
    }
}

/* the positional layout into the row buckets (cleared by the caller): one
   thread per position, non-zero amplitudes appended to their row */
template <typename AmpT>
__global__ void k_pos_unpack(QwSimDev d, const AmpT *pbuf, QwBufDev buf, int32_t *status)
{
    const int S = d.s, E = d.pos_E;
    const int64_t R = d.pos_R, total = 2 * d.pos_rows * R;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const AmpT v = pbuf[i];
        if (v.x == 0 && v.y == 0) continue;
        const int64_t r = i / R;
        const int q = (int)(i - r * R);
        const int64_t gr = r >> 1; /* the row among all instances' rows */
        int64_t g0 = 0, bk = r;    /* the instance's first row; the bucket */
        if (d.ninst > 1) {
            const int inst = d.pos_rowinst[gr];
            g0 = d.inst_img[inst] / S;
            bk = d.inst_bkt[inst] + 2 * (gr - g0) + (r & 1);
        }
        Regs x;
        x.kc = 0;
        x.A = 0;
        x.b2 = (uint32_t)(q & 1);
        if (q < 2 * S) {
            x.k = d.img[gr * S + (q >> 1)] >> 16;
        } else {
            const int e = (q - 2 * S) >> 1;
            if (e >= (int)d.pos_xcnt[gr]) { /* never written: not a branch */
                atomicOr(status, QW_ST_POS_UNREP);
                continue;
            }
            x.k = (d.pos_xin[gr * E + e] >> 8) - (uint32_t)g0;
        }
        const int64_t r_b = bk;
        const int p = atomicAdd(buf.count + r_b, 1);
        if (p >= d.cap_row) {
            atomicOr(status, QW_ST_ROW_OVERFLOW);
            continue;
        }
        const int64_t sl = r_b * d.cap_row + p;
        buf.key[sl] = encode_r(x, d.nb);
        static_cast<AmpT *>(buf.amp)[sl] = v;
    }
}

/* T~ on |b~> (qw_state_init): every row (jc = 0, j, b1 = 0) of the range
 * holds at most the one branch k = kc = b2 = A = 0.  T~'s Hadamard turns it
 * into the s branches (l, z = 0) with amplitude a / sqrt(s) (a group with a
 * single member at u = 0); then the maps and R of T~ as in the step kernel;
 * the row does not change (no S).  A row holding anything else sets the
 * status bit QW_ST_NOT_BTILDE (the state was not |b~>). */
template <typename AmpT, typename KeyT>
__global__ void __launch_bounds__(WARPS * 32) k_tinit(QwSimDev d, QwBufDev buf, int64_t lo, int64_t hi,
                                                      int32_t *status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int C = d.warp_cap;
    const WalkLayout lay = walk_layout<AmpT, KeyT>(d);
    unsigned char *base = smem + lay.per_warp * warp;
    KeyT *kP = reinterpret_cast<KeyT *>(base + lay.kP);
    KeyT *kQ = reinterpret_cast<KeyT *>(base + lay.kQ);
    AmpT *aP = reinterpret_cast<AmpT *>(base + lay.aP);
    AmpT *aQ = reinterpret_cast<AmpT *>(base + lay.aQ);
    uint32_t *simg = reinterpret_cast<uint32_t *>(base + lay.simg);
    int16_t *hidx = reinterpret_cast<int16_t *>(base + lay.hidx);
    for (int64_t b = lo + (int64_t)blockIdx.x * WARPS + warp; b < hi; b += (int64_t)gridDim.x * WARPS) {
        const int n = buf.count[b];
        if (n <= 0) continue;
        const int64_t row0 = b * (int64_t)d.cap_row;
        if (n != 1 || buf.key[row0] != 0ull) {
            if (lane == 0) atomicOr(status, QW_ST_NOT_BTILDE);
            continue;
        }
        Row r;
        if (!row_of(d, buf, b, r)) continue;
        r.simg = simg;
        r.sfg = nullptr;
        for (int t = lane; t < d.s; t += 32)
            simg[t] = r.valid ? __ldg(d.img + r.img_base + (int64_t)r.j * d.s + t) : 0u;
        const double2 a = Amp<AmpT>::to_d(static_cast<const AmpT *>(buf.amp)[row0]);
        const AmpT h = Amp<AmpT>::from_d(make_double2(d.inv_sqrt_s * a.x, d.inv_sqrt_s * a.y));
        const bool kept = Amp<AmpT>::keep(d, h);
        int m = 0;
        if (kept) {
            for (int u = lane; u < d.s; u += 32) {
                kP[u] = (KeyT)u << 1;
                aP[u] = h;
            }
            m = d.s;
        }
        __syncwarp();
        PairSink<AmpT, KeyT, false> s1(d, r, kQ, aQ, C, nullptr, nullptr, nullptr);
        map_rot_pairs<1, AmpT, KeyT>(d, r, kP, aP, m, s1, hidx);
        m = sink_count(s1, status);
        /* write back in place: the row keeps its registers (jc, j, b1) */
        for (int i = lane; i < m && i < d.cap_row; i += 32) {
            buf.key[row0 + i] = (uint64_t)kQ[i]; /* b2 | k | kc, A = 0, no b1 tag */
            static_cast<AmpT *>(buf.amp)[row0 + i] = aQ[i];
        }
        if (m > d.cap_row && lane == 0) atomicOr(status, QW_ST_ROW_OVERFLOW);
        __syncwarp();
        if (lane == 0) buf.count[b] = m < d.cap_row ? m : d.cap_row;
    }
}

/* ---- small kernels ------------------------------------------------------------ */

/* Row buckets moved to a larger row capacity: bucket b's entries from
 * b * cap_old to b * cap_new (counts and the garbage-row table unchanged). */
__global__ void k_regrow(int64_t buckets, const int32_t *count, int cap_old, int cap_new, const uint64_t *key_old,
                         const unsigned char *amp_old, uint64_t *key_new, unsigned char *amp_new, int amp_bytes)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (int64_t b = warp; b < buckets; b += nw) {
        int n = count[b];
        if (n > cap_old) n = cap_old;
        for (int i = lane; i < n; i += 32) {
            const int64_t so = b * (int64_t)cap_old + i, sn = b * (int64_t)cap_new + i;
            key_new[sn] = key_old[so];
            for (int t = 0; t < amp_bytes; t += 8)
                *reinterpret_cast<uint64_t *>(amp_new + sn * amp_bytes + t) =
                    *reinterpret_cast<const uint64_t *>(amp_old + so * amp_bytes + t);
        }
    }
}


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
__global__ void k_init_b(QwSimDev d, QwBufDev buf, int inst, const double *b_re, const double *b_im, int n,
                         const double *scale)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double2 v = make_double2(b_re[j], b_im ? b_im[j] : 0.0);
    if (v.x == 0.0 && v.y == 0.0) return;
    if (d.nparts > 1 && qw_part_owner_of(d, 0u, (uint32_t)j) != d.part) return; /* another partition's row */
    if (scale) v = make_double2(v.x / *scale, v.y / *scale);
    const int64_t b = d.inst_bkt[inst] + ((int64_t)j << 1);
    const int64_t slot = b * (int64_t)d.cap_row;
    buf.key[slot] = 0ull;
    store_amp<AmpT>(buf.amp, slot, v);
    buf.count[b] = 1;
}

/* Append imported branches (row key, local key, amplitude) to their rows. */
template <typename AmpT>
__global__ void k_import(QwSimDev d, QwBufDev buf, const uint64_t *rowkey, const uint64_t *local,
                         const double2 *amp, int64_t count, int32_t *status)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint64_t rk = rowkey[i];
    const uint32_t inst = (uint32_t)(rk >> 40), jc = (uint32_t)((rk >> 20) & 0xfffffu);
    const uint32_t j = (uint32_t)((rk >> 1) & 0x7ffffu), b1 = (uint32_t)(rk & 1);
    const int64_t b = bucket_of(d, buf, inst, jc, j, b1, status);
    if (b < 0) return;
    const int pos = atomicAdd(buf.count + b, 1);
    if (pos >= d.cap_row) {
        atomicOr(status, QW_ST_ROW_OVERFLOW);
        return;
    }
    const int64_t slot = b * (int64_t)d.cap_row + pos;
    buf.key[slot] = local[i];
    store_amp<AmpT>(buf.amp, slot, amp[i]);
}

/* Branches received from other partitions (their S outputs for rows this
 * partition owns) appended to the buckets of their rows. */
/* one received entry appended to its row */
template <typename AmpT>
__device__ __forceinline__ void part_append(const QwSimDev &d, const QwBufDev &buf, const QwPartEntry &x,
                                            int32_t *status)
{
    const uint64_t rk = x.rowkey;
    const uint32_t inst = (uint32_t)(rk >> 40), jc = (uint32_t)((rk >> 20) & 0xfffffu);
    const uint32_t j = (uint32_t)((rk >> 1) & 0x7ffffu), b1 = (uint32_t)(rk & 1);
    const int64_t b = bucket_of(d, buf, inst, jc, j, b1, status);
    if (b < 0) return;
    const int pos = atomicAdd(buf.count + b, 1);
    if (pos >= d.cap_row) {
        atomicOr(status, QW_ST_ROW_OVERFLOW);
        return;
    }
    const int64_t slot = b * (int64_t)d.cap_row + pos;
    buf.key[slot] = x.local;
    store_amp<AmpT>(buf.amp, slot, make_double2(x.re, x.im));
}

template <typename AmpT>
__global__ void k_part_inbox(QwSimDev d, QwBufDev buf, const QwPartEntry *e, int64_t count, int32_t *status)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        part_append<AmpT>(d, buf, e[i], status);
}

/* The entries the other partitions' S sent here, appended straight from
 * their outbox segments (their counts read on the device: no host round
 * trip), one thread per entry slot of every source. */
template <typename AmpT>
__global__ void k_part_gather(QwSimDev d, QwBufDev buf, QwPartSources src, int32_t *status)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nthr = (int64_t)gridDim.x * blockDim.x;
    for (int k = 0; k < src.n; ++k) {
        const unsigned long long c = *src.count[k];
        const int64_t m = (int64_t)c < src.cap ? (int64_t)c : src.cap;
        for (int64_t i = tid; i < m; i += nthr) part_append<AmpT>(d, buf, src.e[k][i], status);
    }
}

/* The renormalisation factor of a partition from the norms of all parts'
 * outputs of the step: scale = sqrt(target / sum) (1 without renorm). */
__global__ void k_part_scale(QwPartNorms nm, const double *target, double *scale_out, int renorm)
{
    double sum = 0.0;
    for (int p = 0; p < nm.n; ++p) sum += *nm.norm[p];
    *scale_out = (renorm && sum > 0.0) ? sqrt(*target / sum) : 1.0;
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

/* p[j] = ||Y||^2 for the current term j = *jctr, then advance the term. */
__global__ void k_qls_norm(const double2 *y, int n, double *p, int64_t *jctr)
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
        const int64_t j = *jctr;
        p[j] = t;
        *jctr = j + 1;
    }
}

template <typename AmpT, int MODE> size_t step_smem(const QwSimDev &d)
{
    return (size_t)WARPS * ((size_t)d.warp_cap * 2 * (sizeof(double2) + sizeof(uint64_t)) +
                            (((size_t)d.s * sizeof(uint32_t) + 15) & ~(size_t)15));
}

template <typename AmpT, bool PF, bool SEG, typename KeyT>
int walk_grid_k(const QwSimDev &d)
{
    const size_t sm = (size_t)WARPS * walk_layout<AmpT, KeyT>(d).per_warp;
    cudaFuncSetAttribute(k_walk<AmpT, PF, SEG, KeyT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk<AmpT, PF, SEG, KeyT>, WARPS * 32, sm);
    if (per_sm < 1) per_sm = 1;
    int64_t want = (d.total_buckets + WARPS - 1) / WARPS;
    int64_t g = (int64_t)per_sm * qw_sm_count();
    if (want < g) g = want;
    return (int)(g < 1 ? 1 : g);
}

template <typename AmpT, bool PF, bool SEG>
int walk_grid_t(const QwSimDev &d)
{
    return key32_fits(d) ? walk_grid_k<AmpT, PF, SEG, uint32_t>(d) : walk_grid_k<AmpT, PF, SEG, uint64_t>(d);
}

template <typename AmpT, bool PF, bool SEG>
cudaError_t launch_walk_t(const QwSimDev &d, const QwBufDev &in, const QwBufDev &out,
                          const QwBufDev &clr, const QwStepArgs &a, int grid, cudaStream_t st)
{
    if (key32_fits(d)) {
        const size_t sm = (size_t)WARPS * walk_layout<AmpT, uint32_t>(d).per_warp;
        k_walk<AmpT, PF, SEG, uint32_t><<<grid, WARPS * 32, sm, st>>>(d, in, out, clr, a);
    } else {
        const size_t sm = (size_t)WARPS * walk_layout<AmpT, uint64_t>(d).per_warp;
        k_walk<AmpT, PF, SEG, uint64_t><<<grid, WARPS * 32, sm, st>>>(d, in, out, clr, a);
    }
    return cudaGetLastError();
}

template <typename AmpT>
size_t walk_smem_bytes(const QwSimDev &d)
{
    return (size_t)WARPS * (key32_fits(d) ? walk_layout<AmpT, uint32_t>(d).per_warp
                                          : walk_layout<AmpT, uint64_t>(d).per_warp);
}

template <typename AmpT, typename KeyT>
void launch_tinit_k(const QwSimDev &d, const QwBufDev &buf, int64_t lo, int64_t hi, int grid, int32_t *status,
                    cudaStream_t st)
{
    const size_t sm = (size_t)WARPS * walk_layout<AmpT, KeyT>(d).per_warp;
    cudaFuncSetAttribute(k_tinit<AmpT, KeyT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_tinit<AmpT, KeyT><<<grid, WARPS * 32, sm, st>>>(d, buf, lo, hi, status);
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

/* slot kernel: s in {8, 16, 32} */
template <typename AmpT, int S, typename KeyT>
int slot_grid_k(const QwSimDev &d)
{
    const size_t sm = (size_t)WARPS * slot_per_warp<AmpT, KeyT>(d);
    cudaFuncSetAttribute(k_walk_slot<AmpT, S, KeyT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk_slot<AmpT, S, KeyT>, WARPS * 32, sm);
    if (per_sm < 1) per_sm = 1;
    const int64_t groups = ((d.dense_buckets >> 1) + (32 / S) - 1) / (32 / S);
    int64_t want = (groups + d.spill_slots + WARPS - 1) / WARPS;
    int64_t g = (int64_t)per_sm * qw_sm_count();
    if (want < g) g = want;
    return (int)(g < 1 ? 1 : g);
}

template <typename AmpT, int S>
int slot_grid_s(const QwSimDev &d)
{
    return key32_fits(d) ? slot_grid_k<AmpT, S, uint32_t>(d) : slot_grid_k<AmpT, S, uint64_t>(d);
}

template <typename AmpT>
int slot_grid_t(const QwSimDev &d)
{
    if (d.s == 8) return slot_grid_s<AmpT, 8>(d);
    if (d.s == 16) return slot_grid_s<AmpT, 16>(d);
    return slot_grid_s<AmpT, 32>(d);
}

template <typename AmpT, int S>
cudaError_t launch_slot_s(const QwSimDev &d, const QwBufDev &in, const QwBufDev &out, const QwBufDev &clr,
                          const QwStepArgs &a, int grid, cudaStream_t st)
{
    if (key32_fits(d)) {
        const size_t sm = (size_t)WARPS * slot_per_warp<AmpT, uint32_t>(d);
        k_walk_slot<AmpT, S, uint32_t><<<grid, WARPS * 32, sm, st>>>(d, in, out, clr, a);
    } else {
        const size_t sm = (size_t)WARPS * slot_per_warp<AmpT, uint64_t>(d);
        k_walk_slot<AmpT, S, uint64_t><<<grid, WARPS * 32, sm, st>>>(d, in, out, clr, a);
    }
    return cudaGetLastError();
}

template <typename AmpT>
cudaError_t launch_slot_t(const QwSimDev &d, const QwBufDev &in, const QwBufDev &out, const QwBufDev &clr,
                          const QwStepArgs &a, int grid, cudaStream_t st)
{
    if (d.s == 8) return launch_slot_s<AmpT, 8>(d, in, out, clr, a, grid, st);
    if (d.s == 16) return launch_slot_s<AmpT, 16>(d, in, out, clr, a, grid, st);
    return launch_slot_s<AmpT, 32>(d, in, out, clr, a, grid, st);
}

template <typename AmpT>
size_t slot_smem_bytes(const QwSimDev &d)
{
    return (size_t)WARPS * (key32_fits(d) ? slot_per_warp<AmpT, uint32_t>(d) : slot_per_warp<AmpT, uint64_t>(d));
}

template <typename AmpT, int S>
int pos_grid_s(const QwSimDev &d)
{
    constexpr int PW = PosCfg<AmpT>::warps;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk_pos<AmpT, S, PW>, PW * 32, 0);
    if (per_sm < 1) per_sm = 1;
    /* complex64: as many groups for every warp -- with k = ceil(groups /
       resident warps) groups a warp, the fewest blocks that cover them (a warp
       with fewer groups than the others would wait for them at the end of the
       step); complex128, bound by each SM's FP64 pipe: every resident block,
       so that every SM holds the same share (measured at N = 16384: 24.0 vs
       25.4 us per flushed complex64 step, 57.0 vs 51.2 us complex128) */
    constexpr int RPP = 32 / (S > 32 ? 32 : S);
    const int64_t groups = (d.pos_rows + RPP - 1) / RPP;
    const int64_t cap = (int64_t)per_sm * qw_sm_count();
    const int64_t want = (groups + PW - 1) / PW;
    int64_t g = want < cap ? want : cap;
    if (PosCfg<AmpT>::even) {
        const int64_t k = (groups + cap * PW - 1) / (cap * PW);
        g = (groups + k * PW - 1) / (k * PW);
    }
    return (int)(g < 1 ? 1 : g);
}

template <typename AmpT>
int pos_grid_t(const QwSimDev &d)
{
    if (d.s == 8) return pos_grid_s<AmpT, 8>(d);
    if (d.s == 16) return pos_grid_s<AmpT, 16>(d);
    if (d.s == 32) return pos_grid_s<AmpT, 32>(d);
    return pos_grid_s<AmpT, 64>(d);
}

template <typename AmpT>
cudaError_t launch_pos_t(const QwSimDev &d, const void *pin, void *pout, const QwStepArgs &a, int grid,
                         cudaStream_t st)
{
    const AmpT *i = static_cast<const AmpT *>(pin);
    AmpT *o = static_cast<AmpT *>(pout);
    constexpr int PW = PosCfg<AmpT>::warps;
    if (d.s == 8) k_walk_pos<AmpT, 8, PW><<<grid, PW * 32, 0, st>>>(d, i, o, a);
    else if (d.s == 16) k_walk_pos<AmpT, 16, PW><<<grid, PW * 32, 0, st>>>(d, i, o, a);
    else if (d.s == 32) k_walk_pos<AmpT, 32, PW><<<grid, PW * 32, 0, st>>>(d, i, o, a);
    else k_walk_pos<AmpT, 64, PW><<<grid, PW * 32, 0, st>>>(d, i, o, a);
    return cudaGetLastError();
}

} // namespace

/* SM count of the current device, cached per device (launch shapes follow
   the device the simulator issues on) */
int qw_sm_count(void)
{
    constexpr int kDevs = 128;
    static int cache[kDevs] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
    int n = dev < kDevs ? cache[dev] : 0;
    if (!n) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
        if (dev < kDevs) cache[dev] = n;
    }
    return n;
}

int qw_slot_supported(const QwSimDev &d)
{
    return d.s == 8 || d.s == 16 || d.s == 32;
}

int qw_pos_supported(const QwSimDev &d)
{
    return d.s == 8 || d.s == 16 || d.s == 32 || d.s == 64;
}

size_t qw_step_smem_bytes(const QwSimDev &d, int fp32, int mode)
{
    if (mode == QW_MODE_WALK_SLOT) return fp32 ? slot_smem_bytes<float2>(d) : slot_smem_bytes<double2>(d);
    if (mode == QW_MODE_WALK_LITERAL || mode == QW_MODE_T)
        return fp32 ? step_smem<float2, QW_MODE_T>(d) : step_smem<double2, QW_MODE_T>(d);
    return fp32 ? walk_smem_bytes<float2>(d) : walk_smem_bytes<double2>(d);
}

int qw_step_grid(const QwSimDev &d, int fp32, int mode)
{
    if (mode == QW_MODE_WALK_SLOT) return fp32 ? slot_grid_t<float2>(d) : slot_grid_t<double2>(d);
    if (mode == QW_MODE_WALK_FUSED)
        return fp32 ? walk_grid_t<float2, false, false>(d) : walk_grid_t<double2, false, false>(d);
    if (mode == QW_MODE_WALK_FUSED_PF)
        return fp32 ? walk_grid_t<float2, true, false>(d) : walk_grid_t<double2, true, false>(d);
    if (mode == QW_MODE_WALK_SEG)
        return fp32 ? walk_grid_t<float2, false, true>(d) : walk_grid_t<double2, false, true>(d);
    if (mode == QW_MODE_WALK_SEG_PF)
        return fp32 ? walk_grid_t<float2, true, true>(d) : walk_grid_t<double2, true, true>(d);
    if (fp32) {
        if (mode == QW_MODE_WALK_LITERAL) return step_grid_t<float2, QW_MODE_WALK_LITERAL>(d);
        return step_grid_t<float2, QW_MODE_T>(d);
    }
    if (mode == QW_MODE_WALK_LITERAL) return step_grid_t<double2, QW_MODE_WALK_LITERAL>(d);
    return step_grid_t<double2, QW_MODE_T>(d);
}

cudaError_t qw_launch_step(const QwSimDev &d, const QwBufDev &in, const QwBufDev &out,
                           const QwBufDev &clr, const QwStepArgs &a, int fp32, int grid,
                           cudaStream_t st)
{
    if (a.mode == QW_MODE_WALK_SLOT)
        return fp32 ? launch_slot_t<float2>(d, in, out, clr, a, grid, st)
                    : launch_slot_t<double2>(d, in, out, clr, a, grid, st);
    if (a.mode == QW_MODE_WALK_FUSED)
        return fp32 ? launch_walk_t<float2, false, false>(d, in, out, clr, a, grid, st)
                    : launch_walk_t<double2, false, false>(d, in, out, clr, a, grid, st);
    if (a.mode == QW_MODE_WALK_FUSED_PF)
        return fp32 ? launch_walk_t<float2, true, false>(d, in, out, clr, a, grid, st)
                    : launch_walk_t<double2, true, false>(d, in, out, clr, a, grid, st);
    if (a.mode == QW_MODE_WALK_SEG)
        return fp32 ? launch_walk_t<float2, false, true>(d, in, out, clr, a, grid, st)
                    : launch_walk_t<double2, false, true>(d, in, out, clr, a, grid, st);
    if (a.mode == QW_MODE_WALK_SEG_PF)
        return fp32 ? launch_walk_t<float2, true, true>(d, in, out, clr, a, grid, st)
                    : launch_walk_t<double2, true, true>(d, in, out, clr, a, grid, st);
    if (fp32) {
        if (a.mode == QW_MODE_WALK_LITERAL)
            return launch_step_t<float2, QW_MODE_WALK_LITERAL>(d, in, out, clr, a, grid, st);
        return launch_step_t<float2, QW_MODE_T>(d, in, out, clr, a, grid, st);
    }
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

int qw_pos_grid(const QwSimDev &d, int fp32)
{
    return fp32 ? pos_grid_t<float2>(d) : pos_grid_t<double2>(d);
}

cudaError_t qw_launch_walk_pos(const QwSimDev &d, const void *pin, void *pout, const QwStepArgs &a, int fp32,
                               int grid, cudaStream_t st)
{
    if (!qw_pos_supported(d)) return cudaErrorInvalidValue;
    return fp32 ? launch_pos_t<float2>(d, pin, pout, a, grid, st) : launch_pos_t<double2>(d, pin, pout, a, grid, st);
}

cudaError_t qw_launch_tinit_pos(const QwSimDev &d, void *pbuf, int64_t g0, int64_t n, const double *b_re,
                                const double *b_im, const double *scale, int fp32, cudaStream_t st)
{
    const int grid = 4 * qw_sm_count();
    if (fp32) k_tinit_pos<float2><<<grid, 256, 0, st>>>(d, static_cast<float2 *>(pbuf), g0, n, b_re, b_im, scale);
    else k_tinit_pos<double2><<<grid, 256, 0, st>>>(d, static_cast<double2 *>(pbuf), g0, n, b_re, b_im, scale);
    return cudaGetLastError();
}

cudaError_t qw_launch_measure_pos(const QwSimDev &d, const void *pbuf, int64_t g0, int64_t n, int fp32,
                                  const double *scale, int reg, double *probs, int64_t len, cudaStream_t st)
{
    /* a warp per j: enough blocks that every j's loads are in flight at once */
    int64_t want = (n + 7) / 8;
    const int64_t cap = 32 * (int64_t)qw_sm_count();
    const int grid = (int)(want < 1 ? 1 : (want < cap ? want : cap));
    if (fp32)
        k_measure_pos<float2><<<grid, 256, 0, st>>>(d, static_cast<const float2 *>(pbuf), g0, n, scale, reg, probs, len);
    else
        k_measure_pos<double2><<<grid, 256, 0, st>>>(d, static_cast<const double2 *>(pbuf), g0, n, scale, reg, probs,
                                                     len);
    return cudaGetLastError();
}

cudaError_t qw_launch_pos_pack(const QwSimDev &d, const QwBufDev &buf, void *pbuf, int fp32, int32_t *status,
                               cudaStream_t st)
{
    const int grid = 4 * qw_sm_count();
    if (fp32) k_pos_pack<float2><<<grid, 256, 0, st>>>(d, buf, static_cast<float2 *>(pbuf), status);
    else k_pos_pack<double2><<<grid, 256, 0, st>>>(d, buf, static_cast<double2 *>(pbuf), status);
    return cudaGetLastError();
}

cudaError_t qw_launch_pos_unpack(const QwSimDev &d, const void *pbuf, const QwBufDev &buf, int fp32,
                                 int32_t *status, cudaStream_t st)
{
    const int grid = 4 * qw_sm_count();
    if (fp32) k_pos_unpack<float2><<<grid, 256, 0, st>>>(d, static_cast<const float2 *>(pbuf), buf, status);
    else k_pos_unpack<double2><<<grid, 256, 0, st>>>(d, static_cast<const double2 *>(pbuf), buf, status);
    return cudaGetLastError();
}

cudaError_t qw_launch_init_b(const QwSimDev &d, const QwBufDev &buf, int inst, const double *b_re,
                             const double *b_im, int n, int fp32, const double *scale, cudaStream_t st)
{
    const int grid = (n + 255) / 256;
    if (fp32) k_init_b<float2><<<grid, 256, 0, st>>>(d, buf, inst, b_re, b_im, n, scale);
    else k_init_b<double2><<<grid, 256, 0, st>>>(d, buf, inst, b_re, b_im, n, scale);
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

cudaError_t qw_launch_part_inbox(const QwSimDev &d, const QwBufDev &buf, const QwPartEntry *e, int64_t count, int fp32,
                                 int32_t *status, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    int64_t grid = (count + 255) / 256;
    if (grid > 8 * qw_sm_count()) grid = 8 * qw_sm_count();
    if (fp32) k_part_inbox<float2><<<(unsigned)grid, 256, 0, st>>>(d, buf, e, count, status);
    else k_part_inbox<double2><<<(unsigned)grid, 256, 0, st>>>(d, buf, e, count, status);
    return cudaGetLastError();
}

cudaError_t qw_launch_part_gather(const QwSimDev &d, const QwBufDev &buf, const QwPartSources &src, int fp32,
                                  int32_t *status, cudaStream_t st)
{
    if (src.n <= 0) return cudaSuccess;
    int64_t grid = (src.cap + 255) / 256;
    if (grid > 8 * qw_sm_count()) grid = 8 * qw_sm_count();
    if (grid < 1) grid = 1;
    if (fp32) k_part_gather<float2><<<(unsigned)grid, 256, 0, st>>>(d, buf, src, status);
    else k_part_gather<double2><<<(unsigned)grid, 256, 0, st>>>(d, buf, src, status);
    return cudaGetLastError();
}

cudaError_t qw_launch_part_scale(const QwPartNorms &nm, const double *target, double *scale_out, int renorm,
                                 cudaStream_t st)
{
    k_part_scale<<<1, 1, 0, st>>>(nm, target, scale_out, renorm);
    return cudaGetLastError();
}

cudaError_t qw_launch_regrow(const QwSimDev &d, const QwBufDev &from, int cap_old, uint64_t *key_new, void *amp_new,
                             int fp32, cudaStream_t st)
{
    const int grid = 4 * qw_sm_count();
    k_regrow<<<grid, 256, 0, st>>>(d.total_buckets, from.count, cap_old, d.cap_row, from.key,
                                   static_cast<const unsigned char *>(from.amp), key_new,
                                   static_cast<unsigned char *>(amp_new), fp32 ? 8 : 16);
    return cudaGetLastError();
}

cudaError_t qw_launch_qls_norm(const double2 *y, int n, double *p, int64_t *jctr, cudaStream_t st)
{
    k_qls_norm<<<1, 1024, 0, st>>>(y, n, p, jctr);
    return cudaGetLastError();
}

/* ---- measurement without device allocation ------------------------------------ */
/*
 * Histogram scratch of qw_measure_register_noalloc, a fixed array in the
 * library's device image instead of an allocated buffer.  Every GPU that
 * loads the library holds it (QW_MEASURE_NOALLOC_MAX_LEN doubles, 512 KiB)
 * until the process exits.  All calls share it: each call zeroes the bins it
 * uses before the kernel accumulates into them, and two calls whose work
 * overlaps on the GPU (different streams, no ordering between them) race on it.
 * Host code may not pass the symbol itself to a kernel -- on the host it
 * names a shadow variable, not device memory -- so the device address is
 * looked up with cudaGetSymbolAddress, once per device, with that device
 * current, and cached.
 */
static __device__ __align__(256) double g_measure_scratch[QW_MEASURE_NOALLOC_MAX_LEN];

namespace {
constexpr int kMaxDevices = 128;
std::mutex g_scratch_mu;
double *g_scratch_addr[kMaxDevices] = {nullptr};
} // namespace

cudaError_t qw_launch_measure_noalloc(const QwSimDev &d, const QwBufDev &buf, int inst, int fp32,
                                      const double *scale, int reg, double *host_probs,
                                      int64_t len, int device, cudaStream_t st, const void *pbuf, int64_t g0,
                                      int64_t pn)
{
    if (device < 0 || device >= kMaxDevices || len < 1 || len > QW_MEASURE_NOALLOC_MAX_LEN)
        return cudaErrorInvalidValue;
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_addr[device]) {
            int prev = -1;
            cudaError_t e = cudaGetDevice(&prev);
            if (e != cudaSuccess) return e;
            if (prev != device && (e = cudaSetDevice(device)) != cudaSuccess) return e;
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_measure_scratch);
            if (prev != device) cudaSetDevice(prev);
            if (e != cudaSuccess) return e;
            g_scratch_addr[device] = static_cast<double *>(p);
        }
        scratch = g_scratch_addr[device];
    }
    cudaError_t e = cudaMemsetAsync(scratch, 0, (size_t)len * sizeof(double), st);
    if (e != cudaSuccess) return e;
    const int grid = 4 * qw_sm_count();
    if (pbuf) e = qw_launch_measure_pos(d, pbuf, g0, pn, fp32, scale, reg, scratch, len, st);
    else if (fp32) k_measure<float2><<<grid, 256, 0, st>>>(d, buf, inst, scale, reg, scratch, len);
    else k_measure<double2><<<grid, 256, 0, st>>>(d, buf, inst, scale, reg, scratch, len);
    if (!pbuf) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(host_probs, scratch, (size_t)len * sizeof(double), cudaMemcpyDeviceToHost, st);
}

cudaError_t qw_launch_tinit(const QwSimDev &d, const QwBufDev &buf, int64_t lo, int64_t hi, int fp32,
                            int32_t *status, cudaStream_t st)
{
    int64_t rows = hi - lo;
    int grid = (int)((rows + WARPS - 1) / WARPS);
    if (grid > 8 * qw_sm_count()) grid = 8 * qw_sm_count();
    if (grid < 1) grid = 1;
    const bool k32 = key32_fits(d);
    if (fp32) {
        if (k32) launch_tinit_k<float2, uint32_t>(d, buf, lo, hi, grid, status, st);
        else launch_tinit_k<float2, uint64_t>(d, buf, lo, hi, grid, status, st);
    } else {
        if (k32) launch_tinit_k<double2, uint32_t>(d, buf, lo, hi, grid, status, st);
        else launch_tinit_k<double2, uint64_t>(d, buf, lo, hi, grid, status, st);
    }
    return cudaGetLastError();
}

cudaError_t qw_launch_import(const QwSimDev &d, const QwBufDev &buf, const uint64_t *rowkey,
                             const uint64_t *local, const double2 *amp, int64_t count, int fp32,
                             int32_t *status, cudaStream_t st)
{
    const int64_t grid = (count + 255) / 256;
    if (grid < 1) return cudaSuccess;
    if (fp32) k_import<float2><<<(unsigned)grid, 256, 0, st>>>(d, buf, rowkey, local, amp, count, status);
    else k_import<double2><<<(unsigned)grid, 256, 0, st>>>(d, buf, rowkey, local, amp, count, status);
    return cudaGetLastError();
}
