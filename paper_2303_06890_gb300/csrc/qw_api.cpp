/*
 * qw_api.cpp -- host side of the C ABI declared in include/qwalk.h.
 *
 * Validates the CSC input, builds the padded QRAM image of Fig. 1 and the
 * rotation table, owns the device buffers, and issues the kernels of
 * qw_kernels.cu in stream order.  No arithmetic of the walk runs here except
 * the CKS coefficients of Eq. (fx), which are host-side parameters of the
 * solver.
 */
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/qwalk.h"
#include "qw_internal.h"

namespace {

struct Scalars {
    int32_t status;
    int32_t pad0;
    int64_t steps_done;
    double norm[2];
    double scale[2];
    double renorm_target;
    unsigned int done_ctr;
    unsigned int pad1;
    unsigned long long counter;
    unsigned long long stats[QW_NSTAT];
    int64_t qls_j; /* current QLS term */
    unsigned int deferred_ctr; /* slot kernel: units left to its last block */
    unsigned int work_ctr;     /* slot kernel: groups claimed */
};

/* the head of Scalars the host reads at every synchronising call */
struct StatusView {
    int32_t status, pad;
    int64_t done;
};
static_assert(offsetof(Scalars, steps_done) == offsetof(StatusView, done), "Scalars head layout");

thread_local std::string g_create_error;

int64_t next_pow2(int64_t x)
{
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

int ceil_log2(int64_t x)
{
    int b = 0;
    while (((int64_t)1 << b) < x) b++;
    return b;
}

} // namespace

/* A flat list of branches in device memory (qw_flat.cu): kw-word packed keys
 * and complex FP64 amplitudes, stream-ordered allocations on the simulator's
 * stream. */
struct FlatList {
    int kw = 2;
    void *K = nullptr;
    double2 *A = nullptr;
    int64_t M = 0;
};

/* Branch counts of a faithful sequence for qw_step_stats: [0] at the start,
 * [1] after R^dag, [2] after the first H, [3] after the second, [4] after R. */
struct FaithCounts {
    int64_t c[5] = {0, 0, 0, 0, 0};
    int nh = 0;
};

struct qw_sim {
    qw_sim_opts opts;
    cudaStream_t stream = nullptr;
    int device = 0;                  /* CUDA device current at creation */
    cudaMemPool_t fpool = nullptr;   /* flat-path scratch (flat_alloc) */
    int fp32 = 0;
    int renorm = 0;
    int mode = QW_MODE_WALK_FUSED;
    QwSimDev d{};
    std::vector<int32_t> n_of;       /* N per instance */
    std::vector<int64_t> bkt_of;     /* bucket base per instance (+1) */
    std::vector<double> init_norm2;  /* ||b||^2 of each instance at its last init */
    double host_target = 0.0;        /* staging for an async copy of the renorm target */
    QwBufDev buf[3]{};
    int cur = 0;                     /* buffer holding the state */
    int scale_slot = 0;              /* Scalars.scale slot of the state's pending scale */
    int sync_cur = 0, sync_slot = 0; /* cur / scale_slot at the last clean sync */
    int64_t sync_done = 0;           /* device steps_done at the last clean sync */
    bool has_state = false;
    bool fresh_T = false;            /* state is T~|b~> and untouched since */
    int grid_walk = 1, grid_t = 1;
    /* device allocations */
    uint32_t *img = nullptr;
    double2 *fg = nullptr;
    float4 *fg32 = nullptr;
    int32_t *inst_n = nullptr;
    int64_t *inst_img = nullptr, *inst_bkt = nullptr;
    uint16_t *unit_inst = nullptr;
    void *slot_rot = nullptr;
    double *partials = nullptr;
    int partials_cap = 0;
    int32_t *deferred = nullptr; /* slot kernel: units left to its last block */
    QwPartEntry *outbox = nullptr;      /* row-partitioned walk: outbox segments */
    unsigned long long *outbox_count = nullptr;
    QwPartEntry *inbox = nullptr;       /* staging of received entries (qw_part_walk) */
    int64_t inbox_cap = 0;
    Scalars *sc = nullptr;
    double2 *qls_y = nullptr;
    double *qls_p = nullptr; /* p_j, j = 0..j0 */
    double *qls_c = nullptr; /* coefficients a_j, j = 0..j0 */
    int64_t qls_p_cap = 0;
    double *b_dev = nullptr;     /* |b> staging: re then im, b_stride doubles each */
    int64_t b_stride = 0;
    double *meas_dev = nullptr;  /* register marginal scratch */
    int64_t meas_cap = 0;
    Scalars *h_sc = nullptr;     /* pinned host copies: Scalars reset, status read */
    StatusView *h_st = nullptr;
    int64_t device_bytes = 0;
    int64_t launches = 0;
    int64_t issued = 0;    /* walk steps issued since the last synchronising call */
    int64_t last_good = 0; /* clean steps of those, as the last check_status found */
    /* captured 6-step graphs, one per (buffer, scale slot) phase */
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
    /* captured 3-term QLS graphs (6 walk steps, 3 norms), one per phase */
    cudaGraphExec_t qexec[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
    /* an open register-faithful session: its list of branches */
    FlatList fq;
    FaithCounts fq_counts;
    bool fq_open = false;
    /* positional layout (walk_variant 7): tables, the three row arrays that
       rotate like buf, and whether the state lives there */
    uint16_t *pos_tp = nullptr;
    uint32_t *pos_xin = nullptr;
    uint16_t *pos_xcnt = nullptr;
    uint32_t *pos_rowbase = nullptr;
    uint16_t *pos_rowinst = nullptr;
    void *pbuf[3] = {nullptr, nullptr, nullptr};
    size_t pbuf_bytes = 0;
    bool pos_built = false;
    bool pos_live = false; /* the state is pbuf[cur], not buf[cur] */
    bool pos_try = true;   /* the bucket state may have positions (unknown or yes) */
    int grid_pos = 1;
    int mode_alt = QW_MODE_WALK_FUSED, grid_alt = 1; /* the bucket kernel for a state without positions */
    cudaGraphExec_t pexec[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
    cudaGraphExec_t pqexec[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
    std::string err;
};

/* the flat and register-faithful steps synchronise between their stages:
   never captured in a graph */
static bool host_staged(const qw_sim *sim)
{
    return sim->mode == QW_MODE_WALK_FLAT || sim->mode == QW_MODE_WALK_FAITHFUL;
}

static const int kGraphSteps = 6; /* a multiple of the 3-buffer and 2-slot periods */
static const int kGraphTerms = 3;  /* QLS terms per graph: 2 walk steps each */

static void drop_graphs(qw_sim *sim)
{
    for (auto *set : {&sim->gexec, &sim->qexec, &sim->pexec, &sim->pqexec})
        for (auto &row : *set)
            for (auto &g : row)
                if (g) {
                    cudaGraphExecDestroy(g);
                    g = nullptr;
                }
}

static int fail(qw_sim *sim, int code, const std::string &msg)
{
    if (sim) sim->err = msg;
    return code;
}

static int cuda_fail(qw_sim *sim, cudaError_t e, const char *what)
{
    return fail(sim, QW_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define QW_CUDA(sim, call)                                                                         \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return cuda_fail((sim), e_, #call);                                 \
    } while (0)

template <typename T> static cudaError_t dalloc(qw_sim *sim, T **p, size_t count)
{
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T) + 16);
    if (e == cudaSuccess) sim->device_bytes += (int64_t)(count * sizeof(T));
    return e;
}

extern "C" void qw_sim_opts_default(qw_sim_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = QW_FP64;
    o->fuse_reflection = 1;
    o->prune_tau = 0.0;
    o->row_capacity = 0;
    o->warp_capacity = 0;
    o->renorm = -1;
    o->stream = nullptr;
    o->walk_variant = 0;
    o->graphs = 1;
    o->overflow_fallback = 1;
    o->nparts = 1;
    o->part = 0;
    o->outbox_capacity = 0;
}

/* Validate one CSC matrix; on success return its largest column count. */
static int validate_csc(qw_sim *sim, const qw_csc &m, int idx, int32_t *maxcount)
{
    const std::string tag = "matrix " + std::to_string(idx) + ": ";
    if (m.n < 2 || m.n > 65536) return fail(sim, QW_ERR_ARG, tag + "n must be in [2, 65536]");
    if (!m.colptr || (m.nnz > 0 && (!m.rowidx || !m.val_q15)))
        return fail(sim, QW_ERR_ARG, tag + "null CSC array");
    if (m.colptr[0] != 0 || m.colptr[m.n] != m.nnz || m.nnz < 0)
        return fail(sim, QW_ERR_CSC, tag + "colptr[0] must be 0 and colptr[n] = nnz");
    int32_t mx = 0;
    for (int32_t c = 0; c < m.n; ++c) {
        const int32_t lo = m.colptr[c], hi = m.colptr[c + 1];
        if (hi < lo) return fail(sim, QW_ERR_CSC, tag + "colptr decreases");
        mx = std::max(mx, hi - lo);
        for (int32_t t = lo; t < hi; ++t) {
            const int32_t r = m.rowidx[t];
            if (r < 0 || r >= m.n) return fail(sim, QW_ERR_CSC, tag + "row index out of range");
            if (t > lo && m.rowidx[t - 1] >= r)
                return fail(sim, QW_ERR_CSC, tag + "row indices unsorted or duplicate");
            if (r == c && m.val_q15[t] < 0)
                return fail(sim, QW_ERR_CSC, tag + "negative diagonal element");
        }
    }
    /* symmetry: (r, c, v) present => (c, r, v) present */
    for (int32_t c = 0; c < m.n; ++c) {
        for (int32_t t = m.colptr[c]; t < m.colptr[c + 1]; ++t) {
            const int32_t r = m.rowidx[t];
            const int32_t *b = m.rowidx + m.colptr[r], *e = m.rowidx + m.colptr[r + 1];
            const int32_t *p = std::lower_bound(b, e, c);
            if (p == e || *p != c || m.val_q15[p - m.rowidx] != m.val_q15[t])
                return fail(sim, QW_ERR_CSC, tag + "matrix is not symmetric");
        }
    }
    *maxcount = mx;
    return QW_OK;
}

/* Padded QRAM image of one matrix (Fig. 1): row j's s slots sorted by
 * column; missing slots hold explicit zeros at the first free columns
 * j+1, j+2, ... (cyclic). Word = column << 16 | Q1.15 value bits. */
static void build_image(const qw_csc &m, int s, uint32_t *out)
{
    std::vector<char> used((size_t)m.n, 0);
    std::vector<std::pair<int32_t, uint16_t>> slot;
    slot.reserve((size_t)s);
    for (int32_t j = 0; j < m.n; ++j) {
        slot.clear();
        for (int32_t t = m.colptr[j]; t < m.colptr[j + 1]; ++t) {
            slot.emplace_back(m.rowidx[t], (uint16_t)m.val_q15[t]);
            used[(size_t)m.rowidx[t]] = 1;
        }
        int32_t c = j;
        while ((int)slot.size() < s) {
            c = (c + 1) % m.n;
            if (used[(size_t)c]) continue;
            used[(size_t)c] = 1;
            slot.emplace_back(c, (uint16_t)0);
        }
        std::sort(slot.begin(), slot.end());
        for (int t = 0; t < s; ++t) {
            out[(size_t)j * s + t] = ((uint32_t)slot[(size_t)t].first << 16) | slot[(size_t)t].second;
            used[(size_t)slot[(size_t)t].first] = 0;
        }
    }
}

static int pos_build(qw_sim *sim);

/* (sqrt|a|, sqrt(1 - |a|)) as float pairs (hi, lo) for the Q1.15 code q:
 * hi the correctly rounded FP32 square root, lo the Newton correction
 * (x - hi^2) / (2 hi) with the residual exact by FMA, rounded once -- hi + lo
 * within ~2^-47 relative of the root.  k_walk_pos computes the same bits on
 * the device from the QRAM value word (IEEE square root, FMA and division are
 * correctly rounded on both sides). */
static float4 rot_pair_f32(int16_t q)
{
    const float x = (float)(q < 0 ? -(int)q : (int)q) * (1.0f / 32768.0f); /* exact */
    const float y = 1.0f - x;                                                  /* exact */
    const float fh = std::sqrt(x), gh = std::sqrt(y);
    const float fl = fh > 0.0f ? std::fma(-fh, fh, x) / (2.0f * fh) : 0.0f;
    const float gl = gh > 0.0f ? std::fma(-gh, gh, y) / (2.0f * gh) : 0.0f;
    return make_float4(fh, fl, gh, gl);
}

extern "C" int qw_sim_create(const qw_csc *mats, int32_t ninst, const qw_sim_opts *opts_in,
                             qw_sim **out)
{
    if (!out) return QW_ERR_ARG;
    *out = nullptr;
    if (!mats || ninst < 1 || ninst > 65535) {
        g_create_error = "qw_sim_create: mats is NULL or num_instances out of [1, 65535]";
        return QW_ERR_ARG;
    }
    qw_sim *sim = new (std::nothrow) qw_sim();
    if (!sim) return QW_ERR_CUDA;
    if (opts_in) sim->opts = *opts_in;
    else qw_sim_opts_default(&sim->opts);
    const qw_sim_opts &o = sim->opts;
    int rc = QW_OK;
    int32_t s = -1;
    int32_t nmax = 0;
    for (int i = 0; i < ninst && rc == QW_OK; ++i) {
        int32_t mx = 0;
        rc = validate_csc(sim, mats[i], i, &mx);
        if (rc != QW_OK) break;
        int32_t si = mats[i].s_pad ? mats[i].s_pad : (int32_t)next_pow2(std::max(mx, 1));
        if ((si & (si - 1)) || si < mx || si > mats[i].n) {
            rc = fail(sim, QW_ERR_CSC, "matrix " + std::to_string(i) +
                                           ": s_pad must be a power of two in [max column count, n]");
            break;
        }
        if (s >= 0 && si != s) {
            rc = fail(sim, QW_ERR_CSC, "all instances must have the same padded sparsity s");
            break;
        }
        s = si;
        nmax = std::max(nmax, mats[i].n);
    }
    if (rc != QW_OK) {
        g_create_error = "qw_sim_create: " + sim->err;
        delete sim;
        return rc;
    }
    if (o.precision != QW_FP64 && o.precision != QW_FP32_AMP) {
        delete sim;
        g_create_error = "qw_sim_create: unknown precision";
        return QW_ERR_ARG;
    }
    cudaGetDevice(&sim->device);
    sim->fp32 = o.precision == QW_FP32_AMP;
    sim->renorm = o.renorm < 0 ? sim->fp32 : (o.renorm != 0);
    static const int kVariantMode[QW_WALK_VARIANTS] = {QW_MODE_WALK_FUSED, QW_MODE_WALK_FUSED_PF, QW_MODE_WALK_SEG,
                                                       QW_MODE_WALK_SEG_PF, QW_MODE_WALK_SLOT, QW_MODE_WALK_FLAT,
                                                       QW_MODE_WALK_FAITHFUL, QW_MODE_WALK_POS};
    if (o.walk_variant < 0 || o.walk_variant >= QW_WALK_VARIANTS) {
        delete sim;
        g_create_error = "qw_sim_create: walk_variant must be 0..7";
        return QW_ERR_ARG;
    }
    sim->mode = (o.fuse_reflection || kVariantMode[o.walk_variant] == QW_MODE_WALK_FAITHFUL)
                    ? kVariantMode[o.walk_variant]
                    : QW_MODE_WALK_LITERAL;
    sim->stream = (cudaStream_t)o.stream;

    QwSimDev &d = sim->d;
    d.nb = std::max(1, ceil_log2(nmax));
    d.s = s;
    d.L = ceil_log2(s);
    d.ninst = ninst;
    const double tau = o.prune_tau > 0 ? o.prune_tau : (sim->fp32 ? std::ldexp(1.0, -24) : 1e-13);
    d.tau2 = tau * tau;
    {
        const double hi = tau * (1.0 + std::ldexp(1.0, -30));
        const double lo = tau * std::sqrt(0.5) * (1.0 - std::ldexp(1.0, -30));
        std::memcpy(&d.tau_hi_bits, &hi, 8);
        std::memcpy(&d.tau_lo_bits, &lo, 8);
        d.tau2f = (float)(tau * tau);
    }
    d.rot_calc = o.rot_bits == 0;
    d.inv_sqrt_s = 1.0 / std::sqrt((double)s);
    d.two_over_s = 2.0 / (double)s;
    d.cap_row = o.row_capacity > 0 ? o.row_capacity : std::max(8, 4 * s);
    int64_t wc = o.warp_capacity;
    if (wc <= 0) {
        wc = sim->mode != QW_MODE_WALK_LITERAL ? next_pow2(std::max<int64_t>(64, 2 * (int64_t)d.cap_row))
                                             : std::min<int64_t>(512, next_pow2(std::max<int64_t>(32, 4 * s * s)));
    }
    wc = std::max<int64_t>(wc, s);
    wc = std::max<int64_t>(wc, d.cap_row);
    d.warp_cap = (int)wc;
    if (sim->mode == QW_MODE_WALK_SLOT && !qw_slot_supported(d)) {
        g_create_error = "qw_sim_create: walk_variant 4 (one lane per QRAM slot) needs s = 8, 16 or 32";
        qw_sim_destroy(sim);
        return QW_ERR_ARG;
    }
    if (sim->mode == QW_MODE_WALK_POS && !qw_pos_supported(d)) {
        g_create_error = "qw_sim_create: walk_variant 7 (positional layout) needs s = 8, 16, 32 or 64";
        qw_sim_destroy(sim);
        return QW_ERR_ARG;
    }
    if (o.rot_bits < 0 || o.rot_bits > 52) {
        g_create_error = "qw_sim_create: rot_bits must be in [0, 52]";
        qw_sim_destroy(sim);
        return QW_ERR_ARG;
    }
    if (o.nparts < 1 || o.nparts > 64 || o.part < 0 || o.part >= o.nparts || o.outbox_capacity < 0) {
        g_create_error = "qw_sim_create: nparts must be in [1, 64] and part in [0, nparts)";
        qw_sim_destroy(sim);
        return QW_ERR_ARG;
    }
    if (o.nparts > 1 && (ninst != 1 || sim->mode == QW_MODE_WALK_LITERAL || host_staged(sim) ||
                         sim->mode == QW_MODE_WALK_POS)) {
        g_create_error = "qw_sim_create: a partitioned walk needs one instance, fuse_reflection = 1 and "
                         "walk_variant <= 4";
        qw_sim_destroy(sim);
        return QW_ERR_ARG;
    }
    if (o.spill_rows < 0 || (o.spill_rows & (o.spill_rows - 1)) != 0 || o.spill_rows > (1 << 24)) {
        g_create_error = "qw_sim_create: spill_rows must be 0 or a power of two <= 2^24";
        qw_sim_destroy(sim);
        return QW_ERR_ARG;
    }

    /* per-instance tables and the QRAM image */
    std::vector<int32_t> hn((size_t)ninst);
    std::vector<int64_t> himg((size_t)ninst), hbkt((size_t)ninst + 1);
    int64_t img_words = 0, buckets = 0;
    for (int i = 0; i < ninst; ++i) {
        hn[(size_t)i] = mats[i].n;
        himg[(size_t)i] = img_words;
        hbkt[(size_t)i] = buckets;
        img_words += (int64_t)mats[i].n * s;
        buckets += (int64_t)2 << ceil_log2(mats[i].n);
    }
    hbkt[(size_t)ninst] = buckets;
    d.spill_slots = o.spill_rows > 0 ? o.spill_rows
                                     : (int)std::min<int64_t>(4096, std::max<int64_t>(256, next_pow2(buckets / 8)));
    d.dense_buckets = buckets;
    d.n_single = ninst == 1 ? mats[0].n : 0;
    if (sim->mode == QW_MODE_WALK_FAITHFUL && (ninst != 1 || !qw_faithful_layout(d, nullptr, nullptr))) {
        g_create_error = "qw_sim_create: walk_variant 6 (register-faithful) needs one instance, s <= 128 and "
                         "working registers that fit 10 key words";
        qw_sim_destroy(sim);
        return QW_ERR_ARG;
    }
    d.total_buckets = buckets + d.spill_slots;
    sim->n_of = hn;
    sim->bkt_of = hbkt;
    d.nparts = o.nparts;
    d.part = o.part;
    d.part_rows = ((int64_t)mats[0].n + o.nparts - 1) / o.nparts;
    d.outbox_cap = o.nparts > 1 ? (o.outbox_capacity > 0 ? o.outbox_capacity : 2 * (int64_t)mats[0].n * s) : 0;
    std::vector<uint32_t> himage((size_t)img_words);
    for (int i = 0; i < ninst; ++i) build_image(mats[i], s, himage.data() + himg[(size_t)i]);
    std::vector<double2> hfg(65536);
    std::vector<float4> hfg32(65536);
    for (int c = 0; c < 65536; ++c) {
        const int16_t q = (int16_t)(uint16_t)c;
        const double mag = std::fabs((double)q / 32768.0);
        double f = std::sqrt(mag), g = std::sqrt(1.0 - mag);
        if (o.rot_bits > 0) { /* the angle in a fixed-point register of rot_bits bits */
            const double step = std::ldexp(1.5707963267948966, -o.rot_bits);
            const double th = std::nearbyint(std::acos(std::sqrt(mag)) / step) * step;
            f = std::cos(th);
            g = std::sin(th);
        }
        hfg[(size_t)c] = make_double2(f, g);
        if (o.rot_bits > 0) {
            const float fh = (float)f, gh = (float)g;
            hfg32[(size_t)c] = make_float4(fh, (float)(f - (double)fh), gh, (float)(g - (double)gh));
        } else { /* the float pairs the positional kernel derives from the code itself */
            hfg32[(size_t)c] = rot_pair_f32(q);
        }
    }

    auto bail = [&](cudaError_t e, const char *what) {
        g_create_error = std::string("qw_sim_create: ") + what + ": " + cudaGetErrorString(e);
        qw_sim_destroy(sim);
        return QW_ERR_CUDA;
    };
    cudaError_t e;
#define QW_TRY(call)                                                                               \
    if ((e = (call)) != cudaSuccess) return bail(e, #call)
    {
        /* one block holds its warps' row buffers (a few times warp_capacity
           entries each); an automatic warp_capacity halves until they fit,
           down to what a row needs (segments of two rows then stay off) */
        int optin = 0;
        QW_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, sim->device));
        while (o.warp_capacity <= 0 && qw_step_smem_bytes(d, sim->fp32, sim->mode) > (size_t)optin &&
               d.warp_cap / 2 >= std::max(d.s, d.cap_row))
            d.warp_cap /= 2;
        const size_t need = qw_step_smem_bytes(d, sim->fp32, sim->mode);
        if (sim->mode == QW_MODE_WALK_SLOT && d.warp_cap < 2 * d.cap_row) {
            g_create_error = "qw_sim_create: walk_variant 4 runs the rows it does not cover as two-row segments, "
                             "which need warp_capacity >= 2 row_capacity";
            qw_sim_destroy(sim);
            return QW_ERR_ARG;
        }
        if (need > (size_t)optin) {
            g_create_error = "qw_sim_create: the step kernel needs " + std::to_string(need) +
                             " bytes of shared memory per block, the device allows " + std::to_string(optin) +
                             ": lower warp_capacity or row_capacity";
            qw_sim_destroy(sim);
            return QW_ERR_ARG;
        }
    }
    QW_TRY(dalloc(sim, &sim->img, (size_t)img_words));
    QW_TRY(dalloc(sim, &sim->fg, 65536));
    QW_TRY(dalloc(sim, &sim->fg32, 65536));
    QW_TRY(dalloc(sim, &sim->inst_n, (size_t)ninst));
    QW_TRY(dalloc(sim, &sim->inst_img, (size_t)ninst));
    QW_TRY(dalloc(sim, &sim->inst_bkt, (size_t)ninst + 1));
    QW_TRY(cudaMemcpy(sim->img, himage.data(), himage.size() * 4, cudaMemcpyHostToDevice));
    QW_TRY(cudaMemcpy(sim->fg, hfg.data(), hfg.size() * sizeof(double2), cudaMemcpyHostToDevice));
    QW_TRY(cudaMemcpy(sim->fg32, hfg32.data(), hfg32.size() * sizeof(float4), cudaMemcpyHostToDevice));
    { /* rotation values per QRAM slot, in the step kernel's precision (16 bytes either way) */
        std::vector<float4> hs((size_t)img_words);
        for (size_t w = 0; w < himage.size(); ++w) {
            const uint32_t code = himage[w] & 0xffffu;
            if (sim->fp32) {
                hs[w] = hfg32[code];
            } else {
                static_assert(sizeof(float4) == sizeof(double2), "16-byte slot entries");
                std::memcpy(&hs[w], &hfg[code], sizeof(double2));
            }
        }
        QW_TRY(dalloc(sim, (float4 **)&sim->slot_rot, hs.size()));
        QW_TRY(cudaMemcpy(sim->slot_rot, hs.data(), hs.size() * sizeof(float4), cudaMemcpyHostToDevice));
    }
    QW_TRY(cudaMemcpy(sim->inst_n, hn.data(), hn.size() * 4, cudaMemcpyHostToDevice));
    QW_TRY(cudaMemcpy(sim->inst_img, himg.data(), himg.size() * 8, cudaMemcpyHostToDevice));
    QW_TRY(cudaMemcpy(sim->inst_bkt, hbkt.data(), hbkt.size() * 8, cudaMemcpyHostToDevice));
    if (ninst > 1) { /* instance of each dense bucket pair (2 j, 2 j + 1) */
        std::vector<uint16_t> hu((size_t)(buckets / 2));
        for (int i = 0; i < ninst; ++i)
            for (int64_t u = hbkt[(size_t)i] / 2; u < hbkt[(size_t)i + 1] / 2; ++u) hu[(size_t)u] = (uint16_t)i;
        QW_TRY(dalloc(sim, &sim->unit_inst, hu.size()));
        QW_TRY(cudaMemcpy(sim->unit_inst, hu.data(), hu.size() * 2, cudaMemcpyHostToDevice));
    }
    d.img = sim->img;
    d.fg = sim->fg;
    d.fg32 = sim->fg32;
    d.inst_n = sim->inst_n;
    d.inst_img = sim->inst_img;
    d.inst_bkt = sim->inst_bkt;
    d.unit_inst = sim->unit_inst;
    d.slot_rot = sim->slot_rot;
    const size_t amp_bytes = sim->fp32 ? sizeof(float2) : sizeof(double2);
    const size_t slots = (size_t)d.total_buckets * (size_t)d.cap_row;
    for (int bi = 0; bi < 3; ++bi) {
        QwBufDev &b = sim->buf[bi];
        QW_TRY(dalloc(sim, &b.key, slots));
        QW_TRY(dalloc(sim, (unsigned char **)&b.amp, slots * amp_bytes));
        QW_TRY(dalloc(sim, &b.count, (size_t)d.total_buckets));
        QW_TRY(dalloc(sim, &b.spill, (size_t)d.spill_slots));
        QW_TRY(cudaMemset(b.count, 0, (size_t)d.total_buckets * 4));
        QW_TRY(cudaMemset(b.spill, 0xff, (size_t)d.spill_slots * 8));
    }
    sim->grid_walk = qw_step_grid(d, sim->fp32, sim->mode);
    sim->grid_t = qw_step_grid(d, sim->fp32, QW_MODE_T);
    int gmax = std::max(sim->grid_walk, sim->grid_t);
    if (sim->mode != QW_MODE_WALK_LITERAL) {
        for (int m : {QW_MODE_WALK_FUSED, QW_MODE_WALK_FUSED_PF, QW_MODE_WALK_SEG, QW_MODE_WALK_SEG_PF})
            gmax = std::max(gmax, qw_step_grid(d, sim->fp32, m));
        if (qw_slot_supported(d)) gmax = std::max(gmax, qw_step_grid(d, sim->fp32, QW_MODE_WALK_SLOT));
        if (qw_pos_supported(d) && ninst == 1) gmax = std::max(gmax, qw_pos_grid(d, sim->fp32));
    }
    QW_TRY(dalloc(sim, &sim->partials, (size_t)gmax));
    sim->partials_cap = gmax;
    QW_TRY(dalloc(sim, &sim->deferred, (size_t)(d.dense_buckets / 2 + d.spill_slots)));
    if (d.nparts > 1) {
        QW_TRY(dalloc(sim, &sim->outbox, (size_t)d.nparts * (size_t)d.outbox_cap));
        QW_TRY(dalloc(sim, &sim->outbox_count, (size_t)d.nparts));
        QW_TRY(cudaMemset(sim->outbox_count, 0, (size_t)d.nparts * 8));
        d.outbox = sim->outbox;
        d.outbox_count = sim->outbox_count;
    }
    QW_TRY(dalloc(sim, &sim->sc, 1));
    Scalars z{};
    z.scale[0] = z.scale[1] = 1.0;
    z.renorm_target = 1.0;
    QW_TRY(cudaMemcpy(sim->sc, &z, sizeof z, cudaMemcpyHostToDevice));
    sim->init_norm2.assign((size_t)ninst, 0.0);
    QW_TRY(dalloc(sim, &sim->qls_y, (size_t)nmax));
    QW_TRY(dalloc(sim, &sim->b_dev, 2 * (size_t)nmax));
    sim->b_stride = nmax;
    QW_TRY(cudaMallocHost((void **)&sim->h_sc, sizeof(Scalars)));
    QW_TRY(cudaMallocHost((void **)&sim->h_st, sizeof(StatusView)));
    QW_TRY(cudaDeviceSynchronize());
#undef QW_TRY
    if (sim->mode == QW_MODE_WALK_POS) {
        const int prc = pos_build(sim);
        if (prc != QW_OK) {
            g_create_error = "qw_sim_create: " + sim->err;
            qw_sim_destroy(sim);
            return prc;
        }
        sim->grid_walk = sim->grid_alt;
    }
    *out = sim;
    return QW_OK;
}

extern "C" int qw_sim_destroy(qw_sim *sim)
{
    if (!sim) return QW_OK;
    if (sim->fq_open) {
        cudaFreeAsync(sim->fq.K, sim->stream);
        cudaFreeAsync(sim->fq.A, sim->stream);
    }
    if (sim->stream) cudaStreamSynchronize(sim->stream);
    else cudaDeviceSynchronize();
    if (sim->fpool) cudaMemPoolDestroy(sim->fpool);
    cudaFree(sim->pos_tp);
    cudaFree(sim->pos_xin);
    cudaFree(sim->pos_xcnt);
    cudaFree(sim->pos_rowbase);
    cudaFree(sim->pos_rowinst);
    for (void *p : sim->pbuf) cudaFree(p);
    cudaFree(sim->img);
    cudaFree(sim->fg);
    cudaFree(sim->fg32);
    cudaFree(sim->inst_n);
    cudaFree(sim->inst_img);
    cudaFree(sim->inst_bkt);
    cudaFree(sim->unit_inst);
    cudaFree(sim->slot_rot);
    for (auto &b : sim->buf) {
        cudaFree(b.key);
        cudaFree(b.amp);
        cudaFree(b.count);
        cudaFree(b.spill);
    }
    drop_graphs(sim);
    if (sim->cap_stream) cudaStreamDestroy(sim->cap_stream);
    cudaFree(sim->partials);
    cudaFree(sim->deferred);
    cudaFree(sim->outbox);
    cudaFree(sim->outbox_count);
    cudaFree(sim->inbox);
    cudaFree(sim->sc);
    cudaFree(sim->qls_y);
    cudaFree(sim->qls_p);
    cudaFree(sim->qls_c);
    cudaFree(sim->b_dev);
    cudaFree(sim->meas_dev);
    cudaFreeHost(sim->h_sc);
    cudaFreeHost(sim->h_st);
    delete sim;
    return QW_OK;
}

extern "C" const char *qw_last_error(const qw_sim *sim)
{
    if (!sim) return g_create_error.c_str();
    return sim->err.c_str();
}

extern "C" int qw_sim_info(const qw_sim *sim, int32_t *nb, int32_t *s, int32_t *ninst,
                           int64_t *bytes)
{
    if (!sim) return QW_ERR_ARG;
    if (nb) *nb = sim->d.nb;
    if (s) *s = sim->d.s;
    if (ninst) *ninst = sim->d.ninst;
    if (bytes) *bytes = sim->device_bytes;
    return QW_OK;
}

extern "C" int64_t qw_launch_count(const qw_sim *sim) { return sim ? sim->launches : 0; }

static const double *pending_scale(qw_sim *sim)
{
    return sim->renorm ? &sim->sc->scale[sim->scale_slot] : nullptr;
}

/* Synchronise, read the device status word and the clean-step counter.  On
 * an error, steps issued after the failing one did nothing on the device, so
 * the state is the output of the last clean step: move the host view there.
 * Then clear the status and map it to an error code. */
static int check_status(qw_sim *sim, const char *where)
{
    cudaError_t e = cudaMemcpyAsync(sim->h_st, &sim->sc->status, sizeof(StatusView), cudaMemcpyDeviceToHost,
                                    sim->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sim->stream);
    if (e != cudaSuccess) return cuda_fail(sim, e, where);
    const StatusView h = *sim->h_st;
    const int64_t good = h.done - sim->sync_done;
    sim->last_good = good;
    sim->issued = 0;
    if (h.status != 0) {
        sim->cur = (int)((sim->sync_cur + good) % 3);
        sim->scale_slot = sim->sync_slot ^ (int)(good & 1);
    }
    sim->sync_cur = sim->cur;
    sim->sync_slot = sim->scale_slot;
    sim->sync_done = h.done;
    if (h.status == 0) return QW_OK;
    const int32_t zero = 0;
    cudaMemcpyAsync(&sim->sc->status, &zero, 4, cudaMemcpyHostToDevice, sim->stream);
    cudaStreamSynchronize(sim->stream);
    const int32_t st = h.status;
    std::string m = std::string(where) + ": device status";
    if (st & QW_ST_ROW_OVERFLOW) m += " [row bucket overflow: raise row_capacity]";
    if (st & QW_ST_WARP_OVERFLOW) m += " [on-chip row buffer overflow: raise warp_capacity]";
    if (st & QW_ST_SPILL_FULL) m += " [garbage-row table full]";
    if (st & QW_ST_ANCILLA) m += " [register A not returned to zero]";
    if (st & QW_ST_NOT_BTILDE) m += " [a row was not |b~> before T~]";
    if (st & QW_ST_OUTBOX_FULL) m += " [an outbox toward another partition is full: raise outbox_capacity]";
    if (st & QW_ST_SORT_WAIT) m += " [the flat path's radix sort gave up waiting for a tile's count]";
    m += "; state kept after " + std::to_string(good) + " clean steps since the last sync";
    const int code = (st & (QW_ST_ROW_OVERFLOW | QW_ST_WARP_OVERFLOW | QW_ST_SPILL_FULL | QW_ST_OUTBOX_FULL))
                         ? QW_ERR_CAPACITY
                         : QW_ERR_DEVICE_STATUS;
    return fail(sim, code, m);
}

static QwStepArgs step_args(qw_sim *sim, int mode)
{
    QwStepArgs a{};
    a.mode = mode;
    a.renorm = sim->renorm;
    a.scale_in = pending_scale(sim);
    a.partials = sim->partials;
    a.done_ctr = &sim->sc->done_ctr;
    a.norm_out = &sim->sc->norm[sim->scale_slot ^ 1];
    a.scale_out = &sim->sc->scale[sim->scale_slot ^ 1];
    a.renorm_target = &sim->sc->renorm_target;
    a.steps_done = &sim->sc->steps_done;
    a.status = &sim->sc->status;
    a.stats = sim->sc->stats;
    a.qls_y = sim->qls_y;
    a.qls_coefs = sim->qls_c;
    a.qls_j = &sim->sc->qls_j;
    a.deferred = sim->deferred;
    a.deferred_ctr = &sim->sc->deferred_ctr;
    a.work_ctr = &sim->sc->work_ctr;
    return a;
}

static int flat_walk_step(qw_sim *sim, int readout);
static int faithful_walk_step(qw_sim *sim, int readout);
static int pos_unpack(qw_sim *sim);
static int sync_walk(qw_sim *sim, const char *where);

/* one walk step: X_cur -> X_cur+1, clearing X_cur+2 */
static int launch_walk(qw_sim *sim, int readout)
{
    if (sim->mode == QW_MODE_WALK_FLAT) return flat_walk_step(sim, readout);
    if (sim->mode == QW_MODE_WALK_FAITHFUL) return faithful_walk_step(sim, readout);
    if (sim->d.nparts > 1) /* the outboxes hold this step's sends only */
        QW_CUDA(sim, cudaMemsetAsync(sim->outbox_count, 0, (size_t)sim->d.nparts * 8, sim->stream));
    sim->issued++;
    const int nxt = (sim->cur + 1) % 3, clr = (sim->cur + 2) % 3;
    cudaError_t e;
    if (sim->mode == QW_MODE_WALK_POS && sim->pos_live) {
        QwStepArgs a = step_args(sim, QW_MODE_WALK_POS);
        a.qls_readout = readout;
        e = qw_launch_walk_pos(sim->d, sim->pbuf[sim->cur], sim->pbuf[nxt], a, sim->fp32, sim->grid_pos,
                               sim->stream);
    } else { /* a positional walk whose state has no positions runs the bucket kernel */
        const int mode = sim->mode == QW_MODE_WALK_POS ? sim->mode_alt : sim->mode;
        QwStepArgs a = step_args(sim, mode);
        a.qls_readout = readout;
        e = qw_launch_step(sim->d, sim->buf[sim->cur], sim->buf[nxt], sim->buf[clr], a, sim->fp32,
                           sim->mode == QW_MODE_WALK_POS ? sim->grid_alt : sim->grid_walk, sim->stream);
    }
    sim->launches++;
    if (e != cudaSuccess) return cuda_fail(sim, e, "walk step launch");
    sim->cur = nxt;
    sim->scale_slot ^= 1;
    return QW_OK;
}

/* Give the row buckets of all three buffers room for `need` branches per
 * row (row_capacity doubles until it fits), keeping their contents.  Refused
 * (QW_ERR_CAPACITY) when the buffers would take more than half of the device
 * memory free now plus what they hold. */
static int grow_rows(qw_sim *sim, int64_t need)
{
    int64_t cap = sim->d.cap_row;
    while (cap < need) cap *= 2;
    if (cap == sim->d.cap_row) return QW_OK;
    const size_t amp_bytes = sim->fp32 ? sizeof(float2) : sizeof(double2);
    const size_t per = 8 + amp_bytes;
    const size_t oldb = 3 * (size_t)sim->d.total_buckets * (size_t)sim->d.cap_row * per;
    const size_t newb = 3 * (size_t)sim->d.total_buckets * (size_t)cap * per;
    QW_CUDA(sim, cudaStreamSynchronize(sim->stream));
    size_t freeb = 0, totb = 0;
    QW_CUDA(sim, cudaMemGetInfo(&freeb, &totb));
    if (newb > (freeb + oldb) / 2)
        return fail(sim, QW_ERR_CAPACITY,
                    "row buckets of " + std::to_string(cap) + " branches per row would need " + std::to_string(newb) +
                        " bytes; device memory is short");
    drop_graphs(sim);
    const int cap_old = sim->d.cap_row;
    const size_t slots = (size_t)sim->d.total_buckets * (size_t)cap;
    sim->d.cap_row = (int)cap;
    for (auto &b : sim->buf) {
        uint64_t *key = nullptr;
        unsigned char *amp = nullptr;
        QW_CUDA(sim, dalloc(sim, &key, slots));
        QW_CUDA(sim, dalloc(sim, &amp, slots * amp_bytes));
        QW_CUDA(sim, qw_launch_regrow(sim->d, b, cap_old, key, amp, sim->fp32, sim->stream));
        QW_CUDA(sim, cudaStreamSynchronize(sim->stream));
        cudaFree(b.key);
        cudaFree(b.amp);
        sim->device_bytes -= (int64_t)((size_t)sim->d.total_buckets * (size_t)cap_old * per);
        b.key = key;
        b.amp = amp;
    }
    return QW_OK;
}

/* Stream-ordered scratch of the flat path and the register-faithful
 * sessions, from a pool of the simulator's own that keeps what was freed
 * (release threshold: no limit), so that a stage's allocations after a
 * synchronisation reuse memory instead of mapping it again; the pool and
 * its memory go with qw_sim_destroy. */
static cudaError_t flat_alloc(qw_sim *sim, size_t bytes, void **p)
{
    *p = nullptr;
    if (!sim->fpool) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = sim->device;
        cudaError_t e = cudaMemPoolCreate(&sim->fpool, &props);
        if (e != cudaSuccess) {
            sim->fpool = nullptr;
            return e;
        }
        uint64_t keep = UINT64_MAX;
        if ((e = cudaMemPoolSetAttribute(sim->fpool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) return e;
    }
    return cudaMallocFromPoolAsync(p, bytes < 16 ? 16 : bytes, sim->fpool, sim->stream);
}

static void flat_release(qw_sim *sim, FlatList &L)
{
    if (L.K) cudaFreeAsync(L.K, sim->stream);
    if (L.A) cudaFreeAsync(L.A, sim->stream);
    L.K = nullptr;
    L.A = nullptr;
    L.M = 0;
}

/* Gather the current state (with its pending renormalisation) into L. */
static cudaError_t flat_gather(qw_sim *sim, FlatList &L, int kw)
{
    cudaStream_t st = sim->stream;
    unsigned long long hc = 0;
    cudaError_t e;
    if ((e = cudaMemsetAsync(&sim->sc->counter, 0, 8, st)) != cudaSuccess) return e;
    if ((e = qw_launch_count(sim->d, sim->buf[sim->cur], -1, &sim->sc->counter, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(&hc, &sim->sc->counter, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    flat_release(sim, L);
    L.kw = kw;
    L.M = (int64_t)hc;
    if ((e = flat_alloc(sim, (size_t)L.M * 8 * kw, &L.K)) != cudaSuccess) return e;
    if ((e = flat_alloc(sim, (size_t)L.M * 16, (void **)&L.A)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(&sim->sc->counter, 0, 8, st)) != cudaSuccess) return e;
    return qw_flat_gather(sim->d, sim->buf[sim->cur], sim->fp32, pending_scale(sim), L.K, L.A, &sim->sc->counter, L.M,
                          st, kw);
}

/* An interference op on the list (0 = R^dag, 1 = R, 2 = H): grouping by a
 * global radix sort, the per-group transform, the compaction of the kept
 * outputs; the host synchronises to size the result. */
static cudaError_t flat_stage(qw_sim *sim, FlatList &L, int op)
{
    const QwSimDev &d = sim->d;
    cudaStream_t st = sim->stream;
    cudaError_t e = cudaSuccess;
    const size_t kb = 8 * (size_t)L.kw;
    void *tk = nullptr, *ta = nullptr, *work = nullptr;
    if (L.M > 1) {
        if ((e = flat_alloc(sim, (size_t)L.M * kb, &tk)) != cudaSuccess) return e;
        if ((e = flat_alloc(sim, (size_t)L.M * 16, &ta)) != cudaSuccess) return e;
        if ((e = flat_alloc(sim, qw_flat_sort_bytes(L.M), &work)) != cudaSuccess) return e;
        int in_tmp = 0;
        e = qw_flat_sort(d, L.K, L.A, tk, static_cast<double2 *>(ta), L.M, op == 2 ? 1 : 0, work,
                         &sim->sc->status, st, L.kw, &in_tmp);
        if (e == cudaSuccess && in_tmp) {
            /* the sorted list is the one in the scratch arrays: swap them */
            std::swap(L.K, tk);
            double2 *sorted = static_cast<double2 *>(ta);
            ta = L.A;
            L.A = sorted;
        }
        cudaFreeAsync(tk, st);
        cudaFreeAsync(ta, st);
        cudaFreeAsync(work, st);
        if (e != cudaSuccess) return e;
    }
    /* H: the groups of the sorted list counted first (head flags and their
       scan; the host reads the count) */
    int64_t G = 0;
    int64_t *starts = nullptr;
    if (op == 2 && L.M > 0) {
        void *heads = nullptr, *gidx = nullptr, *hsums = nullptr;
        uint32_t g32 = 0;
        if ((e = flat_alloc(sim, (size_t)L.M * 4, &heads)) != cudaSuccess) return e;
        if ((e = flat_alloc(sim, (size_t)L.M * 4, &gidx)) != cudaSuccess) return e;
        if ((e = flat_alloc(sim, qw_flat_scan_words(L.M) * 4, &hsums)) != cudaSuccess) return e;
        e = qw_flat_heads(d, L.K, L.M, static_cast<uint32_t *>(heads), st, L.kw);
        if (e == cudaSuccess)
            e = qw_flat_scan(static_cast<uint32_t *>(heads), L.M, static_cast<uint32_t *>(hsums),
                             static_cast<uint32_t *>(gidx), st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&g32, static_cast<uint32_t *>(hsums) + (L.M + 1023) / 1024, 4, cudaMemcpyDeviceToHost,
                                st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        G = (int64_t)g32;
        if (e == cudaSuccess) e = flat_alloc(sim, (size_t)(G + 1) * 8, (void **)&starts);
        if (e == cudaSuccess)
            e = qw_flat_starts(static_cast<uint32_t *>(heads), static_cast<uint32_t *>(gidx), L.M, G, starts, st);
        for (void *p : {heads, gidx, hsums})
            if (p) cudaFreeAsync(p, st);
        if (e != cudaSuccess) return e;
    }
    FlatList R;
    R.kw = L.kw;
    uint32_t total = 0;
    if (op == 2) {
        /* H: the kept outputs of each group counted, scanned, then written */
        void *cnt = nullptr, *gpos = nullptr, *sums = nullptr;
        if (G > 0) {
            if (e == cudaSuccess) e = flat_alloc(sim, (size_t)G * 4, &cnt);
            if (e == cudaSuccess) e = flat_alloc(sim, (size_t)G * 4, &gpos);
            if (e == cudaSuccess) e = flat_alloc(sim, qw_flat_scan_words(G) * 4, &sums);
            if (e == cudaSuccess)
                e = qw_flat_hgroups(d, L.K, L.A, starts, G, static_cast<uint32_t *>(cnt), nullptr, nullptr, nullptr, st,
                                    L.kw);
            if (e == cudaSuccess)
                e = qw_flat_scan(static_cast<uint32_t *>(cnt), G, static_cast<uint32_t *>(sums),
                                 static_cast<uint32_t *>(gpos), st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(&total, static_cast<uint32_t *>(sums) + (G + 1023) / 1024, 4,
                                    cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        }
        R.M = (int64_t)total;
        if (e == cudaSuccess) e = flat_alloc(sim, (size_t)R.M * kb, &R.K);
        if (e == cudaSuccess) e = flat_alloc(sim, (size_t)R.M * 16, (void **)&R.A);
        if (e == cudaSuccess && total > 0)
            e = qw_flat_hgroups(d, L.K, L.A, starts, G, static_cast<uint32_t *>(cnt), static_cast<uint32_t *>(gpos),
                                R.K, R.A, st, L.kw);
        for (void *p : {cnt, gpos, sums, (void *)starts})
            if (p) cudaFreeAsync(p, st);
        flat_release(sim, L);
        L = R;
        return e;
    }
    const int64_t n = L.M * 2;
    void *ok = nullptr, *oa = nullptr, *flags = nullptr, *pos = nullptr, *sums = nullptr;
    if ((e = flat_alloc(sim, (size_t)n * kb, &ok)) != cudaSuccess) return e;
    if ((e = flat_alloc(sim, (size_t)n * 16, &oa)) != cudaSuccess) return e;
    if ((e = flat_alloc(sim, (size_t)n * 4, &flags)) != cudaSuccess) return e;
    if ((e = flat_alloc(sim, (size_t)n * 4, &pos)) != cudaSuccess) return e;
    if ((e = flat_alloc(sim, qw_flat_scan_words(n) * 4, &sums)) != cudaSuccess) return e;
    e = qw_flat_group(d, op, L.K, L.A, L.M, ok, static_cast<double2 *>(oa), static_cast<uint32_t *>(flags), st,
                      L.kw);
    if (e == cudaSuccess && n > 0) {
        e = qw_flat_scan(static_cast<uint32_t *>(flags), n, static_cast<uint32_t *>(sums), static_cast<uint32_t *>(pos),
                         st);
        const int64_t nb = (n + 1023) / 1024;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&total, static_cast<uint32_t *>(sums) + nb, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    R.M = (int64_t)total;
    if (e == cudaSuccess) e = flat_alloc(sim, (size_t)R.M * kb, &R.K);
    if (e == cudaSuccess) e = flat_alloc(sim, (size_t)R.M * 16, (void **)&R.A);
    if (e == cudaSuccess)
        e = qw_flat_compact(ok, static_cast<double2 *>(oa), static_cast<uint32_t *>(flags),
                            static_cast<uint32_t *>(pos), n, R.K, R.A, st, L.kw);
    for (void *p : {ok, oa, flags, pos, sums})
        if (p) cudaFreeAsync(p, st);
    flat_release(sim, L);
    L = R;
    return e;
}

/* Store the list as the output of a step: X_cur+1 (and X_cur+2 cleared, as a
 * step kernel does), the row buckets grown when a row of it does not fit,
 * then the step's norm, renormalisation and counters; counts are the branch
 * numbers after each interference op for qw_step_stats. */
static int flat_store(qw_sim *sim, FlatList &L, const QwStepArgs &a, const int64_t *counts)
{
    QwSimDev &d = sim->d;
    cudaStream_t st = sim->stream;
    void *norm = nullptr, *maxrow = nullptr;
    QW_CUDA(sim, flat_alloc(sim, 8, &norm));
    QW_CUDA(sim, flat_alloc(sim, 4, &maxrow));
    int32_t *status = &sim->sc->status;
    const int nxt = (sim->cur + 1) % 3, clr = (sim->cur + 2) % 3;
    int rc = QW_OK;
    for (int attempt = 0; attempt < 2 && rc == QW_OK; ++attempt) {
        for (int bi : {nxt, clr}) QW_CUDA(sim, qw_launch_clear(d, sim->buf[bi], 0, d.total_buckets, 1, st));
        QW_CUDA(sim, cudaMemsetAsync(norm, 0, 8, st));
        QW_CUDA(sim, cudaMemsetAsync(maxrow, 0, 4, st));
        QW_CUDA(sim, qw_flat_scatter(d, sim->buf[nxt], sim->fp32, L.K, L.A, L.M, status,
                                     static_cast<unsigned int *>(maxrow), static_cast<double *>(norm), st, L.kw));
        unsigned int hmax = 0;
        QW_CUDA(sim, cudaMemcpyAsync(sim->h_st, status, sizeof(StatusView), cudaMemcpyDeviceToHost, st));
        QW_CUDA(sim, cudaMemcpyAsync(&hmax, maxrow, 4, cudaMemcpyDeviceToHost, st));
        QW_CUDA(sim, cudaStreamSynchronize(st));
        if (sim->h_st->status != QW_ST_ROW_OVERFLOW || attempt == 1 || !sim->opts.overflow_fallback) break;
        /* a row of the result is longer than row_capacity: grow the buckets
           and store again */
        const int32_t zero = 0;
        QW_CUDA(sim, cudaMemcpyAsync(status, &zero, 4, cudaMemcpyHostToDevice, st));
        rc = grow_rows(sim, (int64_t)hmax);
    }
    if (rc == QW_OK) {
        QW_CUDA(sim, qw_flat_finish(a, static_cast<double *>(norm), counts, st));
        sim->launches += 1;
        sim->cur = nxt;
        sim->scale_slot ^= 1;
    }
    cudaFreeAsync(norm, st);
    cudaFreeAsync(maxrow, st);
    if (rc != QW_OK) return rc;
    return check_status(sim, "store of the flat list");
}

/* One walk step on the flat path (qw_flat.cu): X_cur gathered into one list
 * of 16-byte register keys and complex FP64 amplitudes, the paper's
 * schedule op by op -- O_s'^dag O_A' O_s', R^dag (sort, pairs, compaction),
 * O_s'^dag O_A', H (sort, groups, compaction), [QLS read-out], P, H,
 * O_A' O_s', R, O_s'^dag O_A' O_s', A = 0 checked, S -- and the result
 * stored into X_cur+1.  The host synchronises to size each stage; device
 * scratch is stream-ordered (flat_alloc: the simulator's pool) and returned
 * to the pool before the call returns. */
static int flat_walk_step(qw_sim *sim, int readout)
{
    {
        const int prc = pos_unpack(sim);
        if (prc != QW_OK) return prc;
    }
    const QwSimDev &d = sim->d;
    cudaStream_t st = sim->stream;
    FlatList L;
    int32_t *status = &sim->sc->status;
#define QW_FLAT(call)                                                                              \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            flat_release(sim, L);                                                                  \
            return cuda_fail(sim, e_, #call);                                                      \
        }                                                                                          \
    } while (0)
    QW_FLAT(flat_gather(sim, L, 2));
    int64_t counts[5] = {L.M, 0, 0, 0, 0};
    auto map = [&](uint32_t ops) { return qw_flat_map(d, L.K, L.M, ops, status, st, 2); };
    QwStepArgs a = step_args(sim, QW_MODE_WALK_FLAT);
    a.qls_readout = readout;
    /* T~^dag */
    QW_FLAT(map(QW_FLAT_OSDAG | QW_FLAT_OA << 4 | QW_FLAT_OS << 8));
    QW_FLAT(flat_stage(sim, L, 0));
    counts[1] = L.M;
    QW_FLAT(map(QW_FLAT_OSDAG | QW_FLAT_OA << 4));
    QW_FLAT(flat_stage(sim, L, 2));
    counts[2] = L.M;
    if (readout) QW_FLAT(qw_flat_readout(d, L.K, L.A, L.M, a, st, 2));
    /* P, then T~ */
    QW_FLAT(qw_flat_phase(d, L.K, L.A, L.M, st, 2));
    QW_FLAT(flat_stage(sim, L, 2));
    counts[3] = L.M;
    QW_FLAT(map(QW_FLAT_OA | QW_FLAT_OS << 4));
    QW_FLAT(flat_stage(sim, L, 1));
    counts[4] = L.M;
    QW_FLAT(map(QW_FLAT_OSDAG | QW_FLAT_OA << 4 | QW_FLAT_OS << 8 | QW_FLAT_A0 << 12 | QW_FLAT_S << 16));
#undef QW_FLAT
    const int rc = flat_store(sim, L, a, counts);
    flat_release(sim, L);
    return rc;
}

/* ---- positional layout (walk_variant 7, k_walk_pos) ------------------------ */

/* The tables of the positional layout from the QRAM image: for slot (j, l)
 * with column c, the position of the branch k = j in row c -- 2 l' when row
 * c holds column j in slot l', else 2 s + 2 e for the e-th such row x of c
 * (listed in pos_xin) -- and the three row arrays.  The row buckets grow to
 * hold a whole positional row (2 s + 2 E branches). */
static int pos_build(qw_sim *sim)
{
    if (sim->pos_built) return QW_OK;
    QwSimDev &d = sim->d;
    if (d.nparts != 1 || !qw_pos_supported(d))
        return fail(sim, QW_ERR_ARG, "walk_variant 7 (positional) needs s = 8, 16, 32 or 64 and no partitions");
    const int s = d.s;
    const int ninst = d.ninst;
    /* rows of all instances in order: instance i starts at row inst_img[i] / s */
    int64_t nrows = 0;
    std::vector<int64_t> row0((size_t)ninst);
    for (int i = 0; i < ninst; ++i) {
        row0[(size_t)i] = nrows;
        nrows += sim->n_of[(size_t)i];
    }
    std::vector<uint32_t> img((size_t)nrows * s);
    QW_CUDA(sim, cudaMemcpy(img.data(), sim->img, img.size() * 4, cudaMemcpyDeviceToHost));
    std::vector<uint16_t> tp((size_t)nrows * s);
    std::vector<std::vector<uint32_t>> xin((size_t)nrows);
    std::vector<uint32_t> rowbase(ninst > 1 ? (size_t)nrows : 0);
    std::vector<uint16_t> rowinst(ninst > 1 ? (size_t)nrows : 0);
    for (int i = 0; i < ninst; ++i) {
        const int64_t g0 = row0[(size_t)i], n = sim->n_of[(size_t)i];
        for (int64_t j = 0; j < n; ++j) {
            if (ninst > 1) {
                rowbase[(size_t)(g0 + j)] = (uint32_t)g0;
                rowinst[(size_t)(g0 + j)] = (uint16_t)i;
            }
            for (int l = 0; l < s; ++l) {
                const uint32_t c = img[(size_t)((g0 + j) * s + l)] >> 16;
                const uint32_t *row = img.data() + (size_t)(g0 + c) * s;
                int lo = 0, hi = s;
                while (lo < hi) {
                    const int m = (lo + hi) >> 1;
                    if ((row[m] >> 16) < (uint32_t)j) lo = m + 1;
                    else hi = m;
                }
                auto &xc = xin[(size_t)(g0 + c)];
                if (lo < s && (row[lo] >> 16) == (uint32_t)j) {
                    tp[(size_t)((g0 + j) * s + l)] = (uint16_t)(2 * lo);
                } else {
                    tp[(size_t)((g0 + j) * s + l)] = (uint16_t)(2 * s + 2 * xc.size());
                    xc.push_back((uint32_t)(g0 + j) << 8 | (uint32_t)l);
                }
            }
        }
    }
    size_t E = 0;
    for (const auto &v : xin) E = std::max(E, v.size());
    const int64_t R = 2 * s + 2 * (int64_t)E;
    if (R >= 65535 || nrows >= (1 << 24) || 2 * nrows * R >= ((int64_t)1 << 31))
        return fail(sim, QW_ERR_ARG, "positional layout: too many unpaired padded columns in a row, or rows");
    std::vector<uint32_t> hx((size_t)nrows * std::max<size_t>(E, 1), 0u);
    std::vector<uint16_t> hc((size_t)nrows);
    for (int64_t c = 0; c < nrows; ++c) {
        hc[(size_t)c] = (uint16_t)xin[(size_t)c].size();
        for (size_t e = 0; e < xin[(size_t)c].size(); ++e) hx[(size_t)c * E + e] = xin[(size_t)c][e];
    }
    if (d.cap_row < R) {
        const int rc = grow_rows(sim, R);
        if (rc != QW_OK) return rc;
    }
    QW_CUDA(sim, dalloc(sim, &sim->pos_tp, tp.size()));
    QW_CUDA(sim, dalloc(sim, &sim->pos_xin, hx.size()));
    QW_CUDA(sim, dalloc(sim, &sim->pos_xcnt, hc.size()));
    QW_CUDA(sim, cudaMemcpy(sim->pos_tp, tp.data(), tp.size() * 2, cudaMemcpyHostToDevice));
    QW_CUDA(sim, cudaMemcpy(sim->pos_xin, hx.data(), hx.size() * 4, cudaMemcpyHostToDevice));
    QW_CUDA(sim, cudaMemcpy(sim->pos_xcnt, hc.data(), hc.size() * 2, cudaMemcpyHostToDevice));
    if (ninst > 1) {
        QW_CUDA(sim, dalloc(sim, &sim->pos_rowbase, rowbase.size()));
        QW_CUDA(sim, dalloc(sim, &sim->pos_rowinst, rowinst.size()));
        QW_CUDA(sim, cudaMemcpy(sim->pos_rowbase, rowbase.data(), rowbase.size() * 4, cudaMemcpyHostToDevice));
        QW_CUDA(sim, cudaMemcpy(sim->pos_rowinst, rowinst.data(), rowinst.size() * 2, cudaMemcpyHostToDevice));
    }
    sim->pbuf_bytes = (size_t)2 * (size_t)nrows * (size_t)R * (sim->fp32 ? sizeof(float2) : sizeof(double2));
    for (auto &p : sim->pbuf) {
        unsigned char *b = nullptr;
        QW_CUDA(sim, dalloc(sim, &b, sim->pbuf_bytes));
        QW_CUDA(sim, cudaMemset(b, 0, sim->pbuf_bytes));
        p = b;
    }
    d.pos_R = (int)R;
    d.pos_E = (int)E;
    d.pos_rows = nrows;
    d.pos_tp = sim->pos_tp;
    d.pos_xin = sim->pos_xin;
    d.pos_xcnt = sim->pos_xcnt;
    d.pos_rowbase = sim->pos_rowbase;
    d.pos_rowinst = sim->pos_rowinst;
    sim->grid_pos = qw_pos_grid(d, sim->fp32);
    if (sim->grid_pos > sim->partials_cap) { /* one norm partial per block */
        drop_graphs(sim); /* they hold the old array */
        cudaFree(sim->partials);
        sim->partials = nullptr;
        sim->partials_cap = 0;
        QW_CUDA(sim, dalloc(sim, &sim->partials, (size_t)sim->grid_pos));
        sim->partials_cap = sim->grid_pos;
    }
    sim->mode_alt = d.warp_cap < 2 * d.cap_row ? QW_MODE_WALK_FUSED
                    : (qw_slot_supported(d) ? QW_MODE_WALK_SLOT : QW_MODE_WALK_SEG);
    sim->grid_alt = qw_step_grid(d, sim->fp32, sim->mode_alt);
    sim->pos_built = true;
    return QW_OK;
}

/* Move the state from the buckets into the positional layout when every
 * branch has a position (then pos_live); otherwise it stays in the buckets
 * and pos_try is cleared until the state is replaced.  Synchronises. */
static int pos_pack(qw_sim *sim)
{
    cudaStream_t st = sim->stream;
    QW_CUDA(sim, cudaMemsetAsync(sim->pbuf[sim->cur], 0, sim->pbuf_bytes, st));
    QW_CUDA(sim, qw_launch_pos_pack(sim->d, sim->buf[sim->cur], sim->pbuf[sim->cur], sim->fp32, &sim->sc->status, st));
    sim->launches++;
    QW_CUDA(sim, cudaMemcpyAsync(sim->h_st, &sim->sc->status, sizeof(StatusView), cudaMemcpyDeviceToHost, st));
    QW_CUDA(sim, cudaStreamSynchronize(st));
    if (sim->h_st->status == QW_ST_POS_UNREP) {
        const int32_t zero = 0;
        QW_CUDA(sim, cudaMemcpy(&sim->sc->status, &zero, 4, cudaMemcpyHostToDevice));
        sim->pos_try = false;
        return QW_OK;
    }
    if (sim->h_st->status != 0) return check_status(sim, "positional layout");
    sim->pos_live = true;
    return QW_OK;
}

/* The state back into the row buckets (stream-ordered, no synchronisation).
 * All three bucket buffers are cleared: a bucket step appends to the next
 * buffer, which bucket steps run before the positional ones may have left
 * holding an old state. */
static int pos_unpack(qw_sim *sim)
{
    if (!sim->pos_live) return QW_OK;
    for (const QwBufDev &b : sim->buf)
        QW_CUDA(sim, qw_launch_clear(sim->d, b, 0, sim->d.total_buckets, 1, sim->stream));
    QW_CUDA(sim, qw_launch_pos_unpack(sim->d, sim->pbuf[sim->cur], sim->buf[sim->cur], sim->fp32, &sim->sc->status,
                                      sim->stream));
    sim->launches += 4;
    sim->pos_live = false;
    return QW_OK;
}

/* First row of instance inst among all instances' rows (positional layout). */
static int64_t pos_row0(const qw_sim *sim, int inst)
{
    int64_t g0 = 0;
    for (int i = 0; i < inst; ++i) g0 += sim->n_of[(size_t)i];
    return g0;
}

/* Before a positional walk: the state into the positional layout if it
 * may fit (synchronises then). */
static int pos_prepare(qw_sim *sim)
{
    if (sim->mode != QW_MODE_WALK_POS || sim->pos_live || !sim->pos_try) return QW_OK;
    int rc = pos_build(sim);
    if (rc == QW_OK) rc = sync_walk(sim, "positional layout");
    if (rc == QW_OK) rc = pos_pack(sim);
    return rc;
}

/* ---- register-faithful sub-operations (qw_flat.cu, 10-word keys) ---------- */

/* One sub-operation (QW_FQ_*) on L.  The operators on the base registers are
 * preceded by the check that every working register is 0. */
static cudaError_t faithful_op(qw_sim *sim, FlatList &L, int op, FaithCounts &fc)
{
    const QwSimDev &d = sim->d;
    cudaStream_t st = sim->stream;
    int32_t *status = &sim->sc->status;
    if (op >= QW_FQ_ADDR_COL && op <= QW_FQ_QRAM_VAL) return qw_faithful_op(d, L.K, L.M, op, status, st);
    if (op < QW_FQ_R || op > QW_FQ_FREE_A) return cudaErrorInvalidValue;
    cudaError_t e = qw_faithful_check_idle(d, L.K, L.M, status, st);
    if (e != cudaSuccess) return e;
    switch (op) {
    case QW_FQ_R:
        e = flat_stage(sim, L, 1);
        fc.c[4] = L.M;
        return e;
    case QW_FQ_RDAG:
        e = flat_stage(sim, L, 0);
        fc.c[1] = L.M;
        return e;
    case QW_FQ_H:
        e = flat_stage(sim, L, 2);
        fc.c[fc.nh < 1 ? 2 : 3] = L.M;
        fc.nh++;
        return e;
    case QW_FQ_P: return qw_flat_phase(d, L.K, L.A, L.M, st, L.kw);
    case QW_FQ_S: return qw_flat_map(d, L.K, L.M, QW_FLAT_S, status, st, L.kw);
    case QW_FQ_FREE_A: return qw_flat_map(d, L.K, L.M, QW_FLAT_A0, status, st, L.kw);
    default: return cudaSuccess; /* QW_FQ_ALLOC_A: A is 0 wherever it is free */
    }
}

static bool faithful_fits(const qw_sim *sim)
{
    return sim->d.ninst == 1 && qw_faithful_layout(sim->d, nullptr, nullptr) != 0;
}

/* One walk step in the register-faithful schedule (walk_variant 6): the
 * QW_FQ_STEP sequence on the gathered list, the QLS read-out after the first
 * H, the result stored as X_cur+1. */
static int faithful_walk_step(qw_sim *sim, int readout)
{
    {
        const int prc = pos_unpack(sim);
        if (prc != QW_OK) return prc;
    }
    static const int32_t kStep[QW_FQ_STEP_LEN] = QW_FQ_STEP;
    FlatList L;
    FaithCounts fc;
    QwStepArgs a = step_args(sim, QW_MODE_WALK_FAITHFUL);
    a.qls_readout = readout;
    cudaError_t e = flat_gather(sim, L, QW_FQ_KEY_WORDS);
    fc.c[0] = L.M;
    for (int i = 0; i < QW_FQ_STEP_LEN && e == cudaSuccess; ++i) {
        e = faithful_op(sim, L, kStep[i], fc);
        if (e == cudaSuccess && readout && kStep[i] == QW_FQ_H && fc.nh == 1)
            e = qw_flat_readout(sim->d, L.K, L.A, L.M, a, sim->stream, L.kw);
    }
    if (e != cudaSuccess) {
        flat_release(sim, L);
        return cuda_fail(sim, e, "register-faithful walk step");
    }
    const int rc = flat_store(sim, L, a, fc.c);
    flat_release(sim, L);
    return rc;
}

static int faithful_session_closed(qw_sim *sim)
{
    return sim->fq_open ? fail(sim, QW_ERR_STATE, "a register-faithful session is open: call qw_faithful_end")
                        : QW_OK;
}

extern "C" int qw_faithful_info(const qw_sim *sim, int32_t *addr_bits, int32_t *key_bits, int64_t *live_bits)
{
    if (!sim) return QW_ERR_ARG;
    int aw = 0, bits = 0;
    const int fits = qw_faithful_layout(sim->d, &aw, &bits);
    if (addr_bits) *addr_bits = aw;
    if (key_bits) *key_bits = bits;
    /* the base registers (jc, j, b1, kc, k, b2: 4 nb + 2), A, the address,
       left, right, mid, midval, flag, cl, ce and L + 1 frames */
    if (live_bits)
        *live_bits = 4 * (int64_t)sim->d.nb + 2 + 16 + aw + 3 * aw + 16 + 3 + (int64_t)(sim->d.L + 1) * (aw + 16 + 2);
    return fits && sim->d.ninst == 1 ? QW_OK : QW_ERR_ARG;
}

extern "C" int qw_faithful_begin(qw_sim *sim)
{
    if (!sim) return QW_ERR_ARG;
    if (!sim->has_state) return fail(sim, QW_ERR_STATE, "no state: call qw_state_init first");
    int rc = faithful_session_closed(sim);
    if (rc != QW_OK) return rc;
    if (!faithful_fits(sim))
        return fail(sim, QW_ERR_ARG, "register-faithful keys: one instance, and the working registers must fit "
                                     "10 words with s <= 128");
    rc = sync_walk(sim, "qw_faithful_begin");
    if (rc != QW_OK) return rc;
    rc = pos_unpack(sim);
    if (rc != QW_OK) return rc;
    cudaError_t e = flat_gather(sim, sim->fq, QW_FQ_KEY_WORDS);
    if (e != cudaSuccess) {
        flat_release(sim, sim->fq);
        return cuda_fail(sim, e, "qw_faithful_begin");
    }
    sim->launches++;
    sim->fq_open = true;
    sim->fq_counts = FaithCounts{};
    sim->fq_counts.c[0] = sim->fq.M;
    return QW_OK;
}

extern "C" int qw_faithful_apply(qw_sim *sim, const int32_t *ops, int32_t nops)
{
    if (!sim) return QW_ERR_ARG;
    if (!sim->fq_open) return fail(sim, QW_ERR_STATE, "no register-faithful session: call qw_faithful_begin");
    if (nops < 0 || (nops > 0 && !ops)) return fail(sim, QW_ERR_ARG, "bad sub-operation list");
    for (int32_t i = 0; i < nops; ++i)
        if (ops[i] < QW_FQ_ADDR_COL || ops[i] > QW_FQ_FREE_A)
            return fail(sim, QW_ERR_ARG, "unknown sub-operation code " + std::to_string(ops[i]));
    for (int32_t i = 0; i < nops; ++i) {
        cudaError_t e = faithful_op(sim, sim->fq, ops[i], sim->fq_counts);
        if (e != cudaSuccess) return cuda_fail(sim, e, "qw_faithful_apply");
        sim->launches++;
    }
    return check_status(sim, "qw_faithful_apply");
}

extern "C" int qw_faithful_export(qw_sim *sim, uint64_t *regs, double *amps, int64_t cap, int64_t *count)
{
    if (!sim || !count) return QW_ERR_ARG;
    if (!sim->fq_open) return fail(sim, QW_ERR_STATE, "no register-faithful session: call qw_faithful_begin");
    if (cap > 0 && (!regs || !amps)) return fail(sim, QW_ERR_ARG, "null output arrays");
    const int64_t M = sim->fq.M;
    *count = M;
    if (M == 0 || cap <= 0) return QW_OK;
    const size_t C = QW_FQ_COLS;
    uint64_t *dt = nullptr;
    QW_CUDA(sim, cudaMallocAsync((void **)&dt, (size_t)M * C * 8, sim->stream));
    QW_CUDA(sim, qw_faithful_export(sim->d, sim->fq.K, M, dt, sim->stream));
    sim->launches++;
    std::vector<uint64_t> t((size_t)M * C);
    std::vector<double2> a((size_t)M);
    QW_CUDA(sim, cudaMemcpyAsync(t.data(), dt, (size_t)M * C * 8, cudaMemcpyDeviceToHost, sim->stream));
    QW_CUDA(sim, cudaMemcpyAsync(a.data(), sim->fq.A, (size_t)M * 16, cudaMemcpyDeviceToHost, sim->stream));
    QW_CUDA(sim, cudaFreeAsync(dt, sim->stream));
    QW_CUDA(sim, cudaStreamSynchronize(sim->stream));
    std::vector<int64_t> order((size_t)M);
    for (int64_t i = 0; i < M; ++i) order[(size_t)i] = i;
    std::sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
        const uint64_t *p = t.data() + (size_t)x * C, *q = t.data() + (size_t)y * C;
        for (size_t c = 0; c < C; ++c)
            if (p[c] != q[c]) return p[c] < q[c];
        return false;
    });
    const int64_t nout = std::min(M, cap);
    for (int64_t i = 0; i < nout; ++i) {
        const int64_t src = order[(size_t)i];
        std::memcpy(regs + (size_t)i * C, t.data() + (size_t)src * C, C * 8);
        amps[2 * i] = a[(size_t)src].x;
        amps[2 * i + 1] = a[(size_t)src].y;
    }
    return QW_OK;
}

extern "C" int qw_faithful_end(qw_sim *sim, int32_t keep)
{
    if (!sim) return QW_ERR_ARG;
    if (!sim->fq_open) return fail(sim, QW_ERR_STATE, "no register-faithful session: call qw_faithful_begin");
    if (!keep) {
        flat_release(sim, sim->fq);
        sim->fq_open = false;
        return QW_OK;
    }
    FlatList &L = sim->fq;
    QW_CUDA(sim, qw_faithful_check_idle(sim->d, L.K, L.M, &sim->sc->status, sim->stream));
    QW_CUDA(sim, qw_flat_map(sim->d, L.K, L.M, QW_FLAT_A0, &sim->sc->status, sim->stream, L.kw));
    int rc = check_status(sim, "qw_faithful_end");
    if (rc != QW_OK) return rc;
    QwStepArgs a = step_args(sim, QW_MODE_WALK_FAITHFUL);
    rc = flat_store(sim, L, a, sim->fq_counts.c);
    flat_release(sim, L);
    sim->fq_open = false;
    return rc;
}

extern "C" int qw_state_init(qw_sim *sim, int32_t inst, const double *b_re, const double *b_im,
                             int32_t n, int32_t apply_T)
{
    if (!sim) return QW_ERR_ARG;
    if (sim->fq_open) return faithful_session_closed(sim);
    if (inst < 0 || inst >= sim->d.ninst) return fail(sim, QW_ERR_ARG, "instance out of range");
    if (!b_re || n != sim->n_of[(size_t)inst]) return fail(sim, QW_ERR_ARG, "b must hold N values");
    /* T~|b~> of a positional walk is written straight into the layout (one
       instance, or several already there); otherwise into the row buckets */
    const bool pos_init = apply_T && sim->mode == QW_MODE_WALK_POS && sim->pos_built &&
                          (sim->d.ninst == 1 || sim->pos_live);
    if (!pos_init) {
        if (sim->d.ninst > 1) { /* the other instances keep their state: back into the buckets */
            const int prc = pos_unpack(sim);
            if (prc != QW_OK) return prc;
        }
        sim->pos_live = false; /* the state is replaced in the row buckets */
    }
    sim->pos_try = true;
    /* |b> goes straight from the caller's arrays to the device (asynchronous
       when they are pinned); the previous call's copies ended at its sync */
    double *dre = sim->b_dev, *dim = b_im ? sim->b_dev + sim->b_stride : nullptr;
    QW_CUDA(sim, cudaMemcpyAsync(dre, b_re, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, sim->stream));
    if (b_im)
        QW_CUDA(sim, cudaMemcpyAsync(dim, b_im, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, sim->stream));
    const int64_t lo = sim->bkt_of[(size_t)inst], hi = sim->bkt_of[(size_t)inst + 1];
    const bool all = sim->d.ninst == 1;
    /* clear the instance's rows in every buffer (the whole state for a single
       instance, garbage-row table included) */
    for (int bi = 0; bi < 3 && !pos_init; ++bi) {
        QW_CUDA(sim, qw_launch_clear(sim->d, sim->buf[bi], all ? 0 : lo,
                                     all ? sim->d.total_buckets : hi, all ? 1 : 0, sim->stream));
        sim->launches++;
    }
    if (apply_T && !pos_init && sim->opts.overflow_fallback && sim->d.cap_row < 2 * sim->d.s) {
        /* T~ gives a row of |b~> up to 2 s branches */
        int rc = grow_rows(sim, 2 * (int64_t)sim->d.s);
        if (rc != QW_OK) return rc;
    }
    double nb2 = 0.0;
    for (int j = 0; j < n; ++j) nb2 += b_re[j] * b_re[j] + (b_im ? b_im[j] * b_im[j] : 0.0);
    sim->init_norm2[(size_t)inst] = nb2;
    if (all) {
        Scalars &z = *sim->h_sc;
        z = Scalars{};
        z.scale[0] = z.scale[1] = 1.0;
        z.renorm_target = nb2;
        QW_CUDA(sim, cudaMemcpyAsync(sim->sc, sim->h_sc, sizeof(Scalars), cudaMemcpyHostToDevice, sim->stream));
        sim->scale_slot = sim->sync_slot = 0;
        sim->cur = sim->sync_cur = 0;
        sim->sync_done = 0;
    } else {
        double target = 0.0;
        for (double v : sim->init_norm2) target += v;
        sim->host_target = target;
        QW_CUDA(sim, cudaMemcpyAsync(&sim->sc->renorm_target, &sim->host_target, 8,
                                     cudaMemcpyHostToDevice, sim->stream));
    }
    if (pos_init) {
        int64_t g0 = 0;
        for (int i = 0; i < inst; ++i) g0 += sim->n_of[(size_t)i];
        QW_CUDA(sim, qw_launch_tinit_pos(sim->d, sim->pbuf[sim->cur], g0, n, dre, dim,
                                         all ? nullptr : pending_scale(sim), sim->fp32, sim->stream));
        sim->launches++;
        sim->pos_live = true;
    } else {
        QW_CUDA(sim, qw_launch_init_b(sim->d, sim->buf[sim->cur], inst, dre, dim, n, sim->fp32,
                                      all ? nullptr : pending_scale(sim), sim->stream));
        sim->launches++;
    }
    if (apply_T && !pos_init) {
        /* T~ on |b~>: the one-branch-per-row kernel (a row that is not |b~>
           sets a status bit), or the literal sort-based schedule when that
           was asked for */
        if (sim->mode != QW_MODE_WALK_LITERAL) {
            QW_CUDA(sim, qw_launch_tinit(sim->d, sim->buf[sim->cur], lo, hi, sim->fp32, &sim->sc->status,
                                         sim->stream));
            sim->launches++;
        } else {
            QwStepArgs a = step_args(sim, QW_MODE_T);
            a.scale_in = nullptr;
            a.norm_out = &sim->sc->norm[sim->scale_slot];
            a.scale_out = nullptr;
            a.bucket_lo = lo;
            a.bucket_hi = hi;
            QW_CUDA(sim, qw_launch_step(sim->d, sim->buf[sim->cur], sim->buf[sim->cur], sim->buf[sim->cur],
                                        a, sim->fp32, sim->grid_t, sim->stream));
            sim->launches++;
        }
    }
    int rc = check_status(sim, "qw_state_init");
    if (rc != QW_OK) return rc;
    sim->has_state = true;
    sim->fresh_T = apply_T != 0;
    return QW_OK;
}

/* Capture kGraphSteps walk steps starting at the current (buffer, slot)
 * phase on a private stream; the sequence of kernel arguments repeats with
 * that period, so the graph can be replayed whenever the phase recurs. */
/* One QLS term: T~^dag W^2 T~ as two walk steps, the second reading out
 * Y += a_j Pi_0 tau_j, then p_j = ||Y||^2 and j += 1 on the device. */
static int launch_qls_term(qw_sim *sim)
{
    int rc = launch_walk(sim, 0);
    if (rc == QW_OK) rc = launch_walk(sim, 1);
    if (rc != QW_OK) return rc;
    QW_CUDA(sim, qw_launch_qls_norm(sim->qls_y, sim->n_of[0], sim->qls_p, &sim->sc->qls_j, sim->stream));
    sim->launches++;
    return QW_OK;
}

static int capture_graph(qw_sim *sim, cudaGraphExec_t *out, bool qls)
{
    if (!sim->cap_stream) QW_CUDA(sim, cudaStreamCreateWithFlags(&sim->cap_stream, cudaStreamNonBlocking));
    cudaStream_t user = sim->stream;
    const int cur = sim->cur, slot = sim->scale_slot;
    const int64_t launches = sim->launches, issued = sim->issued;
    sim->stream = sim->cap_stream;
    cudaError_t e = cudaStreamBeginCapture(sim->cap_stream, cudaStreamCaptureModeThreadLocal);
    int rc = QW_OK;
    if (qls) {
        for (int t = 0; t < kGraphTerms && e == cudaSuccess && rc == QW_OK; ++t) rc = launch_qls_term(sim);
    } else {
        for (int t = 0; t < kGraphSteps && e == cudaSuccess && rc == QW_OK; ++t) rc = launch_walk(sim, 0);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(sim->cap_stream, &g);
    sim->stream = user;
    sim->cur = cur;
    sim->scale_slot = slot;
    sim->launches = launches;
    sim->issued = issued;
    if (e != cudaSuccess) return cuda_fail(sim, e, "cudaStreamBeginCapture");
    if (rc != QW_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e2 != cudaSuccess) return cuda_fail(sim, e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(sim, e, "cudaGraphInstantiate");
    return QW_OK;
}

extern "C" int qw_enqueue_walk_steps(qw_sim *sim, int64_t nsteps)
{
    if (!sim) return QW_ERR_ARG;
    if (sim->fq_open) return faithful_session_closed(sim);
    if (nsteps < 0) return fail(sim, QW_ERR_ARG, "nsteps < 0");
    if (!sim->has_state) return fail(sim, QW_ERR_STATE, "no state: call qw_state_init first");
    if (nsteps > 0) sim->fresh_T = false;
    int64_t t = 0;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool capturing = cudaStreamIsCapturing(sim->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
    if (nsteps > 0 && !capturing) {
        const int rc = pos_prepare(sim);
        if (rc != QW_OK) return rc;
    }
    if (sim->opts.graphs && !host_staged(sim) && sim->d.nparts == 1 && nsteps >= kGraphSteps && !capturing) {
        cudaGraphExec_t &g = (sim->pos_live ? sim->pexec : sim->gexec)[sim->cur][sim->scale_slot];
        if (!g) {
            int rc = capture_graph(sim, &g, false);
            if (rc != QW_OK) return rc;
        }
        for (; t + kGraphSteps <= nsteps; t += kGraphSteps) {
            QW_CUDA(sim, cudaGraphLaunch(g, sim->stream));
            sim->launches += kGraphSteps; /* one step kernel launch per step inside the graph */
            sim->issued += kGraphSteps;
        }
    }
    for (; t < nsteps; ++t) {
        int rc = launch_walk(sim, 0);
        if (rc != QW_OK) return rc;
    }
    return QW_OK;
}

/* Synchronise after walk steps.  With overflow_fallback, the steps that did
 * nothing after one outgrew the buckets (the state is at the last clean
 * step) are run on the flat path, which grows the buckets as needed. */
static int sync_walk(qw_sim *sim, const char *where)
{
    const int64_t issued = sim->issued;
    int rc = check_status(sim, where);
    if (rc != QW_ERR_CAPACITY || !sim->opts.overflow_fallback) return rc;
    for (int64_t t = sim->last_good; t < issued; ++t) {
        rc = flat_walk_step(sim, 0);
        if (rc != QW_OK) return rc;
    }
    sim->err.clear();
    return QW_OK;
}

extern "C" int qw_sync(qw_sim *sim)
{
    if (!sim) return QW_ERR_ARG;
    return sync_walk(sim, "qw_sync");
}

extern "C" int qw_apply_walk_step(qw_sim *sim, int64_t nsteps)
{
    int rc = qw_enqueue_walk_steps(sim, nsteps);
    if (rc != QW_OK) return rc;
    return sync_walk(sim, "qw_apply_walk_step");
}

extern "C" int qw_autotune(qw_sim *sim, int32_t steps, int32_t *choice, double *us_per_step)
{
    if (!sim || steps < 1) return QW_ERR_ARG;
    if (sim->fq_open) return faithful_session_closed(sim);
    if (!sim->has_state) return fail(sim, QW_ERR_STATE, "no state: call qw_state_init first");
    if (sim->mode == QW_MODE_WALK_LITERAL) {
        if (choice) *choice = -1;
        return QW_OK;
    }
    /* candidates: walk_variant -> mode.  A segment holds two rows on chip:
       tried only when the warp buffer fits them; the slot kernel (which falls
       back to segments) also needs s = 8, 16 or 32; the positional layout
       s = 8 .. 64 and no partitions (its tables are built first: they may
       grow row_capacity, which the other kernels' launch shapes follow) */
    const bool slot = qw_slot_supported(sim->d);
    const bool pos = qw_pos_supported(sim->d) && sim->d.nparts == 1;
    if (pos) {
        const int rc = pos_build(sim);
        if (rc != QW_OK) return rc;
    }
    const bool seg = sim->d.warp_cap >= 2 * sim->d.cap_row;
    std::vector<std::pair<int, int>> cand = {{0, QW_MODE_WALK_FUSED}, {1, QW_MODE_WALK_FUSED_PF}};
    if (seg) {
        cand.push_back({2, QW_MODE_WALK_SEG});
        cand.push_back({3, QW_MODE_WALK_SEG_PF});
        if (slot) cand.push_back({4, QW_MODE_WALK_SLOT});
    }
    if (pos) cand.push_back({7, QW_MODE_WALK_POS});
    double us[QW_WALK_VARIANTS];
    for (double &u : us) u = 0.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    QW_CUDA(sim, cudaEventCreate(&e0));
    QW_CUDA(sim, cudaEventCreate(&e1));
    int rc = QW_OK;
    const int graphs = sim->opts.graphs;
    sim->opts.graphs = 0; /* time the kernels themselves */
    for (size_t c = 0; c < cand.size() && rc == QW_OK; ++c) {
        const int v = cand[c].first, mode = cand[c].second;
        if (mode != QW_MODE_WALK_POS) rc = pos_unpack(sim);
        if (rc != QW_OK) break;
        sim->mode = mode;
        sim->grid_walk = mode == QW_MODE_WALK_POS ? sim->grid_alt : qw_step_grid(sim->d, sim->fp32, mode);
        if (mode == QW_MODE_WALK_POS) { /* the move into the layout is not timed */
            rc = pos_prepare(sim);
            if (rc != QW_OK) break;
        }
        cudaEventRecord(e0, sim->stream);
        rc = qw_enqueue_walk_steps(sim, steps);
        cudaEventRecord(e1, sim->stream);
        if (rc == QW_OK) rc = check_status(sim, "qw_autotune");
        float ms = 0.f;
        if (rc == QW_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) us[v] = 1000.0 * ms / steps;
    }
    sim->opts.graphs = graphs;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int best = cand[0].first, best_mode = cand[0].second;
    for (const auto &cv : cand)
        if (us[cv.first] > 0.0 && (us[best] <= 0.0 || us[cv.first] < us[best])) {
            best = cv.first;
            best_mode = cv.second;
        }
    if (best_mode != QW_MODE_WALK_POS) {
        const int urc = pos_unpack(sim);
        if (rc == QW_OK) rc = urc;
    }
    sim->mode = best_mode;
    sim->grid_walk = best_mode == QW_MODE_WALK_POS ? sim->grid_alt : qw_step_grid(sim->d, sim->fp32, best_mode);
    drop_graphs(sim);
    if (choice) *choice = best;
    if (us_per_step)
        for (int v = 0; v < QW_WALK_VARIANTS; ++v) us_per_step[v] = us[v];
    return rc;
}

extern "C" int qw_cks_coefficients(double kappa, double eps, double *coeffs, int64_t cap,
                                   int64_t *j0_out, int64_t *b_out)
{
    if (!(kappa >= 1.0) || !(eps > 0.0 && eps < 1.0) || (cap > 0 && !coeffs)) return QW_ERR_ARG;
    const double bd = std::ceil(kappa * kappa * std::log(kappa / eps));
    if (!(bd < 4e9)) return QW_ERR_ARG;
    const int64_t b = (int64_t)bd;
    const int64_t j0 = (int64_t)std::ceil(std::sqrt(bd * std::log(4.0 * bd / eps)));
    if (j0_out) *j0_out = j0;
    if (b_out) *b_out = b;
    if (cap <= 0) return QW_OK;
    /* terms t_i = C(2b, b+i) / 4^b, i = 0..b.  t_0 = prod_{i<=b} (2i-1)/(2i) for
       b <= 4096, else the asymptotic series of the central binomial coefficient
       C(2b,b)/4^b = (pi b)^(-1/2) (1 - 1/(8b) + 1/(128b^2) + 5/(1024b^3)
       - 21/(32768b^4)); then t_{i+1} / t_i = (b - i) / (b + i + 1); tails are
       summed smallest term first. */
    double t0;
    if (b <= 4096) {
        t0 = 1.0;
        for (int64_t i = 1; i <= b; ++i) t0 *= (double)(2 * i - 1) / (double)(2 * i);
    } else {
        const double x = 1.0 / bd;
        const double pi = 3.14159265358979323846;
        t0 = (1.0 - x / 8.0 + x * x / 128.0 + 5.0 * x * x * x / 1024.0 - 21.0 * x * x * x * x / 32768.0) /
             std::sqrt(pi * bd);
    }
    int64_t imax = 0;
    std::vector<double> t;
    double cur = t0;
    t.push_back(cur);
    while (imax < b && cur > 0.0) {
        cur *= (double)(b - imax) / (double)(b + imax + 1);
        t.push_back(cur);
        imax++;
    }
    const int64_t count = std::min<int64_t>(j0 + 1, cap);
    std::vector<double> tail((size_t)t.size() + 1, 0.0);
    for (int64_t i = (int64_t)t.size() - 1; i >= 0; --i) tail[(size_t)i] = tail[(size_t)i + 1] + t[(size_t)i];
    for (int64_t j = 0; j < count; ++j) {
        const double tj = (j + 1 < (int64_t)tail.size()) ? tail[(size_t)j + 1] : 0.0;
        coeffs[j] = 4.0 * ((j & 1) ? -tj : tj);
    }
    return QW_OK;
}

extern "C" int qw_apply_qls(qw_sim *sim, int32_t inst, const double *coeffs, int64_t j0,
                            double *y_out, double *psucc_out)
{
    if (!sim) return QW_ERR_ARG;
    if (sim->fq_open) return faithful_session_closed(sim);
    if (sim->d.ninst != 1 || inst != 0) return fail(sim, QW_ERR_ARG, "QLS needs a single-instance simulator");
    if (sim->d.nparts > 1) return fail(sim, QW_ERR_ARG, "QLS is not run on a partitioned walk");
    if (!coeffs || j0 < 0 || !y_out) return fail(sim, QW_ERR_ARG, "coeffs, j0 and y_out are required");
    if (!sim->has_state || !sim->fresh_T)
        return fail(sim, QW_ERR_STATE, "QLS needs the state T~|b~> (qw_state_init with apply_T = 1)");
    const int n = sim->n_of[0];
    if (sim->qls_p_cap < j0 + 1) {
        drop_graphs(sim); /* the QLS graphs hold the old arrays */
        cudaFree(sim->qls_p);
        cudaFree(sim->qls_c);
        sim->qls_p = sim->qls_c = nullptr;
        sim->qls_p_cap = 0;
        QW_CUDA(sim, cudaMalloc((void **)&sim->qls_p, (size_t)(j0 + 1) * sizeof(double)));
        QW_CUDA(sim, cudaMalloc((void **)&sim->qls_c, (size_t)(j0 + 1) * sizeof(double)));
        sim->qls_p_cap = j0 + 1;
    }
    QW_CUDA(sim, cudaMemcpyAsync(sim->qls_c, coeffs, (size_t)(j0 + 1) * sizeof(double), cudaMemcpyHostToDevice,
                                 sim->stream));
    QW_CUDA(sim, cudaMemsetAsync(sim->qls_y, 0, (size_t)n * sizeof(double2), sim->stream));
    QW_CUDA(sim, cudaMemsetAsync(&sim->sc->qls_j, 0, sizeof(int64_t), sim->stream));
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool capturing = cudaStreamIsCapturing(sim->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
    if (!capturing) {
        const int rc = pos_prepare(sim);
        if (rc != QW_OK) return rc;
    }
    const bool graphs = sim->opts.graphs && !host_staged(sim) && !capturing;
    int64_t j = 0, next_check = 1024;
    while (j <= j0) {
        if (graphs && j0 + 1 - j >= kGraphTerms) {
            cudaGraphExec_t &g = (sim->pos_live ? sim->pqexec : sim->qexec)[sim->cur][sim->scale_slot];
            if (!g) {
                int rc = capture_graph(sim, &g, true);
                if (rc != QW_OK) return rc;
            }
            QW_CUDA(sim, cudaGraphLaunch(g, sim->stream));
            sim->launches += 3 * kGraphTerms;
            sim->issued += 2 * kGraphTerms;
            j += kGraphTerms;
        } else {
            int rc = launch_qls_term(sim);
            if (rc != QW_OK) return rc;
            j += 1;
        }
        if (j >= next_check) { /* stop early on a device error */
            next_check += 1024;
            int st = check_status(sim, "qw_apply_qls");
            if (st != QW_OK) return st;
        }
    }
    sim->fresh_T = false;
    std::vector<double2> hy((size_t)n);
    QW_CUDA(sim, cudaMemcpyAsync(hy.data(), sim->qls_y, (size_t)n * sizeof(double2),
                                 cudaMemcpyDeviceToHost, sim->stream));
    if (psucc_out)
        QW_CUDA(sim, cudaMemcpyAsync(psucc_out, sim->qls_p, (size_t)(j0 + 1) * sizeof(double),
                                     cudaMemcpyDeviceToHost, sim->stream));
    int rc = check_status(sim, "qw_apply_qls");
    if (rc != QW_OK) return rc;
    for (int j = 0; j < n; ++j) {
        y_out[2 * j] = hy[(size_t)j].x;
        y_out[2 * j + 1] = hy[(size_t)j].y;
    }
    return QW_OK;
}

extern "C" int qw_measure_register(qw_sim *sim, int32_t inst, int32_t reg, double *probs, int64_t len)
{
    if (!sim) return QW_ERR_ARG;
    if (inst < 0 || inst >= sim->d.ninst || reg < 0 || reg > 5 || !probs || len < 1)
        return fail(sim, QW_ERR_ARG, "bad instance, register id or output");
    if (!sim->has_state) return fail(sim, QW_ERR_STATE, "no state");
    if (sim->meas_cap < len) { /* kept for later calls */
        QW_CUDA(sim, cudaStreamSynchronize(sim->stream));
        cudaFree(sim->meas_dev);
        sim->meas_dev = nullptr;
        sim->meas_cap = 0;
        QW_CUDA(sim, cudaMalloc((void **)&sim->meas_dev, (size_t)len * sizeof(double)));
        sim->meas_cap = len;
    }
    double *dp = sim->meas_dev;
    QW_CUDA(sim, cudaMemsetAsync(dp, 0, (size_t)len * sizeof(double), sim->stream));
    if (sim->pos_live) /* read the positional layout in place */
        QW_CUDA(sim, qw_launch_measure_pos(sim->d, sim->pbuf[sim->cur], pos_row0(sim, inst), sim->n_of[(size_t)inst],
                                           sim->fp32, pending_scale(sim), reg, dp, len, sim->stream));
    else
        QW_CUDA(sim, qw_launch_measure(sim->d, sim->buf[sim->cur], inst, sim->fp32, pending_scale(sim), reg,
                                       dp, len, sim->stream));
    sim->launches++;
    QW_CUDA(sim, cudaMemcpyAsync(probs, dp, (size_t)len * sizeof(double), cudaMemcpyDeviceToHost,
                                 sim->stream));
    return check_status(sim, "qw_measure_register");
}

/* Same result as qw_measure_register, for callers that must not allocate
 * device memory: the histogram lives in a fixed scratch array of the library
 * (qw_kernels.cu) instead of the simulator's histogram, which
 * qw_measure_register allocates with cudaMalloc when a len exceeds every
 * earlier one.  This call never allocates. */
extern "C" int qw_measure_register_noalloc(qw_sim *sim, int32_t inst, int32_t reg, double *probs,
                                           int64_t len)
{
    if (!sim) return QW_ERR_ARG;
    if (inst < 0 || inst >= sim->d.ninst || reg < 0 || reg > 5 || !probs || len < 1)
        return fail(sim, QW_ERR_ARG, "bad instance, register id or output");
    if (len > QW_MEASURE_NOALLOC_MAX_LEN)
        return fail(sim, QW_ERR_ARG,
                    "qw_measure_register_noalloc: len " + std::to_string(len) + " exceeds the fixed scratch of " +
                        std::to_string(QW_MEASURE_NOALLOC_MAX_LEN) + " bins; use qw_measure_register");
    if (!sim->has_state) return fail(sim, QW_ERR_STATE, "no state");
    QW_CUDA(sim, qw_launch_measure_noalloc(sim->d, sim->buf[sim->cur], inst, sim->fp32, pending_scale(sim),
                                           reg, probs, len, sim->device, sim->stream,
                                           sim->pos_live ? sim->pbuf[sim->cur] : nullptr, pos_row0(sim, inst),
                                           sim->n_of[(size_t)inst]));
    sim->launches++;
    return check_status(sim, "qw_measure_register_noalloc");
}

extern "C" int qw_state_size(qw_sim *sim, int32_t inst, int64_t *count)
{
    if (!sim || !count) return QW_ERR_ARG;
    if (inst < -1 || inst >= sim->d.ninst) return fail(sim, QW_ERR_ARG, "instance out of range");
    if (!sim->has_state) return fail(sim, QW_ERR_STATE, "no state");
    {
        const int prc = pos_unpack(sim); /* the state back into the row buckets */
        if (prc != QW_OK) return prc;
    }
    QW_CUDA(sim, cudaMemsetAsync(&sim->sc->counter, 0, 8, sim->stream));
    QW_CUDA(sim, qw_launch_count(sim->d, sim->buf[sim->cur], inst, &sim->sc->counter, sim->stream));
    sim->launches++;
    unsigned long long c = 0;
    QW_CUDA(sim, cudaMemcpyAsync(&c, &sim->sc->counter, 8, cudaMemcpyDeviceToHost, sim->stream));
    QW_CUDA(sim, cudaStreamSynchronize(sim->stream));
    *count = (int64_t)c;
    return QW_OK;
}

static uint64_t get_bits(const uint64_t *w, int pos, int width)
{
    uint64_t v = 0;
    for (int b = 0; b < width; ++b)
        if ((w[(pos + b) >> 6] >> ((pos + b) & 63)) & 1ull) v |= 1ull << b;
    return v;
}

static void put_bits(uint64_t *w, int pos, uint64_t v, int width)
{
    for (int b = 0; b < width; ++b)
        if ((v >> b) & 1ull) w[(pos + b) >> 6] |= 1ull << ((pos + b) & 63);
}

extern "C" int qw_state_export(qw_sim *sim, int32_t inst, int32_t key_words, uint64_t *keys,
                               double *amps, int64_t cap, int64_t *count)
{
    if (!sim || !count) return QW_ERR_ARG;
    const int nb = sim->d.nb;
    const int bits = 4 * nb + 34;
    if (key_words < 1 || key_words > 10 || key_words * 64 < bits)
        return fail(sim, QW_ERR_ARG, "key_words too small for the packed register layout");
    if (cap > 0 && (!keys || !amps)) return fail(sim, QW_ERR_ARG, "null output arrays");
    int64_t total = 0;
    int rc = qw_state_size(sim, inst, &total);
    if (rc != QW_OK) return rc;
    *count = total;
    if (total == 0 || cap <= 0) return QW_OK;
    uint64_t *drow = nullptr, *dloc = nullptr;
    double2 *damp = nullptr;
    QW_CUDA(sim, cudaMallocAsync((void **)&drow, (size_t)total * 8, sim->stream));
    QW_CUDA(sim, cudaMallocAsync((void **)&dloc, (size_t)total * 8, sim->stream));
    QW_CUDA(sim, cudaMallocAsync((void **)&damp, (size_t)total * 16, sim->stream));
    QW_CUDA(sim, cudaMemsetAsync(&sim->sc->counter, 0, 8, sim->stream));
    QW_CUDA(sim, qw_launch_export(sim->d, sim->buf[sim->cur], inst, sim->fp32, pending_scale(sim), drow,
                                  dloc, damp, &sim->sc->counter, total, sim->stream));
    sim->launches++;
    std::vector<uint64_t> hrow((size_t)total), hloc((size_t)total);
    std::vector<double2> hamp((size_t)total);
    QW_CUDA(sim, cudaMemcpyAsync(hrow.data(), drow, (size_t)total * 8, cudaMemcpyDeviceToHost, sim->stream));
    QW_CUDA(sim, cudaMemcpyAsync(hloc.data(), dloc, (size_t)total * 8, cudaMemcpyDeviceToHost, sim->stream));
    QW_CUDA(sim, cudaMemcpyAsync(hamp.data(), damp, (size_t)total * 16, cudaMemcpyDeviceToHost, sim->stream));
    QW_CUDA(sim, cudaFreeAsync(drow, sim->stream));
    QW_CUDA(sim, cudaFreeAsync(dloc, sim->stream));
    QW_CUDA(sim, cudaFreeAsync(damp, sim->stream));
    rc = check_status(sim, "qw_state_export");
    if (rc != QW_OK) return rc;
    /* pack: b2 | k | kc | b1 | j | jc | A | inst */
    const size_t W = (size_t)key_words;
    std::vector<uint64_t> packed((size_t)total * W, 0ull);
    const uint64_t m = (1ull << nb) - 1;
    for (int64_t i = 0; i < total; ++i) {
        const uint64_t rk = hrow[(size_t)i], lk = hloc[(size_t)i];
        uint64_t *w = packed.data() + (size_t)i * W;
        int p = 0;
        put_bits(w, p, lk & 1ull, 1); p += 1;                      /* b2 */
        put_bits(w, p, (lk >> 1) & m, nb); p += nb;                /* k */
        put_bits(w, p, (lk >> (1 + nb)) & m, nb); p += nb;         /* kc */
        put_bits(w, p, rk & 1ull, 1); p += 1;                      /* b1 */
        put_bits(w, p, (rk >> 1) & 0x7ffffull, nb); p += nb;       /* j */
        put_bits(w, p, (rk >> 20) & 0xfffffull, nb); p += nb;      /* jc */
        put_bits(w, p, (lk >> (1 + 2 * nb)) & 0xffffull, 16); p += 16; /* A */
        put_bits(w, p, rk >> 40, 16);                              /* inst */
    }
    std::vector<int64_t> order((size_t)total);
    for (int64_t i = 0; i < total; ++i) order[(size_t)i] = i;
    std::sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
        const uint64_t *a = packed.data() + (size_t)x * W, *b = packed.data() + (size_t)y * W;
        for (size_t t = W; t-- > 0;)
            if (a[t] != b[t]) return a[t] < b[t];
        return false;
    });
    const int64_t nout = std::min(total, cap);
    for (int64_t i = 0; i < nout; ++i) {
        const int64_t src = order[(size_t)i];
        std::memcpy(keys + (size_t)i * W, packed.data() + (size_t)src * W, W * 8);
        amps[2 * i] = hamp[(size_t)src].x;
        amps[2 * i + 1] = hamp[(size_t)src].y;
    }
    return QW_OK;
}

extern "C" int qw_step_stats(qw_sim *sim, int64_t *out, int32_t len, int32_t reset)
{
    if (!sim || (len > 0 && !out)) return QW_ERR_ARG;
    unsigned long long h[QW_NSTAT] = {0};
    QW_CUDA(sim, cudaMemcpyAsync(h, sim->sc->stats, sizeof h, cudaMemcpyDeviceToHost, sim->stream));
    if (reset) QW_CUDA(sim, cudaMemsetAsync(sim->sc->stats, 0, sizeof h, sim->stream));
    QW_CUDA(sim, cudaStreamSynchronize(sim->stream));
    for (int i = 0; i < len && i < QW_NSTAT; ++i) out[i] = (int64_t)h[i];
    return QW_OK;
}

extern "C" int qw_state_import(qw_sim *sim, int32_t key_words, const uint64_t *keys, const double *amps,
                               int64_t count)
{
    if (!sim) return QW_ERR_ARG;
    if (sim->fq_open) return faithful_session_closed(sim);
    {
        const int prc = pos_unpack(sim); /* the state back into the row buckets */
        if (prc != QW_OK) return prc;
    }
    sim->pos_try = true;
    const int nb = sim->d.nb;
    if (key_words < 1 || key_words > 10 || key_words * 64 < 4 * nb + 34)
        return fail(sim, QW_ERR_ARG, "key_words too small for the packed register layout");
    if (count < 0 || (count > 0 && (!keys || !amps))) return fail(sim, QW_ERR_ARG, "bad arrays");
    const size_t W = (size_t)key_words;
    /* distinct keys */
    std::vector<int64_t> order((size_t)count);
    for (int64_t i = 0; i < count; ++i) order[(size_t)i] = i;
    std::sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
        const uint64_t *a = keys + (size_t)x * W, *b = keys + (size_t)y * W;
        for (size_t t = W; t-- > 0;)
            if (a[t] != b[t]) return a[t] < b[t];
        return false;
    });
    for (int64_t i = 1; i < count; ++i)
        if (std::memcmp(keys + (size_t)order[(size_t)i] * W, keys + (size_t)order[(size_t)i - 1] * W, W * 8) == 0)
            return fail(sim, QW_ERR_ARG, "qw_state_import: duplicate key");
    std::vector<uint64_t> hrow((size_t)count), hloc((size_t)count);
    std::vector<double2> hamp((size_t)count);
    double norm2 = 0.0;
    for (int64_t i = 0; i < count; ++i) {
        const uint64_t *w = keys + (size_t)i * W;
        int p = 0;
        const uint64_t b2 = get_bits(w, p, 1); p += 1;
        const uint64_t k = get_bits(w, p, nb); p += nb;
        const uint64_t kc = get_bits(w, p, nb); p += nb;
        const uint64_t b1 = get_bits(w, p, 1); p += 1;
        const uint64_t j = get_bits(w, p, nb); p += nb;
        const uint64_t jc = get_bits(w, p, nb); p += nb;
        const uint64_t A = get_bits(w, p, 16); p += 16;
        const uint64_t inst = get_bits(w, p, 16); p += 16;
        for (int t = p; t < (int)W * 64; ++t)
            if ((w[t >> 6] >> (t & 63)) & 1ull) return fail(sim, QW_ERR_ARG, "qw_state_import: bits above the layout");
        if (A != 0) return fail(sim, QW_ERR_ARG, "qw_state_import: register A must be 0");
        if ((int64_t)inst >= sim->d.ninst) return fail(sim, QW_ERR_ARG, "qw_state_import: instance out of range");
        hrow[(size_t)i] = qw_rowkey((uint32_t)inst, (uint32_t)jc, (uint32_t)j, (uint32_t)b1);
        hloc[(size_t)i] = b2 | (k << 1) | (kc << (1 + nb));
        hamp[(size_t)i] = make_double2(amps[2 * i], amps[2 * i + 1]);
        norm2 += amps[2 * i] * amps[2 * i] + amps[2 * i + 1] * amps[2 * i + 1];
    }
    if (sim->opts.overflow_fallback && count > 0) { /* a row longer than row_capacity: grow the buckets */
        std::vector<uint64_t> rows(hrow);
        std::sort(rows.begin(), rows.end());
        int64_t longest = 0;
        for (size_t i = 0, j = 0; i < rows.size(); i = j) {
            while (j < rows.size() && rows[j] == rows[i]) ++j;
            longest = std::max<int64_t>(longest, (int64_t)(j - i));
        }
        if (longest > sim->d.cap_row) {
            int rc = grow_rows(sim, longest);
            if (rc != QW_OK) return rc;
        }
    }
    for (int bi = 0; bi < 3; ++bi) {
        QW_CUDA(sim, qw_launch_clear(sim->d, sim->buf[bi], 0, sim->d.total_buckets, 1, sim->stream));
        sim->launches++;
    }
    Scalars z{};
    z.scale[0] = z.scale[1] = 1.0;
    z.renorm_target = norm2;
    QW_CUDA(sim, cudaMemcpyAsync(sim->sc, &z, sizeof z, cudaMemcpyHostToDevice, sim->stream));
    sim->scale_slot = sim->sync_slot = 0;
    sim->cur = sim->sync_cur = 0;
    sim->sync_done = 0;
    drop_graphs(sim);
    if (count > 0) {
        uint64_t *drow = nullptr, *dloc = nullptr;
        double2 *damp = nullptr;
        QW_CUDA(sim, cudaMallocAsync((void **)&drow, (size_t)count * 8, sim->stream));
        QW_CUDA(sim, cudaMallocAsync((void **)&dloc, (size_t)count * 8, sim->stream));
        QW_CUDA(sim, cudaMallocAsync((void **)&damp, (size_t)count * 16, sim->stream));
        QW_CUDA(sim, cudaMemcpyAsync(drow, hrow.data(), (size_t)count * 8, cudaMemcpyHostToDevice, sim->stream));
        QW_CUDA(sim, cudaMemcpyAsync(dloc, hloc.data(), (size_t)count * 8, cudaMemcpyHostToDevice, sim->stream));
        QW_CUDA(sim, cudaMemcpyAsync(damp, hamp.data(), (size_t)count * 16, cudaMemcpyHostToDevice, sim->stream));
        QW_CUDA(sim, qw_launch_import(sim->d, sim->buf[sim->cur], drow, dloc, damp, count, sim->fp32,
                                      &sim->sc->status, sim->stream));
        sim->launches++;
        QW_CUDA(sim, cudaFreeAsync(drow, sim->stream));
        QW_CUDA(sim, cudaFreeAsync(dloc, sim->stream));
        QW_CUDA(sim, cudaFreeAsync(damp, sim->stream));
    }
    int rc = check_status(sim, "qw_state_import");
    if (rc != QW_OK) return rc;
    sim->has_state = true;
    sim->fresh_T = false;
    for (auto &v : sim->init_norm2) v = 0.0;
    return QW_OK;
}

/* ---- row-partitioned walk ---------------------------------------------------------- */

extern "C" int qw_part_owner(int32_t n, int32_t nparts, int32_t jc, int32_t j)
{
    if (n < 1 || nparts < 1 || jc < 0 || j < 0) return -1;
    QwSimDev d{};
    d.n_single = n;
    d.nparts = nparts;
    d.part_rows = ((int64_t)n + nparts - 1) / nparts;
    return qw_part_owner_of(d, (uint32_t)jc, (uint32_t)j);
}

extern "C" int qw_part_outbox(qw_sim *sim, int32_t dest, qw_part_entry *dst, int64_t cap, int64_t *count)
{
    static_assert(sizeof(qw_part_entry) == sizeof(QwPartEntry), "outbox entry layout");
    if (!sim || !count) return QW_ERR_ARG;
    if (sim->d.nparts <= 1) return fail(sim, QW_ERR_STATE, "not a partitioned walk");
    if (dest < 0 || dest >= sim->d.nparts || (cap > 0 && !dst)) return fail(sim, QW_ERR_ARG, "bad destination");
    unsigned long long c = 0;
    QW_CUDA(sim, cudaMemcpyAsync(&c, sim->outbox_count + dest, 8, cudaMemcpyDeviceToHost, sim->stream));
    QW_CUDA(sim, cudaStreamSynchronize(sim->stream));
    const int64_t n = std::min<int64_t>((int64_t)c, sim->d.outbox_cap);
    *count = n;
    const int64_t m = std::min<int64_t>(n, cap);
    if (m > 0)
        QW_CUDA(sim, cudaMemcpyAsync(dst, sim->outbox + (int64_t)dest * sim->d.outbox_cap, (size_t)m * sizeof(QwPartEntry),
                                     cudaMemcpyDeviceToDevice, sim->stream));
    QW_CUDA(sim, cudaStreamSynchronize(sim->stream));
    return QW_OK;
}

extern "C" int qw_part_inbox(qw_sim *sim, const qw_part_entry *entries, int64_t count)
{
    if (!sim || count < 0 || (count > 0 && !entries)) return QW_ERR_ARG;
    if (sim->d.nparts <= 1) return fail(sim, QW_ERR_STATE, "not a partitioned walk");
    if (!sim->has_state) return fail(sim, QW_ERR_STATE, "no state");
    QW_CUDA(sim, qw_launch_part_inbox(sim->d, sim->buf[sim->cur], reinterpret_cast<const QwPartEntry *>(entries),
                                      count, sim->fp32, &sim->sc->status, sim->stream));
    sim->launches++;
    return check_status(sim, "qw_part_inbox");
}

extern "C" int qw_part_norm(qw_sim *sim, double *local_norm2)
{
    if (!sim || !local_norm2) return QW_ERR_ARG;
    QW_CUDA(sim, cudaMemcpyAsync(local_norm2, &sim->sc->norm[sim->scale_slot], 8, cudaMemcpyDeviceToHost, sim->stream));
    QW_CUDA(sim, cudaStreamSynchronize(sim->stream));
    return QW_OK;
}

extern "C" int qw_part_set_norm(qw_sim *sim, double global_norm2)
{
    if (!sim || !(global_norm2 >= 0.0)) return QW_ERR_ARG;
    double target = 1.0;
    QW_CUDA(sim, cudaMemcpyAsync(&target, &sim->sc->renorm_target, 8, cudaMemcpyDeviceToHost, sim->stream));
    QW_CUDA(sim, cudaStreamSynchronize(sim->stream));
    sim->host_target = (sim->renorm && global_norm2 > 0.0) ? std::sqrt(target / global_norm2) : 1.0;
    QW_CUDA(sim, cudaMemcpyAsync(&sim->sc->scale[sim->scale_slot], &sim->host_target, 8, cudaMemcpyHostToDevice,
                                 sim->stream));
    QW_CUDA(sim, cudaStreamSynchronize(sim->stream));
    return QW_OK;
}

extern "C" int qw_part_walk(qw_sim **sims, int32_t np, int64_t nsteps)
{
    if (!sims || np < 1 || np > 64 || nsteps < 0) return QW_ERR_ARG;
    for (int p = 0; p < np; ++p) {
        if (!sims[p] || sims[p]->d.nparts != np || sims[p]->d.part != p || sims[p]->device != sims[0]->device)
            return sims[p] ? fail(sims[p], QW_ERR_ARG, "qw_part_walk: not partitions 0 .. nparts - 1 of one walk")
                           : QW_ERR_ARG;
        if (!sims[p]->has_state) return fail(sims[p], QW_ERR_STATE, "no state");
        if (sims[p]->fq_open) return faithful_session_closed(sims[p]);
    }
    /* Per step, with no host synchronisation: every part's step kernel on
       its stream; then on each part q's stream, once every step is done, the
       entries the others' S sent to q are appended straight from their outbox
       segments (counts read on the device) and q's renormalisation factor is
       set from the norms of all parts' outputs.  A part's next step waits
       for every exchange of the previous one (its outbox is read there). */
    std::vector<cudaEvent_t> ev_step((size_t)np, nullptr), ev_x((size_t)np, nullptr);
    int rc = QW_OK;
    for (int p = 0; p < np && rc == QW_OK; ++p) {
        if (cudaEventCreateWithFlags(&ev_step[(size_t)p], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev_x[(size_t)p], cudaEventDisableTiming) != cudaSuccess)
            rc = fail(sims[p], QW_ERR_CUDA, "qw_part_walk: cudaEventCreate");
    }
    auto cuda = [&](qw_sim *sim, cudaError_t e, const char *what) {
        if (e != cudaSuccess && rc == QW_OK) rc = cuda_fail(sim, e, what);
    };
    for (int64_t t = 0; t < nsteps && rc == QW_OK; ++t) {
        for (int p = 0; p < np && rc == QW_OK; ++p) {
            qw_sim *sp = sims[p];
            if (t > 0)
                for (int q = 0; q < np; ++q)
                    if (q != p) cuda(sp, cudaStreamWaitEvent(sp->stream, ev_x[(size_t)q], 0), "cudaStreamWaitEvent");
            if (rc == QW_OK) rc = launch_walk(sp, 0);
            if (rc == QW_OK) cuda(sp, cudaEventRecord(ev_step[(size_t)p], sp->stream), "cudaEventRecord");
        }
        for (int q = 0; q < np && rc == QW_OK; ++q) {
            qw_sim *sq = sims[q];
            QwPartSources src{};
            QwPartNorms nm{};
            src.cap = sq->d.outbox_cap;
            for (int p = 0; p < np; ++p) {
                nm.norm[nm.n++] = &sims[p]->sc->norm[sims[p]->scale_slot]; /* the step's output norm */
                if (p == q) continue;
                cuda(sq, cudaStreamWaitEvent(sq->stream, ev_step[(size_t)p], 0), "cudaStreamWaitEvent");
                src.e[src.n] = sims[p]->outbox + (int64_t)q * sims[p]->d.outbox_cap;
                src.count[src.n] = sims[p]->outbox_count + q;
                src.n++;
                if (sims[p]->d.outbox_cap < src.cap) src.cap = sims[p]->d.outbox_cap;
            }
            cuda(sq, qw_launch_part_gather(sq->d, sq->buf[sq->cur], src, sq->fp32, &sq->sc->status, sq->stream),
                 "part gather launch");
            cuda(sq, qw_launch_part_scale(nm, &sq->sc->renorm_target, &sq->sc->scale[sq->scale_slot], sq->renorm,
                                          sq->stream),
                 "part scale launch");
            sq->launches += 2;
            cuda(sq, cudaEventRecord(ev_x[(size_t)q], sq->stream), "cudaEventRecord");
        }
    }
    /* the device status of every part (outbox or row overflow) */
    for (int p = 0; p < np; ++p) {
        if (sims[p]) {
            const int prc = check_status(sims[p], "qw_part_walk");
            if (rc == QW_OK) rc = prc;
        }
    }
    for (int p = 0; p < np; ++p) {
        if (ev_step[(size_t)p]) cudaEventDestroy(ev_step[(size_t)p]);
        if (ev_x[(size_t)p]) cudaEventDestroy(ev_x[(size_t)p]);
    }
    return rc;
}
