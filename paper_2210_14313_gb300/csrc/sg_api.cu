// Host side of libsg: the C ABI of include/sg.h, the planner that turns an
// integral into items / patterns / chunks, per-stream device workspaces and
// the launch sequence (setup -> prep -> fold [-> guard pass] [-> adjoint]).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/sg.h"
#include "sg_user.h"
#include "sg_kernels.h"
#include "sg_lacc.h"
#include "sg_plan.h"
#include "sg_rules.h"

#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return SG_ECUDA;    \
    } while (0)


// ---------------------------------------------------------------------------
// status strings
// ---------------------------------------------------------------------------

extern "C" const char *sg_status_string(sg_status s) {
    switch (s) {
    case SG_OK: return "ok";
    case SG_EINVAL: return "invalid argument";
    case SG_ERANGE: return "size beyond a supported limit";
    case SG_ENOMEM: return "out of memory";
    case SG_ECUDA: return "CUDA runtime error";
    case SG_ETIMEOUT: return "timeout";
    case SG_EUNSUPPORTED: return "unsupported combination";
    }
    return "unknown status";
}

static std::mutex g_mu;

// ---------------------------------------------------------------------------
// per-device context: SM count and the binomial table
// ---------------------------------------------------------------------------

struct DevCtx {
    int sms = 0;
    u64 *binom = nullptr;
    std::map<std::pair<int, int>, int> occ;  // (prec, warps per CTA) -> resident CTAs per SM
};

static int dev_occupancy(DevCtx *C, int prec, int warps) {
    auto key = std::make_pair(prec, warps);
    auto it = C->occ.find(key);
    if (it != C->occ.end()) return it->second;
    int n = sg_fold_occupancy(prec, 0, warps);
    if (n < 1) n = 1;
    C->occ[key] = n;
    return n;
}

static long long resident_warps(DevCtx *C, int prec, const sg_tuning &t) {
    const int per_sm = std::max(1, std::min(dev_occupancy(C, prec, t.warps_per_cta), t.ctas_per_sm));
    return (long long)C->sms * per_sm * t.warps_per_cta;
}
static std::map<int, DevCtx> g_dev;

static sg_status dev_ctx(DevCtx **out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    auto it = g_dev.find(dev);
    if (it != g_dev.end()) {
        *out = &it->second;
        return SG_OK;
    }
    DevCtx c;
    CK(cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev));
    std::vector<u64> B((size_t)SG_BINOM_K * (SG_MAX_D + 1));
    sg_fill_binomials(B.data());
    if (cudaMalloc(&c.binom, B.size() * sizeof(u64)) != cudaSuccess) return SG_ENOMEM;
    CK(cudaMemcpy(c.binom, B.data(), B.size() * sizeof(u64), cudaMemcpyHostToDevice));
    g_dev[dev] = c;
    *out = &g_dev[dev];
    return SG_OK;
}

// ---------------------------------------------------------------------------
// rules
// ---------------------------------------------------------------------------

extern "C" sg_status sg_rule_init(sg_rule_kind kind, int max_level, sg_rule *out) {
    return sg_rule_init_growth(kind, SG_GROWTH_STANDARD, max_level, out);
}

extern "C" sg_status sg_rule_init_growth(sg_rule_kind kind, sg_growth growth, int max_level, sg_rule *out) {
    if (!out || (kind != SG_RULE_TRAPEZOID && kind != SG_RULE_CLENSHAW_CURTIS &&
                 kind != SG_RULE_GAUSS_PATTERSON && kind != SG_RULE_GAUSS_LEGENDRE))
        return SG_EINVAL;
    if (growth != SG_GROWTH_STANDARD && growth != SG_GROWTH_SLOW) return SG_EINVAL;
    if (max_level < 1 || max_level > SG_MAX_LEVEL) return SG_ERANGE;
    const int ikind = (int)kind | (growth == SG_GROWTH_SLOW ? SG_KIND_SLOW : 0);
    for (int l = 1; l <= max_level; l++)
        if (sg_level_nodes(ikind, l) == 0) return SG_ERANGE;
    sg_rule_s *r = new sg_rule_s();
    r->kind = ikind;
    r->max_level = max_level;
    if (cudaGetDevice(&r->device) != cudaSuccess) {
        delete r;
        return SG_ECUDA;
    }
    std::vector<double> tx(2 * 4097 + 2), tw(2 * 4097 + 2);
    std::vector<double2> all;
    for (int bk = 0; bk < 4; bk++)
        for (int k = 1; k < max_level; k++) {
            int n = sg_block(ikind, bk, k, tx.data(), tw.data());
            r->x[bk][k].assign(tx.begin(), tx.begin() + n);
            r->w[bk][k].assign(tw.begin(), tw.begin() + n);
            r->off[bk][k] = (int)all.size();
            for (int j = 0; j < n; j++) all.push_back(make_double2(tx[j], tw[j]));
        }
    if (all.empty()) all.push_back(make_double2(0.5, 1.0));
    if (cudaMalloc(&r->d_xw, all.size() * sizeof(double2)) != cudaSuccess) {
        delete r;
        return SG_ENOMEM;
    }
    if (cudaMemcpy(r->d_xw, all.data(), all.size() * sizeof(double2), cudaMemcpyHostToDevice) !=
        cudaSuccess) {
        cudaFree(r->d_xw);
        delete r;
        return SG_ECUDA;
    }
    *out = r;
    return SG_OK;
}

static void plans_drop_rule(sg_rule r);
static void drop_all_graphs();

extern "C" sg_status sg_rule_destroy(sg_rule r) {
    if (!r) return SG_OK;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        plans_drop_rule(r);
    }
    cudaFree(r->d_xw);
    delete r;
    return SG_OK;
}

extern "C" sg_status sg_rule_nodes(sg_rule r, int level, double *x, double *w, int *n) {
    if (!r || !n) return SG_EINVAL;
    if (level < 1 || level > r->max_level) return SG_ERANGE;
    int m = sg_level_nodes(r->kind, level);
    if (x && w) {
        if (*n < m) return SG_ERANGE;
        sg_rule_level(r->kind, level, x, w);
    }
    *n = m;
    return SG_OK;
}

// ---------------------------------------------------------------------------
// tuning
// ---------------------------------------------------------------------------

// index 0: FP64, 1: mixed, 2: float-float
static sg_tuning g_tune[3] = {{2048, 4, 8}, {32768, 8, 4}, {32768, 8, 4}};

static bool prec_ok(int p) { return p == SG_PREC_FP64 || p == SG_PREC_MIXED || p == SG_PREC_FF; }

// Per-class chunk sizes of the batch path (sg_autotune_classes,
// sg_tuning_load): a class is (family, rule kind, ceil(log2 d), q - d,
// precision); its items are planned with the class's points per chunk.
typedef std::tuple<int, int, int, int, int> ClassKey;
static std::map<ClassKey, int> g_class_ppc;

static int d_bucket(int d) {
    int b = 0;
    while ((1 << b) < d) b++;
    return b;
}

static ClassKey class_key(const sg_item &it, int prec) {
    return ClassKey(it.fam, it.rule->kind, d_bucket(it.d), it.q - it.d, prec);
}

// Requires g_mu held.
static int class_ppc(const sg_item &it, int prec) {
    auto f = g_class_ppc.find(class_key(it, prec));
    return f == g_class_ppc.end() ? 0 : f->second;
}

extern "C" sg_status sg_get_tuning(sg_precision prec, sg_tuning *t) {
    if (!t || !prec_ok(prec)) return SG_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    *t = g_tune[prec];
    return SG_OK;
}

extern "C" sg_status sg_set_tuning(sg_precision prec, const sg_tuning *t) {
    if (!t || !prec_ok(prec)) return SG_EINVAL;
    if (t->points_per_chunk < 32 || t->points_per_chunk > (1 << 26) || t->ctas_per_sm < 1 ||
        t->ctas_per_sm > 32 || t->warps_per_cta < 1 || t->warps_per_cta > 32)
        return SG_ERANGE;
    std::lock_guard<std::mutex> lk(g_mu);
    g_tune[prec] = *t;
    return SG_OK;
}

// ---------------------------------------------------------------------------
// planning
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// plans on the device
// ---------------------------------------------------------------------------

template <typename T>
static size_t carve(size_t &cur, size_t n) {
    size_t off = (cur + 255) & ~(size_t)255;
    cur = off + n * sizeof(T);
    return off;
}

static void plan_free(Plan *P) {
    if (P->dmem) cudaFree(P->dmem);
    plan_free_host(P);
}

// Resolves the rule-block pointers and copies a host plan to the device.
static sg_status plan_upload(Plan *P, const u64 *d_binom) {
    cudaGetDevice(&P->device);
    // device copy, one allocation
    size_t sz = 0;
    const size_t o_int = carve<SgIntegralDev>(sz, P->integrals.size());
    const size_t o_blk = carve<SgBlockDev>(sz, P->blocks.size());
    const size_t o_be = carve<long long>(sz, P->block_end.size());
    const size_t o_it = carve<SgItemDev>(sz, P->items.size());
    const size_t o_ro = carve<SgItemRole>(sz, P->roles.size());
    const size_t o_ii = carve<int>(sz, P->item_integral.size());
    const size_t o_pa = carve<SgPatDev>(sz, P->pats.size());
    const size_t o_pc = carve<u64>(sz, P->pat_chunk0.size());
    const size_t o_ip = carve<int>(sz, P->int_item_ptr.size());
    const size_t o_iv = carve<int>(sz, P->int_items.size() + 1);
    const size_t o_do = carve<int>(sz, P->delta_off.size() + 1);
    const size_t o_dm = carve<int>(sz, P->delta_m.size() + 1);
    const size_t o_cs = carve<SgChunkStart>(sz, (size_t)P->nchunks);
    const size_t o_w64 = carve<SgW64>(sz, P->wt64.size());
    const size_t o_wff = carve<float2>(sz, P->wtff.size());
    std::vector<unsigned char> host(sz, 0);
    memcpy(&host[o_int], P->integrals.data(), P->integrals.size() * sizeof(SgIntegralDev));
    memcpy(&host[o_blk], P->blocks.data(), P->blocks.size() * sizeof(SgBlockDev));
    memcpy(&host[o_be], P->block_end.data(), P->block_end.size() * sizeof(long long));
    memcpy(&host[o_it], P->items.data(), P->items.size() * sizeof(SgItemDev));
    memcpy(&host[o_ro], P->roles.data(), P->roles.size() * sizeof(SgItemRole));
    memcpy(&host[o_ii], P->item_integral.data(), P->item_integral.size() * sizeof(int));
    memcpy(&host[o_pa], P->pats.data(), P->pats.size() * sizeof(SgPatDev));
    memcpy(&host[o_pc], P->pat_chunk0.data(), P->pat_chunk0.size() * sizeof(u64));
    memcpy(&host[o_ip], P->int_item_ptr.data(), P->int_item_ptr.size() * sizeof(int));
    memcpy(&host[o_iv], P->int_items.data(), P->int_items.size() * sizeof(int));
    if (!P->delta_off.empty()) {
        memcpy(&host[o_do], P->delta_off.data(), P->delta_off.size() * sizeof(int));
        memcpy(&host[o_dm], P->delta_m.data(), P->delta_m.size() * sizeof(int));
    }
    if (!P->wt64.empty()) {
        memcpy(&host[o_w64], P->wt64.data(), P->wt64.size() * sizeof(SgW64));
        memcpy(&host[o_wff], P->wtff.data(), P->wtff.size() * sizeof(float2));
    }
    if (cudaMalloc(&P->dmem, sz) != cudaSuccess) {
        P->dmem = nullptr;
        return SG_ENOMEM;
    }
    if (cudaMemcpy(P->dmem, host.data(), sz, cudaMemcpyHostToDevice) != cudaSuccess) return SG_ECUDA;
    unsigned char *b = (unsigned char *)P->dmem;
    P->d_integrals = (SgIntegralDev *)(b + o_int);
    P->d_blocks = (SgBlockDev *)(b + o_blk);
    P->d_block_end = (long long *)(b + o_be);
    P->d_items = (SgItemDev *)(b + o_it);
    P->d_roles = (SgItemRole *)(b + o_ro);
    P->d_item_integral = (int *)(b + o_ii);
    P->d_pats = (SgPatDev *)(b + o_pa);
    P->d_pat_chunk0 = (u64 *)(b + o_pc);
    P->d_int_item_ptr = (int *)(b + o_ip);
    P->d_int_items = (int *)(b + o_iv);
    P->d_delta_off = (int *)(b + o_do);
    P->d_delta_m = (int *)(b + o_dm);
    P->d_delta_xw = P->reqs[0].rule->d_xw;
    P->d_wt64 = (const SgW64 *)(b + o_w64);
    P->d_wtff = (const float2 *)(b + o_wff);
    // chunk starts: unranked once per plan on the device (the legacy stream,
    // like the copy above, and waited for, since callers' streams may not
    // synchronise with it)
    P->d_chunk_start = (SgChunkStart *)(b + o_cs);
    if (P->nchunks > 0) {
        if (sg_launch_chunk_starts(P->d_items, P->d_pats, P->d_pat_chunk0, (long long)P->pats.size(), P->nchunks,
                                   d_binom, P->d_chunk_start, 0) != cudaSuccess ||
            cudaStreamSynchronize(0) != cudaSuccess)
            return SG_ECUDA;
    }
    return SG_OK;
}

static sg_status build_plan(const std::vector<Req> &reqs, int prec, const sg_tuning &tune,
                            long long warps, const u64 *d_binom, Plan **out) {
    static unsigned long long next_id = 0;
    Plan *P = nullptr;
    sg_status st = build_plan_host(reqs, prec, tune, warps, &P);
    if (st != SG_OK) return st;
    P->id = ++next_id;
    st = plan_upload(P, d_binom);
    if (st != SG_OK) {
        plan_free(P);
        return st;
    }
    *out = P;
    return SG_OK;
}

// ---------------------------------------------------------------------------
// plan cache
// ---------------------------------------------------------------------------

struct PlanKey {
    std::vector<Req> reqs;
    int prec;
    sg_tuning t;
    int device;
    bool operator<(const PlanKey &o) const {
        if (device != o.device) return device < o.device;
        if (prec != o.prec) return prec < o.prec;
        if (t.points_per_chunk != o.t.points_per_chunk) return t.points_per_chunk < o.t.points_per_chunk;
        if (t.ctas_per_sm != o.t.ctas_per_sm) return t.ctas_per_sm < o.t.ctas_per_sm;
        if (t.warps_per_cta != o.t.warps_per_cta) return t.warps_per_cta < o.t.warps_per_cta;
        if (reqs.size() != o.reqs.size()) return reqs.size() < o.reqs.size();
        for (size_t i = 0; i < reqs.size(); i++) {
            const Req &a = reqs[i], &b = o.reqs[i];
            auto ta = std::make_tuple(a.rule, a.fam, a.d, a.L, a.form, a.param_off, a.grad, a.ppc);
            auto tb = std::make_tuple(b.rule, b.fam, b.d, b.L, b.form, b.param_off, b.grad, b.ppc);
            if (ta != tb) return ta < tb;
        }
        return false;
    }
};
static std::map<PlanKey, Plan *> g_plans;

// Cached graphs hold kernel parameters that point into plans' device memory:
// every graph is dropped before any plan is freed.
static void plans_drop_rule(sg_rule r) {
    bool any = false;
    for (auto &kv : g_plans)
        for (auto &q : kv.first.reqs) any |= q.rule == r;
    if (any) drop_all_graphs();
    for (auto it = g_plans.begin(); it != g_plans.end();) {
        bool uses = false;
        for (auto &q : it->first.reqs) uses |= q.rule == r;
        if (uses) {
            cudaDeviceSynchronize();
            plan_free(it->second);
            it = g_plans.erase(it);
        } else {
            ++it;
        }
    }
}

// Requires g_mu held.
static sg_status get_plan(const std::vector<Req> &reqs, int prec, Plan **out) {
    DevCtx *C = nullptr;
    sg_status st = dev_ctx(&C);
    if (st != SG_OK) return st;
    PlanKey k;
    k.reqs = reqs;
    k.prec = prec;
    k.t = g_tune[prec];
    cudaGetDevice(&k.device);
    auto it = g_plans.find(k);
    if (it != g_plans.end()) {
        *out = it->second;
        return SG_OK;
    }
    // FP64 folds come in two builds (sg_kernels.cu): a single integral, which
    // is latency-bound, takes the one without a register budget (2 CTAs per
    // SM); batches take the one for 3 CTAs per SM
    const bool narrow = prec == SG_PREC_FP64 && reqs.size() == 1 && reqs[0].ppc == 0;
    sg_tuning t = k.t;
    if (narrow) t.ctas_per_sm = std::min(t.ctas_per_sm, 2);
    Plan *P = nullptr;
    st = build_plan(reqs, prec, t, resident_warps(C, prec == SG_PREC_FP64 && !narrow ? 3 : prec, t), C->binom, &P);
    if (st != SG_OK) return st;
    P->narrow = narrow;
    if (g_plans.size() > 256) {  // bound the cache
        cudaDeviceSynchronize();
        drop_all_graphs();
        for (auto &kv : g_plans) plan_free(kv.second);
        g_plans.clear();
    }
    g_plans[k] = P;
    *out = P;
    return SG_OK;
}

// ---------------------------------------------------------------------------
// per-stream workspaces
// ---------------------------------------------------------------------------

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

struct GraphEntry {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
};

struct Workspace {
    int device = 0;
    cudaStream_t stream = nullptr;
    DevBuf tab32, tab64, tabff, slots, gslots, counters, flags, bases, vars, out, vout, grad, params, lacc, ilacc;
    // the first 16 bytes of `counters` (work counter, finished-CTA count and
    // window flag of single-integral folds) and `lacc` are zero between
    // calls; false until a fresh allocation has been cleared
    bool la_clean = false;
    void *h_pinned = nullptr;
    size_t h_cap = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev_join = nullptr;
    cudaStream_t own = nullptr;  // capture/replay stream of batch graphs (never the legacy stream)
    unsigned epoch = 0;
    std::map<std::tuple<unsigned long long, const double *, double, unsigned>, GraphEntry> graphs;  // plan id
    // fold-kernel timing (sg_profile_begin / sg_profile_end)
    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof;
    size_t prof_used = 0;
};

// Records an event pair around a fold launch when profiling is on.
static cudaError_t prof_mark(Workspace *W, bool start, cudaStream_t s) {
    if (!W->profiling) return cudaSuccess;
    if (start) {
        if (W->prof_used == W->prof.size()) {
            std::pair<cudaEvent_t, cudaEvent_t> ev;
            cudaError_t e = cudaEventCreate(&ev.first);
            if (e == cudaSuccess) e = cudaEventCreate(&ev.second);
            if (e != cudaSuccess) return e;
            W->prof.push_back(ev);
        }
        return cudaEventRecord(W->prof[W->prof_used].first, s);
    }
    return cudaEventRecord(W->prof[W->prof_used++].second, s);
}
static std::map<std::pair<int, cudaStream_t>, Workspace *> g_ws;

static void drop_graphs(Workspace *W) {
    for (auto &kv : W->graphs) {
        if (kv.second.x) cudaGraphExecDestroy(kv.second.x);
        if (kv.second.g) cudaGraphDestroy(kv.second.g);
    }
    W->graphs.clear();
}

static void drop_all_graphs() {
    for (auto &kv : g_ws) {
        Workspace *W = kv.second;
        cudaStreamSynchronize(W->stream);
        if (W->own) cudaStreamSynchronize(W->own);
        drop_graphs(W);
    }
}

static sg_status get_ws(cudaStream_t s, Workspace **out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    auto key = std::make_pair(dev, s);
    auto it = g_ws.find(key);
    if (it != g_ws.end()) {
        *out = it->second;
        return SG_OK;
    }
    Workspace *W = new Workspace();
    W->device = dev;
    W->stream = s;
    if (cudaEventCreate(&W->ev0) != cudaSuccess || cudaEventCreate(&W->ev1) != cudaSuccess ||
        cudaEventCreateWithFlags(&W->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&W->own, cudaStreamNonBlocking) != cudaSuccess) {
        delete W;
        return SG_ECUDA;
    }
    g_ws[key] = W;
    *out = W;
    return SG_OK;
}

static sg_status ensure(Workspace *W, DevBuf &b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.p && b.cap >= bytes) return SG_OK;
    cudaStreamSynchronize(W->stream);
    if (W->own) cudaStreamSynchronize(W->own);
    drop_graphs(W);
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    size_t cap = std::max(bytes, b.cap + b.cap / 2);
    cap = (cap + 4095) & ~(size_t)4095;
    if (cudaMalloc(&b.p, cap) != cudaSuccess) {
        b.p = nullptr;
        b.cap = 0;
        cudaGetLastError();
        return SG_ENOMEM;
    }
    b.cap = cap;
    W->epoch++;
    W->la_clean = false;
    return SG_OK;
}

static sg_status ensure_host(Workspace *W, size_t bytes) {
    if (W->h_pinned && W->h_cap >= bytes) return SG_OK;
    cudaStreamSynchronize(W->stream);
    if (W->h_pinned) cudaFreeHost(W->h_pinned);
    W->h_pinned = nullptr;
    size_t cap = std::max<size_t>(bytes, 4096);
    if (cudaMallocHost(&W->h_pinned, cap) != cudaSuccess) {
        W->h_pinned = nullptr;
        W->h_cap = 0;
        cudaGetLastError();
        return SG_ENOMEM;
    }
    W->h_cap = cap;
    return SG_OK;
}

#define ST(call)                         \
    do {                                 \
        sg_status s_ = (call);           \
        if (s_ != SG_OK) return s_;      \
    } while (0)

// Effective unit roundoff of a precision: the error estimate of a result is
// 0.05 * this * cond.  Double: 2^-53; float-float: 2^-44 (about 44
// significant bits).  The float fold's rounding errors reach 0.33 * 2^-24 *
// cond (the largest over the 4096 integrals of the batch workload, measured
// against the separable pin), so its estimate uses 10 * 2^-24: 0.5 * 2^-24 *
// cond, an upper bound there, which the precision guard relies on.
static double unit_roundoff(int prec) {
    return prec == 1 ? 5.9604644775390625e-07 : (prec == 2 ? 5.6843418860808015e-14 : 1.1102230246251565e-16);
}

// Counters: [u64 work][u32 CTAs finished][u32 window flag][u32 item tickets]
// [u32 group tickets].
static size_t counter_bytes(const Plan *P) { return 16 + 4 * (P->items.size() + P->ngroups); }

// The launch's long accumulator of a single-integral fold (sum, absolute sum),
// and one per item of a batch.
static const size_t kLaccBytes = (size_t)2 * SG_LA_DIGITS * sizeof(long long);
static const size_t kItemLaccBytes = kLaccBytes;

// A contiguous range of a plan's chunk queue for one launch of a sharded
// batch (sg_integrate_batch_shard): its items are not assembled.
struct ShardRange {
    unsigned long long lo = 0, hi = 0;  // hi 0: the whole queue
    bool on = false;
};

// Makes every buffer a plan needs large enough (outside any capture).
static sg_status ws_prepare(Workspace *W, const Plan *P, bool need32, bool need64, bool needff,
                            size_t param_doubles) {
    if (need32) ST(ensure(W, W->tab32, (size_t)P->nentries * sizeof(float2)));
    if (need64) ST(ensure(W, W->tab64, (size_t)P->nentries * sizeof(double2)));
    if (needff) ST(ensure(W, W->tabff, (size_t)P->nentries * sizeof(float4)));
    ST(ensure(W, W->slots, (size_t)P->nchunks * sizeof(SgSlot)));
    ST(ensure(W, W->gslots, (size_t)P->ngroups * sizeof(SgGroupSlot)));
    ST(ensure(W, W->ilacc, P->items.size() * kItemLaccBytes));
    ST(ensure(W, W->counters, counter_bytes(P)));
    ST(ensure(W, W->flags, 4 * P->items.size()));
    ST(ensure(W, W->bases, P->integrals.size() * sizeof(SgBaseDev)));
    ST(ensure(W, W->vars, P->items.size() * sizeof(SgItemVar)));
    ST(ensure(W, W->out, (size_t)P->nout * sizeof(SgOutDev)));
    ST(ensure(W, W->vout, (size_t)std::max<long long>(P->nv, 1) * sizeof(double)));
    ST(ensure(W, W->grad, (size_t)2 * std::max(P->max_d, 1) * sizeof(double)));
    if (param_doubles) ST(ensure(W, W->params, param_doubles * sizeof(double)));
    ST(ensure(W, W->lacc, kLaccBytes));
    return SG_OK;
}

// The fold build for a plan and precision (sg_launch_fold's prec code).
static int fold_kind(const Plan *P, int prec) { return prec == SG_PREC_FP64 && !P->narrow ? 3 : prec; }

static SgLaunchCfg fold_cfg(const Plan *P, int prec, DevCtx *C) {
    prec = fold_kind(P, prec);
    SgLaunchCfg c;
    c.warps_per_cta = P->tune.warps_per_cta;
    int occ = dev_occupancy(C, prec, c.warps_per_cta);
    int per_sm = std::max(1, std::min(occ, P->tune.ctas_per_sm));
    long long ctas = (long long)C->sms * per_sm;
    const long long need = (long long)((P->nchunks + c.warps_per_cta - 1) / c.warps_per_cta);
    if (need < ctas) ctas = std::max<long long>(need, 1);
    c.ctas = (int)ctas;
    c.dependent = P->nchunks <= SG_DEPENDENT_LAUNCH_MAX_CHUNKS ? 1 : 0;
    return c;
}

// Enqueues the whole computation of a plan on W->stream (capturable: no
// allocation, no synchronisation).  prec_run: 0 FP64, 1 mixed.
// A user integrand's compiled fold kernel and what it is launched with.
struct UserFold {
    cudaKernel_t kern;
    int K;
    const double *params;
    int d;
};

// Host image of SgUserArgs in sg_user_kernel.cuh (same layout).
struct SgUserArgsHost {
    const double *params;
    int d;
    int pad;
};

static cudaError_t launch_user_fold(const UserFold &uf, SgFoldArgs &fa, const Plan *P, DevCtx *C,
                                    cudaStream_t s) {
    const int warps = 4;
    const size_t smem = (size_t)warps * (SG_USER_APAD * (uf.K + 1) * sizeof(double) + SG_MAX_R * sizeof(int));
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)uf.kern, 32 * warps, smem);
    if (e != cudaSuccess) return e;
    per_sm = std::max(1, std::min(per_sm, 8));
    long long ctas = (long long)C->sms * per_sm;
    const long long need = (long long)((P->nchunks + warps - 1) / warps);
    if (need < ctas) ctas = std::max<long long>(need, 1);
    SgUserArgsHost ua{uf.params, uf.d, 0};
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)ctas);
    lc.blockDim = dim3(32 * warps);
    lc.dynamicSmemBytes = smem;
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = attr;
    lc.numAttrs = P->nchunks <= SG_DEPENDENT_LAUNCH_MAX_CHUNKS ? 1 : 0;
    void *args[] = {&fa, &ua};
    return cudaLaunchKernelExC(&lc, (const void *)uf.kern, args);
}

// single_ok: the plan may use the single-integral fold (not inside a graph
// capture, whose replays would not see the host's record of the counters).
static sg_status run_plan(const Plan *P, Workspace *W, DevCtx *C, const double *d_params,
                          double guard_tol, SgOutDev *d_out, cudaStream_t s, const UserFold *uf = nullptr,
                          bool single_ok = true, ShardRange shard = ShardRange()) {
    const int prec = P->prec;
    const int nitems = (int)P->items.size();
    SgOutDev *outp = d_out ? d_out : (SgOutDev *)W->out.p;
    // one forward integral: chunk sums go into per-CTA long accumulators and
    // the counters return to zero at the end of the fold, so no clearing
    // launch precedes it (except on fresh memory)
    const bool single = single_ok && !shard.on && !uf && guard_tol == 0.0 && nitems == 1 &&
                        P->integrals.size() == 1 && P->roles[0].role == SG_ROLE_FORWARD && P->nchunks > 0;
    // the built-in folds of everything else add each chunk into its item's
    // long accumulator (cleared before every fold launch)
    const bool items_lacc = !single && !uf;
    const size_t ilacc_bytes = (size_t)nitems * kItemLaccBytes;
    if (single) {
        if (!W->la_clean) {
            CK(cudaMemsetAsync(W->counters.p, 0, 16, s));
            CK(cudaMemsetAsync(W->lacc.p, 0, kLaccBytes, s));
        }
    } else {
        CK(cudaMemsetAsync(W->counters.p, 0, counter_bytes(P), s));
    }
    if (guard_tol > 0.0) CK(cudaMemsetAsync(W->flags.p, 0, 4 * (size_t)nitems, s));
    SgSetupArgs sa;
    memset(&sa, 0, sizeof(sa));
    sa.blocks = P->d_blocks;
    sa.block_end = P->d_block_end;
    sa.nblocks = (int)P->blocks.size();
    if (sa.nblocks <= SG_SETUP_INLINE) {
        sa.ninline = sa.nblocks;
        for (int b = 0; b < sa.nblocks; b++) {
            sa.blk_inline[b] = P->blocks[b];
            sa.end_inline[b] = P->block_end[b];
        }
    }
    sa.nentries = P->nentries;
    sa.integrals = P->d_integrals;
    sa.nintegrals = (int)P->integrals.size();
    sa.params = d_params;
    sa.tab32 = prec == 1 ? (float2 *)W->tab32.p : nullptr;
    sa.tab64 = prec == 0 ? (double2 *)W->tab64.p : nullptr;
    sa.tabff = prec == 2 ? (float4 *)W->tabff.p : nullptr;
    sa.bases = (SgBaseDev *)W->bases.p;
    sa.flags = nullptr;
    const double u = unit_roundoff(prec);
    sa.do_items = 1;
    sa.int_item_ptr = P->d_int_item_ptr;
    sa.int_items = P->d_int_items;
    sa.roles = P->d_roles;
    sa.items = P->d_items;
    sa.item_integral = P->d_item_integral;
    sa.vars = (SgItemVar *)W->vars.p;
    sa.out = outp;
    sa.vout = (double *)W->vout.p;
    sa.unit_roundoff = u;
    CK(sg_launch_setup(sa, s));
    if (P->nchunks == 0 && !uf) return SG_OK;  // a user fold also writes the centre-only result
    SgFoldArgs fa;
    memset(&fa, 0, sizeof(fa));
    fa.items = P->d_items;
    fa.vars = (SgItemVar *)W->vars.p;
    fa.nitems = nitems;
    fa.pats = P->d_pats;
    fa.pat_chunk0 = P->d_pat_chunk0;
    fa.chunk_start = P->d_chunk_start;
    fa.npat = (long long)P->pats.size();
    fa.nchunks = P->nchunks;
    fa.tab = prec == 1 ? W->tab32.p : (prec == 2 ? W->tabff.p : W->tab64.p);
    fa.binom = C->binom;
    fa.slots = (SgSlot *)W->slots.p;
    fa.work = (unsigned long long *)W->counters.p;
    fa.item_done = (unsigned int *)((char *)W->counters.p + 16);
    fa.gslots = (SgGroupSlot *)W->gslots.p;
    fa.group_done = fa.item_done + nitems;
    fa.bases = (SgBaseDev *)W->bases.p;
    fa.item_integral = P->d_item_integral;
    fa.out = outp;
    fa.vout = (double *)W->vout.p;
    fa.flags = (guard_tol > 0.0) ? (int *)W->flags.p : nullptr;
    fa.skip_unflagged = nullptr;
    fa.guard_tol = guard_tol;
    fa.unit_roundoff = u;
    fa.single = single ? 1 : 0;
    fa.wtab = prec == 0 ? (const void *)P->d_wt64 : (const void *)P->d_wtff;
    fa.lacc = (long long *)W->lacc.p;
    fa.cta_done = (unsigned int *)((char *)W->counters.p + 8);
    fa.ilacc = items_lacc ? (long long *)W->ilacc.p : nullptr;
    fa.no_assemble = shard.on ? 1 : 0;
    fa.chunk_lo = shard.lo;
    fa.chunk_hi = shard.hi;
    if (items_lacc) CK(cudaMemsetAsync(W->ilacc.p, 0, ilacc_bytes, s));
    CK(prof_mark(W, true, s));
    if (uf) CK(launch_user_fold(*uf, fa, P, C, s));
    else CK(sg_launch_fold(fa, fold_kind(P, prec), 0, fold_cfg(P, prec, C), s));
    CK(prof_mark(W, false, s));
    if (single) W->la_clean = true;
    if (prec == 1 && guard_tol > 0.0) {
        // precision guard: the items whose estimate exceeds guard_tol are
        // recomputed in float-float, which flags again those whose float-float
        // estimate still exceeds it; those are recomputed in FP64
        CK(cudaMemsetAsync(W->counters.p, 0, counter_bytes(P), s));
        CK(cudaMemsetAsync(W->ilacc.p, 0, ilacc_bytes, s));
        sa.tab32 = nullptr;
        sa.tabff = (float4 *)W->tabff.p;
        sa.flags = (int *)W->flags.p;
        sa.do_items = 0;
        CK(sg_launch_setup(sa, s));
        fa.tab = W->tabff.p;
        fa.wtab = P->d_wtff;
        fa.skip_unflagged = (int *)W->flags.p;
        fa.guard_tol = guard_tol;
        fa.unit_roundoff = unit_roundoff(2);
        CK(prof_mark(W, true, s));
        CK(sg_launch_fold(fa, 2, 0, fold_cfg(P, 2, C), s));
        CK(prof_mark(W, false, s));
        CK(cudaMemsetAsync(W->counters.p, 0, counter_bytes(P), s));
        CK(cudaMemsetAsync(W->ilacc.p, 0, ilacc_bytes, s));
        sa.tabff = nullptr;
        sa.tab64 = (double2 *)W->tab64.p;
        CK(sg_launch_setup(sa, s));
        fa.tab = W->tab64.p;
        fa.wtab = P->d_wt64;
        fa.guard_tol = 0.0;
        fa.unit_roundoff = unit_roundoff(0);
        CK(prof_mark(W, true, s));
        CK(sg_launch_fold(fa, fold_kind(P, 0), 0, fold_cfg(P, 0, C), s));
        CK(prof_mark(W, false, s));
    }
    // leave the counters of the single-integral fold as it expects them
    if (!single) CK(cudaMemsetAsync(W->counters.p, 0, 16, s));
    return SG_OK;
}

// ---------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------

// The form SG_FORM_AUTO stands for: the merged form (every distinct point
// of the sparse grid once, with its merged weight).  It evaluates the fewest
// points (n_d^q / 7.6 for Clenshaw-Curtis at d = 200, L = 5; fewer than the
// n_d^q of Eq. 2.6 for Gauss-Legendre, whose difference forms need 2l - 1
// nodes per active direction), and since merging adds terms that share a
// point, its sum of |w_p D_p| is no larger than the difference form's: no
// worse conditioned, and unlike Eq. 2.6 free of binomial coefficients.
static sg_form auto_form(sg_rule, int, int, int) { return SG_FORM_MERGED; }

static sg_status check_one(sg_rule rule, sg_family fam, int d, int q, sg_precision prec,
                           sg_form *form) {
    if (!rule) return SG_EINVAL;
    if ((int)fam < 0 || (int)fam > 4) return SG_EINVAL;
    if (!prec_ok(prec)) return SG_EINVAL;
    if ((int)*form < 0 || (int)*form > 4) return SG_EINVAL;
    if (d < 1 || q < d) return SG_EINVAL;
    if (*form == SG_FORM_AUTO) *form = auto_form(rule, d, q - d, prec);
    if (d > SG_MAX_D) return SG_ERANGE;
    const int L = q - d;
    if (L > SG_MAX_L || L + 1 > rule->max_level) return SG_ERANGE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SG_ECUDA;
    if (dev != rule->device) return SG_EINVAL;
    return SG_OK;
}

static void fill_result(const SgOutDev &o, const Plan *P, int g, double ms, sg_result *r) {
    r->value = o.value;
    r->mant = o.mant;
    r->exp2 = (int64_t)o.exp2;
    r->cond = o.cond;
    r->err_est = o.err_est;
    r->points = P->points[g];
    r->evals = P->evals[g];
    r->seconds = ms * 1e-3;
}

extern "C" sg_status sg_count_points(sg_rule rule, int d, int q, sg_form form, uint64_t *points,
                                     uint64_t *evals) {
    if (!rule || !points) return SG_EINVAL;
    if ((int)form < 0 || (int)form > 4) return SG_EINVAL;
    if (d < 1 || q < d) return SG_EINVAL;
    if (form == SG_FORM_AUTO) form = auto_form(rule, d, q - d, SG_PREC_FP64);
    if (d > SG_MAX_D) return SG_ERANGE;
    const int L = q - d;
    if (L > SG_MAX_L || L + 1 > rule->max_level) return SG_ERANGE;
    u64 pts = 0;
    if (!count_points(rule->kind, d, L, &pts)) return SG_ERANGE;
    if (evals) {
        std::vector<PatSpec> specs;
        gen_patterns(form, d, L, specs);
        drop_empty_patterns(rule, specs);
        unsigned __int128 tot = 0;
        for (auto &sp : specs) {
            unsigned __int128 v = binom128(d, sp.r);
            for (int t = 0; t < sp.r - 1; t++) v *= (unsigned __int128)tab_m(rule, sp.pre[t]);
            v *= (unsigned __int128)tab_m(rule, sp.tail);
            tot += v;
        }
        if (tot > (unsigned __int128)~0ull) return SG_ERANGE;
        *evals = (u64)tot;
    }
    *points = pts;
    return SG_OK;
}

extern "C" sg_status sg_integrate_async(sg_rule rule, sg_family fam, const double *d_params, int d,
                                        int q, sg_precision prec, sg_form form, void *stream,
                                        sg_dev_result *d_out) {
    if (!d_params || !d_out) return SG_EINVAL;
    ST(check_one(rule, fam, d, q, prec, &form));
    std::lock_guard<std::mutex> lk(g_mu);
    cudaGetLastError();  // a failed earlier call must not surface here
    DevCtx *C = nullptr;
    ST(dev_ctx(&C));
    Plan *P = nullptr;
    std::vector<Req> reqs(1);
    memset(reqs.data(), 0, sizeof(Req));
    reqs[0] = Req{rule, (int)fam, d, q - d, (int)form, 0, 0};
    ST(get_plan(reqs, prec, &P));
    Workspace *W = nullptr;
    ST(get_ws((cudaStream_t)stream, &W));
    ST(ws_prepare(W, P, prec == SG_PREC_MIXED, prec == SG_PREC_FP64, prec == SG_PREC_FF, 0));
    return run_plan(P, W, C, d_params, 0.0, (SgOutDev *)d_out, (cudaStream_t)stream);
}

extern "C" sg_status sg_integrate(sg_rule rule, sg_family fam, const double *params,
                                  int params_on_device, int d, int q, sg_precision prec, sg_form form,
                                  void *stream, sg_result *out) {
    if (!params || !out) return SG_EINVAL;
    ST(check_one(rule, fam, d, q, prec, &form));
    std::lock_guard<std::mutex> lk(g_mu);
    cudaGetLastError();  // a failed earlier call must not surface here
    DevCtx *C = nullptr;
    ST(dev_ctx(&C));
    Plan *P = nullptr;
    std::vector<Req> reqs(1);
    memset(reqs.data(), 0, sizeof(Req));
    reqs[0] = Req{rule, (int)fam, d, q - d, (int)form, 0, 0};
    ST(get_plan(reqs, prec, &P));
    Workspace *W = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    ST(get_ws(s, &W));
    ST(ws_prepare(W, P, prec == SG_PREC_MIXED, prec == SG_PREC_FP64, prec == SG_PREC_FF,
                  params_on_device ? 0 : 2 * (size_t)d));
    ST(ensure_host(W, sizeof(SgOutDev)));
    const double *dp = params;
    if (!params_on_device) {
        // host parameters: staged in the pinned buffer after the result record and
        // read there by the setup kernel (the buffer is mapped into the device's
        // address space), else copied to the device
        ST(ensure_host(W, 256 + 2 * (size_t)d * sizeof(double)));
        double *hp = (double *)((char *)W->h_pinned + 256);
        memcpy(hp, params, 2 * (size_t)d * sizeof(double));
        void *dpp = nullptr;
        if (cudaHostGetDevicePointer(&dpp, hp, 0) != cudaSuccess) {
            cudaGetLastError();
            CK(cudaMemcpyAsync(W->params.p, params, 2 * (size_t)d * sizeof(double), cudaMemcpyHostToDevice, s));
            dpp = W->params.p;
        }
        dp = (const double *)dpp;
    }
    // the result record goes straight to the pinned host buffer, mapped into
    // the device's address space: no separate copy back
    void *mapped = nullptr;
    if (cudaHostGetDevicePointer(&mapped, W->h_pinned, 0) != cudaSuccess) {
        cudaGetLastError();
        mapped = nullptr;
    }
    CK(cudaEventRecord(W->ev0, s));
    ST(run_plan(P, W, C, dp, 0.0, (SgOutDev *)mapped, s));
    CK(cudaEventRecord(W->ev1, s));
    if (!mapped) CK(cudaMemcpyAsync(W->h_pinned, W->out.p, sizeof(SgOutDev), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, W->ev0, W->ev1);
    SgOutDev o;
    memcpy(&o, W->h_pinned, sizeof(o));
    fill_result(o, P, 0, ms, out);
    return SG_OK;
}

extern "C" sg_status sg_integrate_user(sg_rule rule, sg_integrand f, const double *params, int nparams,
                                       int params_on_device, int d, int q, void *stream, sg_result *out) {
    if (!rule || !out || nparams < 0 || (nparams > 0 && !params)) return SG_EINVAL;
    UserFold uf;
    int fdev = 0;
    if (!sg_integrand_kernel(f, &uf.kern, &uf.K, &fdev)) return SG_EINVAL;
    if (d < 1 || q < d) return SG_EINVAL;
    if (d > SG_MAX_D) return SG_ERANGE;
    if (q - d > SG_MAX_L || q - d + 1 > rule->max_level) return SG_ERANGE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SG_ECUDA;
    if (dev != rule->device || dev != fdev) return SG_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaGetLastError();
    DevCtx *C = nullptr;
    ST(dev_ctx(&C));
    Plan *P = nullptr;
    std::vector<Req> reqs(1);
    memset(reqs.data(), 0, sizeof(Req));
    reqs[0] = Req{rule, SG_FAM_USER, d, q - d, (int)SG_FORM_TELESCOPED, 0, 0};
    ST(get_plan(reqs, SG_PREC_FP64, &P));
    Workspace *W = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    ST(get_ws(s, &W));
    ST(ws_prepare(W, P, false, true, false, params_on_device ? 0 : std::max<size_t>(1, (size_t)nparams)));
    ST(ensure_host(W, sizeof(SgOutDev)));
    const double *dp = params;
    if (!params_on_device) {
        if (nparams > 0)
            CK(cudaMemcpyAsync(W->params.p, params, (size_t)nparams * sizeof(double), cudaMemcpyHostToDevice, s));
        dp = (const double *)W->params.p;
    }
    uf.params = dp;
    uf.d = d;
    CK(cudaEventRecord(W->ev0, s));
    ST(run_plan(P, W, C, dp, 0.0, nullptr, s, &uf));
    CK(cudaEventRecord(W->ev1, s));
    CK(cudaMemcpyAsync(W->h_pinned, W->out.p, sizeof(SgOutDev), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, W->ev0, W->ev1);
    fill_result(*(SgOutDev *)W->h_pinned, P, 0, ms, out);
    return SG_OK;
}

static sg_status batch_reqs(const sg_item *items, int n, sg_precision prec, std::vector<Req> &reqs,
                            size_t *pool) {
    if (!items || n < 1) return SG_EINVAL;
    if (n > 65536) return SG_ERANGE;
    reqs.resize(n);
    memset(reqs.data(), 0, sizeof(Req) * n);
    size_t need = 0;
    for (int k = 0; k < n; k++) {
        sg_form f = SG_FORM_AUTO;
        ST(check_one(items[k].rule, items[k].fam, items[k].d, items[k].q, prec, &f));
        reqs[k] = Req{items[k].rule, (int)items[k].fam, items[k].d, items[k].q - items[k].d, (int)f,
                      (long long)items[k].param_offset, 0};
        need = std::max(need, (size_t)items[k].param_offset + 2 * (size_t)items[k].d);
    }
    *pool = need;
    return SG_OK;
}

extern "C" sg_status sg_integrate_batch(const sg_item *items, int n, const double *params_pool,
                                        int params_on_device, sg_precision prec, double guard_tol,
                                        void *stream, sg_result *out) {
    if (!params_pool || !out) return SG_EINVAL;
    if (!prec_ok(prec)) return SG_EINVAL;
    if (!(guard_tol >= 0.0)) return SG_EINVAL;
    if (prec != SG_PREC_MIXED) guard_tol = 0.0;
    std::vector<Req> reqs;
    size_t pool = 0;
    ST(batch_reqs(items, n, prec, reqs, &pool));
    std::lock_guard<std::mutex> lk(g_mu);
    cudaGetLastError();  // a failed earlier call must not surface here
    for (int k = 0; k < n; k++) reqs[k].ppc = class_ppc(items[k], prec);
    DevCtx *C = nullptr;
    ST(dev_ctx(&C));
    Plan *P = nullptr;
    ST(get_plan(reqs, prec, &P));
    Workspace *W = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    ST(get_ws(s, &W));
    const bool guard = prec == SG_PREC_MIXED && guard_tol > 0.0;
    ST(ws_prepare(W, P, prec == SG_PREC_MIXED, prec == SG_PREC_FP64 || guard, prec == SG_PREC_FF || guard,
                  params_on_device ? 0 : pool));
    ST(ensure_host(W, (size_t)P->nout * sizeof(SgOutDev)));
    // graphs run on the workspace's own stream, ordered after the caller's work
    cudaStream_t g = W->own;
    CK(cudaEventRecord(W->ev_join, s));
    CK(cudaStreamWaitEvent(g, W->ev_join, 0));
    const double *dp = params_pool;
    if (!params_on_device) {
        CK(cudaMemcpyAsync(W->params.p, params_pool, pool * sizeof(double), cudaMemcpyHostToDevice, g));
        dp = (const double *)W->params.p;
    }
    // the launch sequence is captured once per (plan, params, guard) and replayed
    auto key = std::make_tuple(P->id, dp, guard_tol, W->epoch);
    auto it = W->graphs.find(key);
    if (it == W->graphs.end()) {
        GraphEntry ge;
        CK(cudaStreamBeginCapture(g, cudaStreamCaptureModeThreadLocal));
        sg_status st = run_plan(P, W, C, dp, guard_tol, nullptr, g, nullptr, false);
        cudaError_t ce = cudaStreamEndCapture(g, &ge.g);
        if (st != SG_OK) {
            if (ge.g) cudaGraphDestroy(ge.g);
            cudaGetLastError();
            return st;
        }
        if (ce != cudaSuccess) return SG_ECUDA;
        if (cudaGraphInstantiate(&ge.x, ge.g, 0) != cudaSuccess) {
            cudaGraphDestroy(ge.g);
            cudaGetLastError();
            return SG_ECUDA;
        }
        it = W->graphs.emplace(key, ge).first;
    }
    CK(cudaEventRecord(W->ev0, g));
    CK(cudaGraphLaunch(it->second.x, g));
    CK(cudaEventRecord(W->ev1, g));
    CK(cudaMemcpyAsync(W->h_pinned, W->out.p, (size_t)n * sizeof(SgOutDev), cudaMemcpyDeviceToHost, g));
    CK(cudaStreamSynchronize(g));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, W->ev0, W->ev1);
    const SgOutDev *o = (const SgOutDev *)W->h_pinned;
    for (int k = 0; k < n; k++) fill_result(o[k], P, k, ms, out + k);
    return SG_OK;
}

extern "C" sg_status sg_integrate_grad(sg_rule rule, sg_family fam, const double *params,
                                       int params_on_device, int d, int q, sg_precision prec,
                                       void *stream, sg_result *out, double *dparams,
                                       int dparams_on_device) {
    if (!params || !out || !dparams) return SG_EINVAL;
    sg_form form = SG_FORM_TELESCOPED;  // the adjoint items follow the telescoped form
    ST(check_one(rule, fam, d, q, prec, &form));
    std::lock_guard<std::mutex> lk(g_mu);
    cudaGetLastError();  // a failed earlier call must not surface here
    DevCtx *C = nullptr;
    ST(dev_ctx(&C));
    Plan *P = nullptr;
    std::vector<Req> reqs(1);
    memset(reqs.data(), 0, sizeof(Req));
    reqs[0] = Req{rule, (int)fam, d, q - d, (int)form, 0, 1};
    ST(get_plan(reqs, prec, &P));
    Workspace *W = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    ST(get_ws(s, &W));
    ST(ws_prepare(W, P, prec == SG_PREC_MIXED, prec == SG_PREC_FP64, prec == SG_PREC_FF,
                  params_on_device ? 0 : 2 * (size_t)d));
    ST(ensure_host(W, sizeof(SgOutDev) + 2 * (size_t)d * sizeof(double)));
    const double *dp = params;
    if (!params_on_device) {
        CK(cudaMemcpyAsync(W->params.p, params, 2 * (size_t)d * sizeof(double), cudaMemcpyHostToDevice, s));
        dp = (const double *)W->params.p;
    }
    CK(cudaEventRecord(W->ev0, s));
    ST(run_plan(P, W, C, dp, 0.0, nullptr, s));
    SgGradArgs ga;
    ga.fam = (int)fam;
    ga.d = d;
    ga.L = q - d;
    ga.params = dp;
    ga.delta_xw = rule->d_xw;
    ga.delta_off = P->d_delta_off;
    ga.delta_m = P->d_delta_m;
    ga.v = (const double *)W->vout.p;
    ga.vstride = P->vstride;
    ga.q = (const SgOutDev *)W->out.p;
    ga.qh = fam == SG_FAM_OSCILLATORY ? (const SgOutDev *)W->out.p + 1 : nullptr;
    ga.base = (const SgBaseDev *)W->bases.p;
    ga.grad_rel = (double *)W->grad.p;
    CK(sg_launch_grad(ga, s));
    CK(cudaEventRecord(W->ev1, s));
    CK(cudaMemcpyAsync(W->h_pinned, W->out.p, sizeof(SgOutDev), cudaMemcpyDeviceToHost, s));
    double *hg = (double *)((char *)W->h_pinned + sizeof(SgOutDev));
    CK(cudaMemcpyAsync(hg, W->grad.p, 2 * (size_t)d * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, W->ev0, W->ev1);
    const SgOutDev o = *(const SgOutDev *)W->h_pinned;
    // dQ/dtheta = scale * grad_rel, scale = Q / (base + T)
    for (int j = 0; j < 2 * d; j++) {
        double v = hg[j];
        if (fam != SG_FAM_OSCILLATORY) {
            int e = 0;
            const double m = frexp(v * o.mant / o.sum, &e);
            v = ldexp(m, e + (int)o.exp2);
        }
        hg[j] = v;
    }
    if (dparams_on_device) {
        CK(cudaMemcpyAsync(dparams, hg, 2 * (size_t)d * sizeof(double), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    } else {
        memcpy(dparams, hg, 2 * (size_t)d * sizeof(double));
    }
    fill_result(o, P, 0, ms, out);
    out->evals = P->total_evals;
    return SG_OK;
}

extern "C" sg_status sg_autotune(const sg_item *items, int n, const double *params_pool,
                                 int params_on_device, sg_precision prec, int reps, void *stream,
                                 sg_tuning *best, double *best_ms) {
    if (!best || reps < 1) return SG_EINVAL;
    if (!prec_ok(prec)) return SG_EINVAL;
    sg_tuning saved;
    ST(sg_get_tuning(prec, &saved));
    const int ppc[] = {2048, 8192, 32768, 131072};
    const int cps[] = {4, 8, 16};
    const int wpc[] = {4, 8};
    std::vector<sg_result> res(n);
    double best_t = 1e300;
    sg_tuning bt = saved;
    for (int a : ppc)
        for (int b : cps)
            for (int c : wpc) {
                sg_tuning t{a, b, c};
                ST(sg_set_tuning(prec, &t));
                std::vector<double> ts;
                for (int r = 0; r < reps + 1; r++) {
                    sg_status st = sg_integrate_batch(items, n, params_pool, params_on_device, prec, 0.0,
                                                      stream, res.data());
                    if (st != SG_OK) {
                        sg_set_tuning(prec, &saved);
                        return st;
                    }
                    if (r) ts.push_back(res[0].seconds);
                }
                std::sort(ts.begin(), ts.end());
                const double med = ts[ts.size() / 2];
                if (med < best_t) {
                    best_t = med;
                    bt = t;
                }
            }
    ST(sg_set_tuning(prec, &bt));
    *best = bt;
    if (best_ms) *best_ms = best_t * 1e3;
    return SG_OK;
}

extern "C" sg_status sg_profile_begin(void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    Workspace *W = nullptr;
    ST(get_ws((cudaStream_t)stream, &W));
    W->profiling = true;
    W->prof_used = 0;
    return SG_OK;
}

extern "C" sg_status sg_profile_end(void *stream, double *fold_ms, int *launches) {
    if (!fold_ms || !launches) return SG_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    Workspace *W = nullptr;
    ST(get_ws((cudaStream_t)stream, &W));
    CK(cudaStreamSynchronize(W->stream));
    double tot = 0.0;
    for (size_t i = 0; i < W->prof_used; i++) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, W->prof[i].first, W->prof[i].second));
        tot += ms;
    }
    *fold_ms = tot;
    *launches = (int)W->prof_used;
    W->profiling = false;
    W->prof_used = 0;
    return SG_OK;
}

extern "C" sg_status sg_ceiling(sg_precision prec, int kind, void *stream, double *rate) {
    if (!rate || !prec_ok(prec) || kind < 0 || kind > 2)
        return SG_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaGetLastError();  // a failed earlier call must not surface here
    DevCtx *C = nullptr;
    ST(dev_ctx(&C));
    Workspace *W = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    ST(get_ws(s, &W));
    ST(ensure(W, W->grad, (size_t)C->sms * 8 * 256 * sizeof(double)));
    double work = sg_launch_ceiling(prec, kind, C->sms, (double *)W->grad.p, s);  // warm-up
    CK(cudaGetLastError());
    float best = 1e30f;
    for (int r = 0; r < 3; r++) {
        CK(cudaEventRecord(W->ev0, s));
        work = sg_launch_ceiling(prec, kind, C->sms, (double *)W->grad.p, s);
        CK(cudaEventRecord(W->ev1, s));
        CK(cudaEventSynchronize(W->ev1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, W->ev0, W->ev1));
        if (ms < best) best = ms;
    }
    *rate = work / (best * 1e-3);
    return SG_OK;
}

extern "C" sg_status sg_eval_functions(int kind, sg_precision prec, const double *d_x, double *d_y, int n,
                                       void *stream) {
    if (!d_x || !d_y || n < 0 || kind < 0 || kind > 1) return SG_EINVAL;
    if (!prec_ok(prec)) return SG_EINVAL;
    cudaGetLastError();
    CK(sg_launch_fn(kind, prec, d_x, d_y, n, (cudaStream_t)stream));
    return SG_OK;
}

// ---------------------------------------------------------------------------
// per-class tuning of the batch path
// ---------------------------------------------------------------------------

static const int kClassCandidates[] = {1024, 4096, 16384, 65536, 262144};

static sg_status write_class_table(const char *path) {
    FILE *f = fopen(path, "w");
    if (!f) return SG_EINVAL;
    fprintf(f, "{\"classes\": [\n");
    size_t i = 0;
    for (auto &kv : g_class_ppc) {
        fprintf(f, "  {\"family\": %d, \"rule\": %d, \"dbucket\": %d, \"L\": %d, \"prec\": %d, "
                   "\"points_per_chunk\": %d}%s\n",
                std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first), std::get<3>(kv.first),
                std::get<4>(kv.first), kv.second, ++i < g_class_ppc.size() ? "," : "");
    }
    fprintf(f, "]}\n");
    return fclose(f) == 0 ? SG_OK : SG_EINVAL;
}

extern "C" sg_status sg_autotune_classes(const sg_item *items, int n, const double *params_pool,
                                         int params_on_device, sg_precision prec, int reps, void *stream,
                                         const char *path, int *nclasses) {
    if (!items || n < 1 || !params_pool || reps < 1 || !prec_ok(prec)) return SG_EINVAL;
    std::map<ClassKey, std::vector<sg_item>> groups;
    for (int k = 0; k < n; k++) {
        if (!items[k].rule) return SG_EINVAL;
        groups[class_key(items[k], prec)].push_back(items[k]);
    }
    std::vector<sg_result> res(n);
    for (auto &g : groups) {
        double best_t = 1e300;
        int best = 0;
        for (int ppc : kClassCandidates) {
            {
                std::lock_guard<std::mutex> lk(g_mu);
                g_class_ppc[g.first] = ppc;
            }
            std::vector<double> ts;
            for (int r = 0; r < reps + 1; r++) {
                const sg_status st = sg_integrate_batch(g.second.data(), (int)g.second.size(), params_pool,
                                                        params_on_device, prec, 0.0, stream, res.data());
                if (st == SG_ERANGE) break;  // too many chunks at this size
                if (st != SG_OK) {
                    std::lock_guard<std::mutex> lk(g_mu);
                    g_class_ppc.erase(g.first);
                    return st;
                }
                if (r) ts.push_back(res[0].seconds);
            }
            if (ts.empty()) continue;
            std::sort(ts.begin(), ts.end());
            if (ts[ts.size() / 2] < best_t) {
                best_t = ts[ts.size() / 2];
                best = ppc;
            }
        }
        std::lock_guard<std::mutex> lk(g_mu);
        if (best) g_class_ppc[g.first] = best;
        else g_class_ppc.erase(g.first);
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (nclasses) *nclasses = (int)g_class_ppc.size();
    return path ? write_class_table(path) : SG_OK;
}

// Reads the integer after "key": in s (a table line); false if absent.
static bool json_int(const char *s, const char *key, int *v) {
    char pat[64];
    snprintf(pat, sizeof(pat), "\"%s\":", key);
    const char *p = strstr(s, pat);
    if (!p) return false;
    return sscanf(p + strlen(pat), " %d", v) == 1;
}

extern "C" sg_status sg_tuning_load(const char *path, int *nclasses) {
    if (!path) return SG_EINVAL;
    FILE *f = fopen(path, "r");
    if (!f) return SG_EINVAL;
    std::map<ClassKey, int> table;
    char line[512];
    while (fgets(line, sizeof(line), f)) {
        int fam, rule, db, L, prec, ppc;
        if (!strchr(line, '{') || !json_int(line, "family", &fam)) continue;
        if (!json_int(line, "rule", &rule) || !json_int(line, "dbucket", &db) || !json_int(line, "L", &L) ||
            !json_int(line, "prec", &prec) || !json_int(line, "points_per_chunk", &ppc) || ppc < 32 ||
            !prec_ok(prec)) {
            fclose(f);
            return SG_EINVAL;
        }
        table[ClassKey(fam, rule, db, L, prec)] = ppc;
    }
    fclose(f);
    std::lock_guard<std::mutex> lk(g_mu);
    g_class_ppc = table;
    if (nclasses) *nclasses = (int)table.size();
    return SG_OK;
}

extern "C" sg_status sg_tuning_clear(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_class_ppc.clear();
    return SG_OK;
}

// ---------------------------------------------------------------------------
// sharded batches
// ---------------------------------------------------------------------------

extern "C" sg_status sg_integrate_batch_shard(const sg_item *items, int n, const double *params_pool,
                                              int params_on_device, sg_precision prec, int shard, int nshards,
                                              void *stream, long long *partials, sg_shard_info *info) {
    if (!params_pool || !partials || !prec_ok(prec)) return SG_EINVAL;
    if (nshards < 1 || nshards > 65536) return nshards < 1 ? SG_EINVAL : SG_ERANGE;
    if (shard < 0 || shard >= nshards) return SG_EINVAL;
    std::vector<Req> reqs;
    size_t pool = 0;
    ST(batch_reqs(items, n, prec, reqs, &pool));
    std::lock_guard<std::mutex> lk(g_mu);
    cudaGetLastError();  // a failed earlier call must not surface here
    for (int k = 0; k < n; k++) reqs[k].ppc = class_ppc(items[k], prec);
    DevCtx *C = nullptr;
    ST(dev_ctx(&C));
    Plan *P = nullptr;
    ST(get_plan(reqs, prec, &P));
    Workspace *W = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    ST(get_ws(s, &W));
    ST(ws_prepare(W, P, prec == SG_PREC_MIXED, prec == SG_PREC_FP64, prec == SG_PREC_FF,
                  params_on_device ? 0 : pool));
    const size_t nitems = P->items.size();
    const size_t lbytes = nitems * kItemLaccBytes;
    const size_t vbytes = nitems * sizeof(SgItemVar), bbytes = P->integrals.size() * sizeof(SgBaseDev);
    ST(ensure_host(W, lbytes + vbytes + bbytes));
    const double *dp = params_pool;
    if (!params_on_device) {
        CK(cudaMemcpyAsync(W->params.p, params_pool, pool * sizeof(double), cudaMemcpyHostToDevice, s));
        dp = (const double *)W->params.p;
    }
    // this shard's contiguous range of the plan's chunk queue (an empty range
    // starts at the end of the queue, where the kernel's first grab stops)
    ShardRange r;
    r.on = true;
    r.lo = (unsigned long long)((unsigned __int128)P->nchunks * (unsigned)shard / (unsigned)nshards);
    r.hi = (unsigned long long)((unsigned __int128)P->nchunks * (unsigned)(shard + 1) / (unsigned)nshards);
    if (r.lo == r.hi) r.lo = r.hi = P->nchunks;
    ST(run_plan(P, W, C, dp, 0.0, nullptr, s, nullptr, false, r));
    unsigned char *h = (unsigned char *)W->h_pinned;
    CK(cudaMemcpyAsync(h, W->ilacc.p, lbytes, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h + lbytes, W->vars.p, vbytes, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h + lbytes + vbytes, W->bases.p, bbytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const long long *L = (const long long *)h;
    const SgItemVar *V = (const SgItemVar *)(h + lbytes);
    const SgBaseDev *B = (const SgBaseDev *)(h + lbytes + vbytes);
    for (size_t q = 0; q < nitems; q++) {
        const int g = P->item_integral[q];  // forward items only: the item of input g
        if (g < 0 || P->roles[q].role != SG_ROLE_FORWARD) continue;
        memcpy(partials + (size_t)g * SG_SHARD_LIMBS, L + q * SG_SHARD_LIMBS, SG_SHARD_LIMBS * sizeof(long long));
        if (info) {
            sg_shard_info &I = info[g];
            I.mult = V[q].mult;
            I.base_rel = V[q].base_rel;
            I.scale_m = B[g].scale_m;
            I.scale_e2 = B[g].scale_e2;
            I.unit_roundoff = unit_roundoff(prec);
            I.points = P->points[g];
            I.evals = P->evals[g];
        }
    }
    return SG_OK;
}
