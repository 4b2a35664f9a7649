// sg_integrate_noalloc: one integral with no memory allocation at all.
//
// Who needs this: code that must not call cudaMalloc (or any allocator) at
// the point where it integrates - for example a host thread inside a
// latency-critical loop, where cudaMalloc/cudaFree would synchronise the
// device and stall other streams, or an embedding runtime that owns all
// device memory itself and forbids libraries from allocating behind its
// back.  Such callers pass device inputs and outputs only.
//
// All device scratch of this entry point (the per-direction tables, the
// per-chunk and per-group slots, tickets, the plan and rule nodes, and the
// binomial table used for unranking) lives in one file-scope
// `static __device__` array of fixed size (kNaBytes, about 5.2 MB), which
// every GPU that loads this library holds until the process exits.  Host
// planning uses only the stack; the 1-D rules are computed into stack
// arrays.  The kernels are the library's regular setup / prep / fold
// kernels, handed pointers into the static array.
//
// Set-up: the first call on a device (with that device current) looks up the
// array's device address with cudaGetSymbolAddress and copies the binomial
// table into it with a synchronous cudaMemcpy; make that first call before
// any stream capture.  After that a call copies nothing from host memory:
// its plan (rule nodes, pattern records) travels as the parameter block of
// a one-CTA upload kernel, which writes it into the array and clears the
// tickets in stream order, so the host stack that held the plan may be gone
// by the time the kernel runs.  Every call shares the one array and leaves
// its contents behind.  Calls whose work overlaps on the GPU (different
// streams, or different host threads) race on the array: serialise them.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "../../include/sg.h"
#include "sg_kernels.h"
#include "sg_rules.h"

namespace {

// Limits of the no-allocation path.
constexpr int kNaMaxD = 1024;           // directions
constexpr int kNaMaxL = 6;              // q - d
constexpr long long kNaMaxEntries = 1 << 17;   // (phi, w) table entries
constexpr unsigned long long kNaMaxChunks = 1 << 16;
constexpr int kNaMaxPats = 64;          // 2^(L-1) telescoped patterns for L <= 6 (plus slack)
constexpr int kNaMaxBlocks = 2 * kNaMaxL;
constexpr int kNaMaxNodes = 512;        // rule-block nodes over all blocks
constexpr unsigned long long kNaMaxGroups = kNaMaxChunks / SG_GROUP + kNaMaxPats + 1;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffBinom = 0;
constexpr size_t kOffXw = align256(kOffBinom + sizeof(unsigned long long) * SG_BINOM_K * (SG_MAX_D + 1));
constexpr size_t kOffInt = align256(kOffXw + sizeof(double2) * kNaMaxNodes);
constexpr size_t kOffBlk = align256(kOffInt + sizeof(SgIntegralDev));
constexpr size_t kOffBe = align256(kOffBlk + sizeof(SgBlockDev) * kNaMaxBlocks);
constexpr size_t kOffItem = align256(kOffBe + sizeof(long long) * kNaMaxBlocks);
constexpr size_t kOffRole = align256(kOffItem + sizeof(SgItemDev));
constexpr size_t kOffII = align256(kOffRole + sizeof(SgItemRole));
constexpr size_t kOffPat = align256(kOffII + sizeof(int));
constexpr size_t kOffPc = align256(kOffPat + sizeof(SgPatDev) * kNaMaxPats);
constexpr size_t kOffTab = align256(kOffPc + sizeof(unsigned long long) * kNaMaxPats);
constexpr size_t kOffSlots = align256(kOffTab + sizeof(double2) * kNaMaxEntries);
constexpr size_t kOffGslots = align256(kOffSlots + sizeof(SgSlot) * kNaMaxChunks);
constexpr size_t kOffCnt = align256(kOffGslots + sizeof(SgGroupSlot) * kNaMaxGroups);
constexpr size_t kCntBytes = 16 + 4 * (1 + kNaMaxGroups);
constexpr size_t kOffBase = align256(kOffCnt + kCntBytes);
constexpr size_t kOffVar = align256(kOffBase + sizeof(SgBaseDev));
constexpr size_t kOffFlag = align256(kOffVar + sizeof(SgItemVar));
constexpr size_t kOffVout = align256(kOffFlag + sizeof(int));
constexpr size_t kNaBytes = align256(kOffVout + sizeof(double));

}  // namespace

// The scratch of every sg_integrate_noalloc call on this device.
static __device__ __align__(256) unsigned char g_sg_noalloc_scratch[kNaBytes];

namespace {

struct NaDevice {
    bool ready = false;
    unsigned char *scratch = nullptr;  // device address of g_sg_noalloc_scratch
    int sms = 0;
    int occ[2] = {0, 0};               // resident fold CTAs per SM (FP64, mixed)
};
constexpr int kNaMaxDevices = 64;
NaDevice g_na_dev[kNaMaxDevices];
std::mutex g_na_mu;
unsigned long long g_na_binom[SG_BINOM_K * (SG_MAX_D + 1)];  // host copy, static storage
bool g_na_binom_ready = false;
constexpr int kNaWarps = 8;

// Once per device, with that device current: resolve the array's device
// address (a host-side name of a __device__ array is not a device pointer)
// and upload the binomial table.
sg_status na_setup(int dev, NaDevice **out) {
    NaDevice &D = g_na_dev[dev];
    if (!D.ready) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_sg_noalloc_scratch) != cudaSuccess || !p) return SG_ECUDA;
        if (!g_na_binom_ready) {
            sg_fill_binomials(g_na_binom);
            g_na_binom_ready = true;
        }
        if (cudaMemcpy((unsigned char *)p + kOffBinom, g_na_binom, sizeof(g_na_binom),
                       cudaMemcpyHostToDevice) != cudaSuccess)
            return SG_ECUDA;
        if (cudaDeviceGetAttribute(&D.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return SG_ECUDA;
        D.occ[0] = sg_fold_occupancy(0, 0, kNaWarps);
        D.occ[1] = sg_fold_occupancy(1, 0, kNaWarps);
        if (cudaGetLastError() != cudaSuccess) return SG_ECUDA;
        D.scratch = (unsigned char *)p;
        D.ready = true;
    }
    *out = &D;
    return SG_OK;
}

// Host plan of one integral in the telescoped form, on the stack.  It is
// passed by value as the upload kernel's parameter block (below the 32 KB
// limit of kernel parameters).
struct NaPlan {
    double2 xw[kNaMaxNodes];
    int nxw = 0;
    SgIntegralDev integral;
    SgBlockDev blocks[kNaMaxBlocks];
    long long block_end[kNaMaxBlocks];
    int blk_m[kNaMaxBlocks];
    long long blk_off[kNaMaxBlocks];
    int nblocks = 0;
    SgItemDev item;
    SgItemRole role;
    int item_integral = 0;
    SgPatDev pats[kNaMaxPats];
    unsigned long long pat_chunk0[kNaMaxPats];
    int npat = 0;
    long long nentries = 0;
    unsigned long long nchunks = 0;
};

// Rule block nodes on [0,1]: the difference rule J^{k+1} - J^k on the union
// of both node sets (delta = true), or the telescoped last-direction rule
// J^{k+1} - J^1.  Returns the node count, 0 when the arrays are too small.
int na_block(int kind, bool delta, int k, double2 *xw, int cap) {
    double x1[(1 << kNaMaxL) + 1], w1[(1 << kNaMaxL) + 1];
    double x0[(1 << kNaMaxL) + 1], w0[(1 << kNaMaxL) + 1];
    const int n1 = sg_rule_level(kind, k + 1, x1, w1);
    if (n1 <= 0) return 0;
    int n = 0;
    if (!delta) {
        bool centre = false;
        if (n1 + 1 > cap) return 0;
        for (int j = 0; j < n1; j++) {
            double w = w1[j];
            if (x1[j] == 0.5) {
                w -= 1.0;
                centre = true;
            }
            xw[n++] = make_double2(x1[j], w);
        }
        if (!centre) xw[n++] = make_double2(0.5, -1.0);
        return n;
    }
    const int n0 = sg_rule_level(kind, k, x0, w0);
    if (kind == SG_RULE_GAUSS_LEGENDRE) {
        if (n1 + n0 > cap) return 0;
        for (int j = 0; j < n1; j++) xw[n++] = make_double2(x1[j], w1[j]);
        for (int j = 0; j < n0; j++) xw[n++] = make_double2(x0[j], -w0[j]);
        return n;
    }
    if (n1 > cap) return 0;
    for (int j = 0; j < n1; j++) xw[j] = make_double2(x1[j], w1[j]);
    // nested: node j of level k is node 2j of level k+1 (trapezoid, Clenshaw-
    // Curtis) or node 2j + 1 (Gauss-Patterson)
    const int shift = kind == SG_RULE_GAUSS_PATTERSON ? 1 : 0;
    if (n0 == 1) xw[n1 / 2].y -= w0[0];
    else
        for (int j = 0; j < n0; j++) xw[2 * j + shift].y -= w0[j];
    return n1;
}

unsigned long long na_binom(int n, int k) {
    if (n < 0 || k < 0 || k > n) return 0;
    return g_na_binom[(size_t)k * (SG_MAX_D + 1) + n];
}

// Telescoped patterns of (d, L) with their chunking.  Block ids: DELTA k at
// k-1 (k = 1..L-1), TAIL M at L-1 + M-1 (M = 1..L).
sg_status na_plan(int kind, int fam, int d, int L, int prec, long long resident_warps,
                  const double2 *dev_xw, NaPlan &P) {
    // blocks and table layout
    long long cur = 0;
    for (int b = 0; b < 2 * L - 1; b++) {
        const bool delta = b < L - 1;
        const int k = delta ? b + 1 : b - (L - 1) + 1;
        const int m = na_block(kind, delta, k, P.xw + P.nxw, kNaMaxNodes - P.nxw);
        if (m == 0) return SG_ERANGE;
        P.blocks[b].off = cur;
        P.blocks[b].m = m;
        P.blocks[b].integral = 0;
        P.blocks[b].xw = dev_xw + P.nxw;
        P.blk_m[b] = m;
        P.blk_off[b] = cur;
        P.nxw += m;
        cur += (long long)d * m;
        P.block_end[b] = cur;
    }
    P.nblocks = 2 * L - 1;
    P.nentries = cur;
    if (P.nentries > kNaMaxEntries) return SG_ERANGE;
    if (L == 0) {  // keep one placeholder block so the setup kernel has a valid list
        memset(&P.blocks[0], 0, sizeof(SgBlockDev));
        P.blocks[0].m = 1;
        P.blocks[0].xw = dev_xw;
        P.block_end[0] = 0;
        P.nblocks = 1;
    }
    // patterns: prefix compositions of KP <= L-1 into rp parts (cut points
    // as bit masks), tail TAIL(L - KP)
    struct Spec {
        int r, pre[kNaMaxL];
        int tail;
    } spec[kNaMaxPats];
    int ns = 0;
    for (int KP = 0; KP <= L - 1; KP++) {
        const int tail = (L - 1) + (L - KP) - 1;
        if (KP == 0) {
            spec[ns].r = 1;
            spec[ns].tail = tail;
            ns++;
            continue;
        }
        for (unsigned mask = 0; mask < (1u << (KP - 1)); mask++) {
            const int rp = __builtin_popcount(mask) + 1;
            if (rp > d - 1) continue;
            if (ns >= kNaMaxPats) return SG_ERANGE;
            int part = 1, t = 0;
            for (int bit = 0; bit < KP - 1; bit++) {
                if (mask & (1u << bit)) {
                    spec[ns].pre[t++] = part - 1;  // DELTA(part) has block id part-1
                    part = 1;
                } else {
                    part++;
                }
            }
            spec[ns].pre[t++] = part - 1;
            spec[ns].r = rp + 1;
            spec[ns].tail = tail;
            ns++;
        }
    }
    // evaluations and chunk size
    unsigned long long total = 0, per[kNaMaxPats];
    for (int i = 0; i < ns; i++) {
        unsigned long long A = 1;
        for (int t = 0; t < spec[i].r - 1; t++) A *= (unsigned long long)P.blk_m[spec[i].pre[t]];
        per[i] = A * (unsigned long long)P.blk_m[spec[i].tail];
        total += na_binom(d, spec[i].r) * per[i];
    }
    unsigned long long target = total / (4 * (unsigned long long)(resident_warps > 0 ? resident_warps : 1)) + 1;
    const unsigned long long floor_evals = prec ? 2048 : 128;
    if (target < floor_evals) target = floor_evals;
    const unsigned long long min_target = total / (kNaMaxChunks - kNaMaxPats) + 1;
    if (target < min_target) target = min_target;
    unsigned long long chunk = 0;
    for (int i = 0; i < ns; i++) {
        const unsigned long long nsub = na_binom(d, spec[i].r);
        if (nsub == 0) continue;
        SgPatDev &pd = P.pats[P.npat];
        memset(&pd, 0, sizeof(pd));
        pd.woff = -1;  // weights are products of the block weights (not the merged form)
        pd.item = 0;
        pd.r = spec[i].r;
        unsigned long long A = 1;
        for (int t = 0; t < spec[i].r - 1; t++) {
            pd.pm[t] = P.blk_m[spec[i].pre[t]];
            pd.poff[t] = P.blk_off[spec[i].pre[t]];
            A *= (unsigned long long)pd.pm[t];
        }
        pd.A = (int)A;
        pd.tm = P.blk_m[spec[i].tail];
        pd.toff = P.blk_off[spec[i].tail];
        pd.coef = 1.0;
        pd.nsub = nsub;
        pd.chunk0 = chunk;
        if (per[i] > target && A > 1) {
            unsigned long long parts = (per[i] + target - 1) / target;
            if (parts > A) parts = A;
            pd.ablk = (int)((A + parts - 1) / parts);
            pd.asplit = (int)((A + pd.ablk - 1) / pd.ablk);
            pd.spc = 1;
            chunk += nsub * (unsigned long long)pd.asplit;
        } else {
            pd.asplit = 1;
            pd.ablk = (int)A;
            pd.spc = target / per[i] > 0 ? target / per[i] : 1;
            chunk += (nsub + pd.spc - 1) / pd.spc;
        }
        P.pat_chunk0[P.npat] = pd.chunk0;
        P.npat++;
    }
    if (chunk > kNaMaxChunks) return SG_ERANGE;
    P.nchunks = chunk;
    if (P.npat == 0) {
        memset(&P.pats[0], 0, sizeof(SgPatDev));
        P.pats[0].woff = -1;
        P.pat_chunk0[0] = ~0ull;
    }
    memset(&P.item, 0, sizeof(P.item));
    P.item.d = d;
    P.item.skip = -1;
    P.item.gk = fam == SG_FAM_OSCILLATORY ? SG_GK_OSC : SG_GK_EXPM1;
    P.item.out = 0;
    P.item.tab = 0;
    P.item.pat0 = 0;
    P.item.npat = P.npat;
    P.item.chunk0 = 0;
    P.item.nchunk = chunk;
    P.item.group0 = 0;
    P.item.ngroups = (chunk + SG_GROUP - 1) / SG_GROUP;
    memset(&P.role, 0, sizeof(P.role));
    P.role.role = SG_ROLE_FORWARD;
    P.role.integral = 0;
    P.role.dir = -1;
    P.integral.fam = fam;
    P.integral.d = d;
    P.integral.param_off = 0;
    P.integral.flag_item = -1;
    P.integral.pad = 0;
    P.item_integral = 0;
    return SG_OK;
}

static_assert(sizeof(NaPlan) <= 32000, "the plan must fit the kernel parameter block");

// Copies n bytes (a multiple of 4) with the CTA's threads.
__device__ __forceinline__ void na_copy(unsigned char *dst, const void *src, size_t n) {
    const unsigned *s4 = (const unsigned *)src;
    unsigned *d4 = (unsigned *)dst;
    for (size_t i = threadIdx.x; i < n / 4; i += blockDim.x) d4[i] = s4[i];
}

}  // namespace

// Writes a call's plan into the static array and clears the work counter and
// tickets.  One CTA; the plan arrives in the kernel's parameter block.
__global__ void __launch_bounds__(256) sg_na_upload_kernel(const NaPlan P, unsigned char *S) {
    na_copy(S + kOffXw, P.xw, sizeof(double2) * (P.nxw > 0 ? P.nxw : 1));
    na_copy(S + kOffInt, &P.integral, sizeof(SgIntegralDev));
    na_copy(S + kOffBlk, P.blocks, sizeof(SgBlockDev) * P.nblocks);
    na_copy(S + kOffBe, P.block_end, sizeof(long long) * P.nblocks);
    na_copy(S + kOffItem, &P.item, sizeof(SgItemDev));
    na_copy(S + kOffRole, &P.role, sizeof(SgItemRole));
    na_copy(S + kOffII, &P.item_integral, sizeof(int));
    const int npat = P.npat > 0 ? P.npat : 1;
    na_copy(S + kOffPat, P.pats, sizeof(SgPatDev) * npat);
    na_copy(S + kOffPc, P.pat_chunk0, sizeof(unsigned long long) * npat);
    unsigned *cnt = (unsigned *)(S + kOffCnt);
    for (size_t i = threadIdx.x; i < kCntBytes / 4; i += blockDim.x) cnt[i] = 0u;
}

extern "C" sg_status sg_integrate_noalloc(sg_rule_kind kind, sg_family fam, const double *d_params,
                                          int d, int q, sg_precision prec, void *stream,
                                          sg_dev_result *d_out) {
    if (!d_params || !d_out) return SG_EINVAL;
    if (kind != SG_RULE_TRAPEZOID && kind != SG_RULE_CLENSHAW_CURTIS && kind != SG_RULE_GAUSS_PATTERSON &&
        kind != SG_RULE_GAUSS_LEGENDRE)
        return SG_EINVAL;
    if ((int)fam < 0 || (int)fam > 4 || (prec != SG_PREC_FP64 && prec != SG_PREC_MIXED)) return SG_EINVAL;
    if (d < 1 || q < d) return SG_EINVAL;
    const int L = q - d;
    if (d > kNaMaxD || L > kNaMaxL) return SG_ERANGE;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return SG_ECUDA;
    std::lock_guard<std::mutex> lk(g_na_mu);
    NaDevice *D = nullptr;
    sg_status st = na_setup(dev, &D);
    if (st != SG_OK) return st;
    unsigned char *S = D->scratch;
    const int p = prec == SG_PREC_MIXED ? 1 : 0;
    const int per_sm = D->occ[p] < 8 ? (D->occ[p] > 0 ? D->occ[p] : 1) : 8;
    NaPlan P;
    st = na_plan(kind, fam, d, L, p, (long long)D->sms * per_sm * kNaWarps, (const double2 *)(S + kOffXw), P);
    if (st != SG_OK) return st;
    // plan, rule nodes and cleared tickets into the static array (stream-ordered)
#define NA_CK(call)                                     \
    do {                                                \
        if ((call) != cudaSuccess) return SG_ECUDA;     \
    } while (0)
    sg_na_upload_kernel<<<1, 256, 0, s>>>(P, S);
    NA_CK(cudaGetLastError());

    SgSetupArgs sa;
    memset(&sa, 0, sizeof(sa));
    sa.blocks = (const SgBlockDev *)(S + kOffBlk);
    sa.block_end = (const long long *)(S + kOffBe);
    sa.nblocks = P.nblocks;
    sa.nentries = P.nentries;
    sa.integrals = (const SgIntegralDev *)(S + kOffInt);
    sa.nintegrals = 1;
    sa.params = d_params;
    sa.tab32 = p ? (float2 *)(S + kOffTab) : nullptr;
    sa.tab64 = p ? nullptr : (double2 *)(S + kOffTab);
    sa.bases = (SgBaseDev *)(S + kOffBase);
    sa.flags = nullptr;
    NA_CK(sg_launch_setup(sa, s));
    const double u = p ? 5.9604644775390625e-07 : 1.1102230246251565e-16;  // as the other entry points
    SgPrepArgs pa;
    pa.roles = (const SgItemRole *)(S + kOffRole);
    pa.items = (const SgItemDev *)(S + kOffItem);
    pa.nitems = 1;
    pa.integrals = (const SgIntegralDev *)(S + kOffInt);
    pa.params = d_params;
    pa.bases = (const SgBaseDev *)(S + kOffBase);
    pa.item_integral = (const int *)(S + kOffII);
    pa.vars = (SgItemVar *)(S + kOffVar);
    pa.out = (SgOutDev *)d_out;
    pa.vout = (double *)(S + kOffVout);
    pa.flags = nullptr;
    pa.unit_roundoff = u;
    NA_CK(sg_launch_prep(pa, s));
    if (P.nchunks == 0) return SG_OK;
    SgFoldArgs fa;
    memset(&fa, 0, sizeof(fa));
    fa.items = (const SgItemDev *)(S + kOffItem);
    fa.vars = (const SgItemVar *)(S + kOffVar);
    fa.nitems = 1;
    fa.pats = (const SgPatDev *)(S + kOffPat);
    fa.pat_chunk0 = (const unsigned long long *)(S + kOffPc);
    fa.npat = P.npat;
    fa.nchunks = P.nchunks;
    fa.tab = S + kOffTab;
    fa.binom = (const unsigned long long *)(S + kOffBinom);
    fa.slots = (SgSlot *)(S + kOffSlots);
    fa.gslots = (SgGroupSlot *)(S + kOffGslots);
    fa.work = (unsigned long long *)(S + kOffCnt);
    fa.item_done = (unsigned int *)(S + kOffCnt + 16);
    fa.group_done = fa.item_done + 1;
    fa.bases = (const SgBaseDev *)(S + kOffBase);
    fa.item_integral = (const int *)(S + kOffII);
    fa.out = (SgOutDev *)d_out;
    fa.vout = (double *)(S + kOffVout);
    fa.flags = nullptr;
    fa.skip_unflagged = nullptr;
    fa.guard_tol = 0.0;
    fa.unit_roundoff = u;
    SgLaunchCfg cfg;
    cfg.warps_per_cta = kNaWarps;
    long long ctas = (long long)D->sms * per_sm;
    const long long need = (long long)((P.nchunks + kNaWarps - 1) / kNaWarps);
    if (need < ctas) ctas = need > 0 ? need : 1;
    cfg.ctas = (int)ctas;
    cfg.dependent = P.nchunks <= SG_DEPENDENT_LAUNCH_MAX_CHUNKS ? 1 : 0;
    NA_CK(sg_launch_fold(fa, p, 0, cfg, s));
#undef NA_CK
    return SG_OK;
}
