// Host planner of libsg (see sg_plan.h).
#include "sg_plan.h"
#include "sg_rules.h"
#include "sg_lacc.h"

#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>

unsigned __int128 binom128(long long n, int k) {
    if (k < 0 || n < k) return 0;
    unsigned __int128 r = 1;
    for (int i = 1; i <= k; i++) {
        r = r * (unsigned __int128)(n - k + i) / (unsigned __int128)i;
        if (r > ((unsigned __int128)1 << 120)) return (unsigned __int128)1 << 127;
    }
    return r;
}



void compositions(int K, int r, std::vector<int> &cur, std::vector<std::vector<int>> &out) {
    if (r == 0) {
        if (K == 0) out.push_back(cur);
        return;
    }
    for (int a = 1; a <= K - (r - 1); a++) {
        cur.push_back(a);
        compositions(K - a, r - 1, cur, out);
        cur.pop_back();
    }
}

// Pattern list of one Smolyak sum over d directions with excess budget L.
//  difference:  every composition (k_1..k_r) of K <= L; all blocks DELTA
//  telescoped:  prefix compositions of K_P <= L-1 with DELTA blocks; the
//               last direction folds TAIL(L - K_P) = J^{L-K_P+1} - J^1
//  combination: compositions of K in [max(1, L-d+1), L] with FULL blocks and
//               coefficient (-1)^(L-K) C(d-1, L-K) (Eq. 2.6; the all-centre
//               subgrid contributes no deviation)
void gen_patterns(int form, int d, int L, std::vector<PatSpec> &out) {
    out.clear();
    std::vector<int> cur;
    auto add = [&](const std::vector<int> &pre, int pre_bk, BlockRef tail, double coef) {
        PatSpec p;
        p.r = (int)pre.size() + 1;
        for (size_t t = 0; t < pre.size(); t++) p.pre[t] = BlockRef{pre_bk, pre[t]};
        p.tail = tail;
        p.coef = coef;
        out.push_back(p);
    };
    if (form == SG_FORM_TELESCOPED) {
        for (int KP = 0; KP <= L - 1; KP++) {
            BlockRef tail{SG_BLK_TAIL, L - KP};
            if (KP == 0) {
                add(std::vector<int>(), SG_BLK_DELTA, tail, 1.0);
                continue;
            }
            for (int rp = 1; rp <= std::min(KP, d - 1); rp++) {
                std::vector<std::vector<int>> comps;
                compositions(KP, rp, cur, comps);
                for (auto &c : comps) add(c, SG_BLK_DELTA, tail, 1.0);
            }
        }
        return;
    }
    if (form == SG_FORM_MERGED) {
        // every distinct point: compositions (e_1..e_r) of K <= L into the
        // excesses at which the point's active coordinates first appear;
        // blocks NEW(e), weights from merged_weights
        for (int K = 1; K <= L; K++)
            for (int r = 1; r <= std::min(K, d); r++) {
                std::vector<std::vector<int>> comps;
                compositions(K, r, cur, comps);
                for (auto &c : comps) {
                    std::vector<int> pre(c.begin(), c.end() - 1);
                    add(pre, SG_BLK_NEW, BlockRef{SG_BLK_NEW, c.back()}, 1.0);
                }
            }
        return;
    }
    int Klo = 1;
    if (form == SG_FORM_COMBINATION) Klo = std::max(1, L - d + 1);
    for (int K = Klo; K <= L; K++) {
        double coef = 1.0;
        if (form == SG_FORM_COMBINATION) {
            coef = (double)binom128(d - 1, L - K);
            if ((L - K) % 2) coef = -coef;
        }
        int bk = form == SG_FORM_COMBINATION ? SG_BLK_FULL : SG_BLK_DELTA;
        for (int r = 1; r <= std::min(K, d); r++) {
            std::vector<std::vector<int>> comps;
            compositions(K, r, cur, comps);
            for (auto &c : comps) {
                std::vector<int> pre(c.begin(), c.end() - 1);
                add(pre, bk, BlockRef{bk, c.back()}, coef);
            }
        }
    }
}



int tab_m(sg_rule rule, BlockRef b) { return (int)rule->x[b.bk][b.k].size(); }

// Patterns with an empty block (a difference rule between two levels that use
// the same member of a slowly growing rule) contribute nothing.
void drop_empty_patterns(sg_rule rule, std::vector<PatSpec> &specs) {
    specs.erase(std::remove_if(specs.begin(), specs.end(),
                               [&](const PatSpec &sp) {
                                   if (tab_m(rule, sp.tail) == 0) return true;
                                   for (int t = 0; t < sp.r - 1; t++)
                                       if (tab_m(rule, sp.pre[t]) == 0) return true;
                                   return false;
                               }),
                specs.end());
}

// ---- merged-form weights ----------------------------------------------------
//
// A point of the sparse grid has, in each direction i, a node nu_i that
// first appears at level h_i = e_i + 1 (the centre at level 1: e_i = 0).
// Collecting the difference-form terms (Eq. 2.9 read as tensor products of
// difference rules) of every subgrid k that contains it, its weight is
//   w = sum_{k >= e, |k| <= L} prod_i (w^{k_i + 1}(nu_i) - w^{k_i}(nu_i))
//     = sum_{t <= L} [z^t] prod_{i active} A_{nu_i}(z) * B(z)^(d - r),
// with A_nu(z) = sum_{k >= e} (w^{k+1}(nu) - w^k(nu)) z^k and B the same
// series of the centre (w^l(x): the level-l weight at node x, 0 where x is
// not a node of level l).  The weight depends on the active directions'
// nodes only, not on which directions they are, so one table per pattern
// (e_1..e_r) serves all C(d, r) subsets.  Everything is formed in
// double-double arithmetic (Dekker 1971) and rounded once per format.

namespace {

struct DD {
    double hi, lo;
};

DD dd_two_sum(double a, double b) {
    const double s = a + b, z = s - a;
    return DD{s, (a - (s - z)) + (b - z)};
}

DD dd_add(DD a, DD b) {
    DD s = dd_two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return dd_two_sum(s.hi, s.lo);
}

DD dd_mul(DD a, DD b) {
    const double p = a.hi * b.hi;
    const double e = std::fma(a.hi, b.hi, -p) + (a.hi * b.lo + a.lo * b.hi);
    return dd_two_sum(p, e);
}

typedef std::vector<DD> Poly;  // coefficients of z^0 .. z^L

Poly poly_mul(const Poly &a, const Poly &b, int L) {
    Poly c(L + 1, DD{0.0, 0.0});
    for (int i = 0; i <= L; i++) {
        if (a[i].hi == 0.0 && a[i].lo == 0.0) continue;
        for (int j = 0; i + j <= L; j++) c[i + j] = dd_add(c[i + j], dd_mul(a[i], b[j]));
    }
    return c;
}

// hi + lo as a 64-bit significand and exponent (SgW64): hi's 53 bits, then
// lo in units of 2^-11 of hi's last place, rounded to nearest
SgW64 w64(DD w) {
    SgW64 r;
    r.m = 0;
    r.e = 1;
    r.neg = 0;
    if (w.hi == 0.0) return r;
    unsigned long long b;
    memcpy(&b, &w.hi, sizeof(b));
    int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) return r;  // below the normal range: no merged weight is that small
    r.neg = (int)(b >> 63);
    unsigned long long m = ((b & 0xfffffffffffffull) | (1ull << 52)) << 11;
    const double lu = std::ldexp(r.neg ? -w.lo : w.lo, 1086 - e);  // |lu| <= 2^10
    m += (unsigned long long)(long long)std::llround(lu);
    if (!(m >> 63)) {
        m <<= 1;
        e -= 1;
    }
    r.m = m;
    r.e = e;
    return r;
}

// weight of node x in level l (0 for l = 0 or where x is not a node)
double level_weight(const std::vector<std::vector<double>> &lx, const std::vector<std::vector<double>> &lw,
                    int l, double x) {
    if (l < 1) return 0.0;
    const auto &X = lx[l];
    auto it = std::lower_bound(X.begin(), X.end(), x);
    return (it != X.end() && *it == x) ? lw[l][it - X.begin()] : 0.0;
}

}  // namespace

bool merged_weights(sg_rule rule, int d, int L, double factor, std::vector<PatSpec> &specs, Plan *P) {
    std::vector<std::vector<double>> lx(L + 2), lw(L + 2);
    for (int l = 1; l <= L + 1; l++) {
        const int n = sg_level_nodes(rule->kind, l);
        lx[l].resize(n);
        lw[l].resize(n);
        sg_rule_level(rule->kind, l, lx[l].data(), lw[l].data());
    }
    auto series = [&](double x, int e) {
        Poly a(L + 1, DD{0.0, 0.0});
        for (int k = e; k <= L; k++)
            a[k] = dd_two_sum(level_weight(lx, lw, k + 1, x), -level_weight(lx, lw, k, x));
        return a;
    };
    // B(z)^n for the n = d - r a pattern needs, cumulated: Bc_n[m] = sum_{j<=m} [z^j] B^n
    const Poly B = series(0.5, 0);
    std::map<int, Poly> bcum;
    for (auto &sp : specs) {
        const int n = d - sp.r;
        if (bcum.count(n)) continue;
        Poly acc(L + 1, DD{0.0, 0.0}), base = B;
        acc[0] = DD{1.0, 0.0};
        for (int e = n; e > 0; e >>= 1) {
            if (e & 1) acc = poly_mul(acc, base, L);
            if (e > 1) base = poly_mul(base, base, L);
        }
        for (int m = 1; m <= L; m++) acc[m] = dd_add(acc[m], acc[m - 1]);
        bcum[n] = acc;
    }
    // the nodes each excess adds, with their series
    std::vector<std::vector<Poly>> A(L + 1);
    for (int e = 1; e <= L; e++)
        for (double x : rule->x[SG_BLK_NEW][e]) A[e].push_back(series(x, e));
    for (auto &sp : specs) {
        int ex[SG_MAX_R];
        for (int t = 0; t < sp.r - 1; t++) ex[t] = sp.pre[t].k;
        ex[sp.r - 1] = sp.tail.k;
        int K = 0;
        size_t cnt = 1;
        for (int t = 0; t < sp.r; t++) {
            K += ex[t];
            cnt *= A[ex[t]].size();
        }
        if (P->wt64.size() + cnt > ((size_t)1 << 24)) return false;
        sp.woff = (long long)P->wt64.size();
        const Poly &bc = bcum[d - sp.r];
        // depth-first over the node tuple, the last position fastest, with the
        // partial products kept per depth
        std::vector<Poly> part(sp.r + 1);
        part[0] = Poly(L + 1, DD{0.0, 0.0});
        part[0][0] = DD{1.0, 0.0};
        std::vector<int> idx(sp.r, 0);
        int t = 0;
        for (;;) {
            if (t == sp.r) {
                DD w = {0.0, 0.0};
                for (int s = K; s <= L; s++) w = dd_add(w, dd_mul(part[sp.r][s], bc[L - s]));
                w.hi *= factor;
                w.lo *= factor;
                P->wt64.push_back(w64(w));
                const float hf = (float)w.hi;
                P->wtff.push_back(make_float2(hf, (float)((w.hi - (double)hf) + w.lo)));
                t--;
                while (t >= 0 && ++idx[t] == (int)A[ex[t]].size()) idx[t--] = 0;
                if (t < 0) break;
            }
            part[t + 1] = poly_mul(part[t], A[ex[t]][idx[t]], L);
            t++;
        }
    }
    return true;
}

// n_d^q of Eq. 2.6: sum over the combination-form multi-indices of
// prod n_{l_i}, as a polynomial in the excess, direction by direction.
bool count_points(int kind, int d, int L, u64 *out) {
    std::vector<unsigned __int128> c(L + 1, 0), nc(L + 1);
    c[0] = 1;
    for (int i = 0; i < d; i++) {
        std::fill(nc.begin(), nc.end(), 0);
        for (int K = 0; K <= L; K++)
            for (int k = 0; K + k <= L; k++) nc[K + k] += c[K] * (unsigned __int128)sg_level_nodes(kind, k + 1);
        for (int K = 0; K <= L; K++) {
            c[K] = nc[K];
            if (c[K] > ((unsigned __int128)1 << 100)) return false;
        }
    }
    unsigned __int128 t = 0;
    for (int K = std::max(0, L - d + 1); K <= L; K++) t += c[K];
    if (t > (unsigned __int128)~0ull) return false;
    *out = (u64)t;
    return true;
}

// Run-aware chunks.  The fold walks a chunk's subsets in runs that share
// their first r - 1 directions (the last direction takes every value after
// the prefix's last one), and every run costs at least one warp pass of 32
// lanes plus its prefix fold, however few points it has.  Where runs are
// short (d small against r, or the ends of each prefix's stretch) a chunk
// sized by points alone can hold a dozen runs and take several times as
// long as its neighbours, and in a single integral, whose chunks are about
// one per resident warp, the slowest chunk sets the time.  So for single
// integrals the runs are walked here, on the host, the chunks are sized by
// the lane slots they occupy (passes x 32 plus a prefix fold per run and
// prefix block), and runs are cut between subsets where needed.

// Lane slots of k subsets of one run of a pattern with A prefix tuples and
// tm tail nodes (k * tm tail entries per prefix tuple), with `run` slots for
// the fixed work of a run and prefix block (its prefix fold and the loads
// of new table rows, a few memory latencies whatever the points).
static u64 run_slots(u64 A, u64 tm, u64 k, u64 run) {
    u64 c = 0;
    for (u64 b = 0; b * SG_APAD < A; b++) {
        const u64 At = std::min<u64>(SG_APAD, A - b * SG_APAD);
        c += 32 * ((At * k * tm + 31) / 32) + run;
    }
    return c;
}

// The fixed work of a run in lane slots, by precision: measured on GB300 as
// about 0.3 of an FP64 pass (1.1 - 1.6 us per pass of 32 points), 3 - 4
// float passes (0.4 - 0.5 us each) and 2 float-float passes; the latency of
// a run is the same, the passes it is set against differ.
static u64 run_cost_slots(int prec) { return prec == 0 ? 24 : (prec == 1 ? 112 : 64); }

// Calls fn(len) for the runs of the r-subsets of d directions in the
// fold's order: prefix tuples p_0 < .. < p_{r-2} <= d - 2 in lexicographic
// order, each followed by d - 1 - p_{r-2} subsets (r = 1: one run of d).
template <class F> static void for_each_run(int d, int r, F fn) {
    if (r == 1) {
        fn((u64)d);
        return;
    }
    std::vector<int> p(r - 1);
    for (int t = 0; t < r - 1; t++) p[t] = t;
    for (;;) {
        fn((u64)(d - 1 - p[r - 2]));
        int t = r - 2;
        while (t >= 0 && p[t] >= d - 2 - (r - 2 - t)) t--;
        if (t < 0) return;
        p[t]++;
        for (int u = t + 1; u < r - 1; u++) p[u] = p[u - 1] + 1;
    }
}

// Chunks of one pattern whose subsets need no splitting, each closed when
// its lane slots would pass `budget`; consecutive chunks of equal size share
// one record (the last chunk of a record may be smaller).  With P null the
// chunks are only counted.  Returns the number of chunks.
static u64 chunk_by_runs(const SgPatDev &pd, int d, u64 budget, u64 run, u64 &chunk, Plan *P) {
    const u64 A = (u64)pd.A, tm = (u64)pd.tm;
    std::vector<u64> sizes;  // subsets per chunk
    u64 cur = 0, cur_n = 0;
    auto close = [&]() {
        sizes.push_back(cur_n);
        cur = 0;
        cur_n = 0;
    };
    for_each_run(d, pd.r, [&](u64 m) {
        while (m > 0) {
            if (cur + run_slots(A, tm, m, run) <= budget) {
                cur += run_slots(A, tm, m, run);
                cur_n += m;
                return;
            }
            // the most subsets of this run that still fit (at least one in an empty chunk)
            u64 lo = 0, hi = m;
            while (lo < hi) {
                const u64 mid = (lo + hi + 1) / 2;
                if (cur + run_slots(A, tm, mid, run) <= budget) lo = mid;
                else hi = mid - 1;
            }
            if (lo == 0 && cur_n == 0) lo = 1;
            if (lo > 0) {
                cur += run_slots(A, tm, lo, run);
                cur_n += lo;
                m -= lo;
            }
            close();
        }
    });
    if (cur_n) close();
    if (!P) return sizes.size();
    u64 rank = 0;
    for (size_t i = 0; i < sizes.size();) {
        size_t j = i + 1;
        while (j < sizes.size() && sizes[j] == sizes[i]) j++;
        if (j < sizes.size() && sizes[j] < sizes[i]) j++;
        SgPatDev rec = pd;
        rec.rank0 = rank;
        for (size_t k = i; k < j; k++) rank += sizes[k];
        rec.nsub = rank;
        rec.chunk0 = chunk;
        rec.asplit = 1;
        rec.ablk = pd.A;
        rec.spc = sizes[i];
        chunk += j - i;
        P->pats.push_back(rec);
        P->pat_chunk0.push_back(rec.chunk0);
        i = j;
    }
    return sizes.size();
}

struct ItemBuild {
    SgItemDev it;
    SgItemRole role;
    int integral;   // -1 for adjoint sub-sums
    int L, form;
    std::vector<PatSpec> specs;
    u64 evals = 0;
};


void plan_free_host(Plan *P) { delete P; }

// Builds the items, table layout, patterns and chunks of a list of integrals.
sg_status build_plan_host(const std::vector<Req> &reqs, int prec, const sg_tuning &tune,
                          long long resident_warps, Plan **out) {
    Plan *P = new Plan();
    P->reqs = reqs;
    P->prec = prec;
    P->tune = tune;
    const int nint = (int)reqs.size();
    std::vector<ItemBuild> ib;
    std::vector<std::map<BlockRef, long long>> relmap(nint);  // block -> offset in the integral's table
    long long tab_cursor = 0, vcursor = 0;
    int shift_out = nint;
    for (int g = 0; g < nint; g++) {
        const Req &R = reqs[g];
        sg_rule rule = R.rule;
        u64 pts = 0;
        if (!count_points(rule->kind, R.d, R.L, &pts)) {
            plan_free_host(P);
            return SG_ERANGE;
        }
        P->points.push_back(pts);
        P->max_d = std::max(P->max_d, R.d);
        const int gk = R.fam == SG_FAM_OSCILLATORY ? SG_GK_OSC : SG_GK_EXPM1;
        const size_t first = ib.size();
        auto new_item = [&](int role, int dir, double x, int d_item, int skip, int L_item, int o) {
            ItemBuild b;
            memset(&b.it, 0, sizeof(b.it));
            b.it.d = d_item;
            b.it.skip = skip;
            b.it.gk = gk;
            b.it.out = o;
            b.it.tab = tab_cursor;
            b.role.role = role;
            b.role.integral = g;
            b.role.dir = dir;
            b.role.pad = 0;
            b.role.x = x;
            b.integral = role == SG_ROLE_ADJOINT ? -1 : g;
            b.L = L_item;
            b.form = R.form;
            gen_patterns(R.form, d_item, L_item, b.specs);
            drop_empty_patterns(rule, b.specs);
            // merged form: the point weights (with the factor -2 of the
            // oscillatory deviation, which the other forms fold into the
            // prefix weight)
            if (R.form == SG_FORM_MERGED &&
                !merged_weights(rule, d_item, L_item, gk == SG_GK_OSC ? -2.0 : 1.0, b.specs, P))
                return false;
            ib.push_back(b);
            return true;
        };
        if (!new_item(SG_ROLE_FORWARD, -1, 0.0, R.d, -1, R.L, g)) {
            plan_free_host(P);
            return SG_ERANGE;
        }
        if (R.grad) {
            if (R.fam == SG_FAM_OSCILLATORY)
                new_item(SG_ROLE_FORWARD_SHIFT, -1, 0.0, R.d, -1, R.L, shift_out++);
            int vstride = 0;
            P->delta_off.assign(R.L + 1, 0);
            P->delta_m.assign(R.L + 1, 0);
            for (int k = 1; k <= R.L; k++) {
                P->delta_off[k] = rule->off[SG_BLK_DELTA][k];
                P->delta_m[k] = (int)rule->x[SG_BLK_DELTA][k].size();
                vstride += P->delta_m[k];
            }
            P->vstride = vstride;
            for (int i = 0; i < R.d; i++) {
                int col = 0;
                for (int k = 1; k <= R.L; k++)
                    for (int j = 0; j < P->delta_m[k]; j++, col++)
                        new_item(SG_ROLE_ADJOINT, i, rule->x[SG_BLK_DELTA][k][j], R.d - 1, i, R.L - k,
                                 (int)(vcursor + (long long)i * vstride + col));
            }
            vcursor += (long long)R.d * vstride;
        }
        // table blocks: every block an item of this integral refers to
        std::vector<BlockRef> refs;
        for (size_t t = first; t < ib.size(); t++)
            for (auto &sp : ib[t].specs) {
                for (int q = 0; q < sp.r - 1; q++) refs.push_back(sp.pre[q]);
                refs.push_back(sp.tail);
            }
        std::sort(refs.begin(), refs.end());
        refs.erase(std::unique(refs.begin(), refs.end()), refs.end());
        long long cur = 0;
        for (auto &b : refs) {
            if (b.k < 1 || b.k >= rule->max_level) {
                plan_free_host(P);
                return SG_ERANGE;
            }
            const int m = tab_m(rule, b);
            relmap[g][b] = cur;
            SgBlockDev bd;
            bd.off = tab_cursor + cur;
            bd.m = m;
            bd.integral = g;
            bd.xw = rule->d_xw + rule->off[b.bk][b.k];
            P->blocks.push_back(bd);
            P->block_refs.push_back(b);
            cur += (long long)R.d * m;
            P->block_end.push_back(tab_cursor + cur);
        }
        SgIntegralDev G;
        G.fam = R.fam;
        G.d = R.d;
        G.param_off = R.param_off;
        G.flag_item = -1;
        G.pad = 0;
        P->integrals.push_back(G);
        for (size_t t = first; t < ib.size(); t++) {
            ItemBuild &b = ib[t];
            for (auto &sp : b.specs) {
                const unsigned __int128 ns = binom128(b.it.d, sp.r);
                if (ns > ((unsigned __int128)1 << 62)) {
                    plan_free_host(P);
                    return SG_ERANGE;
                }
                unsigned __int128 A = 1;
                for (int q = 0; q < sp.r - 1; q++) A *= (unsigned __int128)tab_m(rule, sp.pre[q]);
                const unsigned __int128 ev = ns * A * (unsigned __int128)tab_m(rule, sp.tail);
                if (A > (1u << 30) || ev > ((unsigned __int128)1 << 62)) {
                    plan_free_host(P);
                    return SG_ERANGE;
                }
                b.evals += (u64)ev;
            }
        }
        P->evals.push_back(ib[first].evals);
        tab_cursor += cur;
    }
    P->nentries = tab_cursor;
    P->nv = vcursor;
    P->nout = shift_out;
    // largest items first (longest-processing-time order of the work queue)
    std::vector<int> order(ib.size());
    for (size_t t = 0; t < ib.size(); t++) order[t] = (int)t;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return ib[x].evals > ib[y].evals; });
    u64 total = 0;
    for (auto &b : ib) total += b.evals;
    P->total_evals = total;
    // chunk size: several chunks per resident warp, but never so small that
    // the per-chunk work (unranking, prefix folds, one slot) dominates, never
    // above the tuned maximum, and at most 2^24 chunk slots
    const u64 warps = (u64)std::max<long long>(resident_warps, 1);
    // chunks per resident warp and the smallest chunk: a chunk's fixed work
    // (grab, prefix folds, reduction and ticket) is thousands of warp
    // cycles, so chunks are one (FP64, with 32 resident warps per SM) to
    // four (float) per warp; the guided tail below evens out the end of the
    // queue.  Values from sweeps on GB300 (cfg2/cfg3/cfg5 FP64, cfg3 float,
    // cfg2/cfg5 float-float).
    const u64 floor_evals = prec == 0 ? 32 : 1024;
    const u64 per_warp = prec == 1 ? 4 : (prec == 2 ? 2 : 1);
    u64 target = total / (per_warp * warps) + 1;
    if (target < floor_evals) target = floor_evals;
    if (target > (u64)tune.points_per_chunk) target = (u64)tune.points_per_chunk;
    const u64 max_chunks = 1ull << 24;
    if (total / target > max_chunks) target = total / max_chunks + 1;
    // guided tail: the last eighth of the queue gets chunks of a quarter of
    // the size, so that the warps drain it together instead of waiting for
    // a few full-size chunks grabbed last; but no tail chunk below four warp
    // passes, whose fixed work would outweigh their points
    const u64 tail_cut = total - total / 8;
    u64 tail_target = std::min<u64>(target, std::max<u64>(target / 4, 128));
    if (total / tail_target > max_chunks) tail_target = target;
    // single integrals (no class tuning, the chunk size set by the warp count
    // rather than the tuned maximum): run-aware chunks sized by lane slots,
    // about one per resident warp, for every pattern whose runs can be walked
    // within a budget of 2^22 runs per plan
    bool by_runs = target < (u64)tune.points_per_chunk;
    for (const Req &R : reqs) by_runs = by_runs && R.ppc == 0;
    std::vector<std::vector<char>> use_runs(ib.size());
    u64 slot_budget = 0;
    const u64 rc = run_cost_slots(prec);
    if (by_runs) {
        unsigned __int128 run_budget = (unsigned __int128)1 << 22;
        u64 slots = 0;
        auto pattern_shape = [&](const ItemBuild &b, const PatSpec &sp, SgPatDev &pd) {
            sg_rule rule = reqs[b.role.integral].rule;
            memset(&pd, 0, sizeof(pd));
            pd.r = sp.r;
            pd.A = 1;
            for (int t = 0; t < sp.r - 1; t++) pd.A *= tab_m(rule, sp.pre[t]);
            pd.tm = tab_m(rule, sp.tail);
        };
        for (size_t q = 0; q < order.size(); q++) {
            ItemBuild &b = ib[order[q]];
            use_runs[order[q]].assign(b.specs.size(), 0);
            for (size_t k = 0; k < b.specs.size(); k++) {
                const PatSpec &sp = b.specs[k];
                const u64 nsub = (u64)binom128(b.it.d, sp.r);
                if (nsub == 0) continue;
                SgPatDev pd;
                pattern_shape(b, sp, pd);
                const unsigned __int128 runs = sp.r == 1 ? 1 : binom128(b.it.d - 1, sp.r - 1);
                if (runs <= run_budget) {
                    run_budget -= runs;
                    use_runs[order[q]][k] = 1;
                    for_each_run(b.it.d, sp.r, [&](u64 m) { slots += run_slots((u64)pd.A, (u64)pd.tm, m, rc); });
                } else {
                    slots += nsub * (u64)pd.A * (u64)pd.tm;
                }
            }
        }
        // the smallest budget whose chunks (each pattern cut separately, each
        // chunk filled up to whole passes) number no more than the warps
        auto count = [&](u64 budget) {
            u64 n = 0;
            for (size_t q = 0; q < order.size(); q++) {
                ItemBuild &b = ib[order[q]];
                for (size_t k = 0; k < b.specs.size(); k++) {
                    if (!use_runs[order[q]][k]) continue;
                    SgPatDev pd;
                    pattern_shape(b, b.specs[k], pd);
                    if (run_slots((u64)pd.A, (u64)pd.tm, 1, rc) > budget) return ~0ull;
                    u64 none = 0;
                    n += chunk_by_runs(pd, b.it.d, budget, rc, none, nullptr);
                }
            }
            return n;
        };
        u64 lo = std::max<u64>(slots / warps + 1, 32 + rc), hi = lo;
        while (count(hi) > warps && hi < (1ull << 40)) hi *= 2;
        while (lo < hi) {  // the count does not grow with the budget
            const u64 mid = lo + (hi - lo) / 2;
            if (count(mid) <= warps) hi = mid;
            else lo = mid + 1;
        }
        slot_budget = lo;
    }
    u64 done = 0;
    u64 chunk = 0;
    for (size_t q = 0; q < order.size(); q++) {
        ItemBuild &b = ib[order[q]];
        const int g = b.role.integral;
        sg_rule rule = reqs[g].rule;
        // a chunk size tuned for this integral's class replaces the plan's
        const u64 item_target = reqs[g].ppc > 0 ? std::max<u64>((u64)reqs[g].ppc, 256) : target;
        const u64 item_tail = reqs[g].ppc > 0 ? std::max<u64>(item_target / 4, 64) : tail_target;
        b.it.pat0 = (long long)P->pats.size();
        b.it.chunk0 = chunk;
        for (size_t ks = 0; ks < b.specs.size(); ks++) {
            const PatSpec &sp = b.specs[ks];
            SgPatDev pd;
            memset(&pd, 0, sizeof(pd));
            pd.item = (int)q;
            pd.r = sp.r;
            pd.nsub = (u64)binom128(b.it.d, sp.r);
            if (pd.nsub == 0) continue;
            u64 A = 1;
            for (int t = 0; t < sp.r - 1; t++) {
                pd.pm[t] = tab_m(rule, sp.pre[t]);
                pd.poff[t] = relmap[g].at(sp.pre[t]);
                A *= (u64)pd.pm[t];
            }
            pd.A = (int)A;
            pd.tm = tab_m(rule, sp.tail);
            pd.toff = relmap[g].at(sp.tail);
            pd.coef = sp.coef;
            pd.woff = sp.woff;
            const u64 per_sub = A * (u64)pd.tm;
            const u64 nsub = pd.nsub;
            // one record for subsets [r0, r1) with chunk target tgt
            auto emit = [&](u64 r0, u64 r1, u64 tgt) {
                SgPatDev rec = pd;
                rec.rank0 = r0;
                rec.nsub = r1;
                rec.chunk0 = chunk;
                if (per_sub > tgt && A > 1) {
                    // split each subset's prefix tuples over several chunks
                    u64 parts = (per_sub + tgt - 1) / tgt;
                    if (parts > A) parts = A;
                    rec.ablk = (int)((A + parts - 1) / parts);
                    rec.asplit = (int)((A + rec.ablk - 1) / rec.ablk);
                    rec.spc = 1;
                    chunk += (r1 - r0) * (u64)rec.asplit;
                } else {
                    rec.asplit = 1;
                    rec.ablk = (int)A;
                    rec.spc = std::max<u64>(1, tgt / per_sub);
                    chunk += (r1 - r0 + rec.spc - 1) / rec.spc;
                }
                P->pats.push_back(rec);
                P->pat_chunk0.push_back(rec.chunk0);
            };
            const u64 pe = nsub * per_sub;
            if (by_runs && use_runs[order[q]][ks] && run_slots(A, (u64)pd.tm, 1, rc) <= slot_budget) {
                chunk_by_runs(pd, b.it.d, slot_budget, rc, chunk, P);
                done += pe;
                continue;
            }
            if (done >= tail_cut || item_tail == item_target) {
                emit(0, nsub, done >= tail_cut ? item_tail : item_target);
            } else if (done + pe > tail_cut) {
                const u64 head = (tail_cut - done + per_sub - 1) / per_sub;  // subsets before the cut
                if (head >= nsub) {
                    emit(0, nsub, item_target);
                } else {
                    emit(0, head, item_target);
                    emit(head, nsub, item_tail);
                }
            } else {
                emit(0, nsub, item_target);
            }
            done += pe;
        }
        b.it.npat = (int)((long long)P->pats.size() - b.it.pat0);
        b.it.nchunk = chunk - b.it.chunk0;
        b.it.group0 = P->ngroups;
        b.it.ngroups = (b.it.nchunk + SG_GROUP - 1) / SG_GROUP;
        P->ngroups += b.it.ngroups;
        P->items.push_back(b.it);
        P->roles.push_back(b.role);
        P->item_integral.push_back(b.integral);
        if (b.role.role == SG_ROLE_FORWARD) P->integrals[g].flag_item = (int)q;
    }
    if (chunk > (1ull << 26)) {  // tuned chunk sizes too small for this plan
        plan_free_host(P);
        return SG_ERANGE;
    }
    P->nchunks = chunk;
    // items of each integral (the setup kernel's per-integral warp fills their values)
    P->int_item_ptr.assign(nint + 1, 0);
    for (const SgItemRole &R : P->roles) P->int_item_ptr[R.integral + 1]++;
    for (int g = 0; g < nint; g++) P->int_item_ptr[g + 1] += P->int_item_ptr[g];
    P->int_items.assign(P->roles.size(), 0);
    {
        std::vector<int> fill(P->int_item_ptr.begin(), P->int_item_ptr.end() - 1);
        for (size_t it = 0; it < P->roles.size(); it++) P->int_items[fill[P->roles[it].integral]++] = (int)it;
    }
    if (P->pats.empty()) {  // keep the device arrays non-empty
        SgPatDev pd;
        memset(&pd, 0, sizeof(pd));
        pd.woff = -1;
        P->pats.push_back(pd);
        P->pat_chunk0.push_back(~0ull);
    }
    if (P->blocks.empty()) {
        SgBlockDev bd;
        memset(&bd, 0, sizeof(bd));
        bd.m = 1;
        P->blocks.push_back(bd);
        P->block_refs.push_back(BlockRef{0, 0});
        P->block_end.push_back(0);
    }
    *out = P;
    return SG_OK;
}


void sg_fill_binomials(unsigned long long *B) {
    const unsigned long long SAT = ~0ull;
    for (int k = 0; k < SG_BINOM_K; k++)
        for (int n = 0; n <= SG_MAX_D; n++) {
            unsigned long long v;
            if (k == 0) v = 1;
            else if (n < k) v = 0;
            else {
                // C(n,k) = C(n-1,k-1) + C(n-1,k), saturating
                const unsigned long long x = B[(size_t)(k - 1) * (SG_MAX_D + 1) + n - 1];
                const unsigned long long y = B[(size_t)k * (SG_MAX_D + 1) + n - 1];
                v = (x == SAT || y == SAT || x > SAT - y) ? SAT : x + y;
            }
            B[(size_t)k * (SG_MAX_D + 1) + n] = v;
        }
}

// The host combine of a sharded batch (include/sg.h): the shards' limbs added
// as integers, then rounded (sg_la_round_w, the kernels' rounding) and
// assembled with the same operations as the kernels' assemble_item, so that
// every shard count gives the same bits.
extern "C" sg_status sg_shard_combine(const long long *const *partials, int nshards, const sg_shard_info *info,
                                      int n, sg_result *out) {
    if (!partials || !info || !out || nshards < 1 || n < 1) return SG_EINVAL;
    for (int k = 0; k < nshards; k++)
        if (!partials[k]) return SG_EINVAL;
    for (int k = 0; k < n; k++) {
        long long L[SG_SHARD_LIMBS];
        for (int j = 0; j < SG_SHARD_LIMBS; j++) {
            unsigned long long v = 0;  // wrapping two's complement addition
            for (int sh = 0; sh < nshards; sh++) v += (unsigned long long)partials[sh][(size_t)k * SG_SHARD_LIMBS + j];
            L[j] = (long long)v;
        }
        double s, c, as, ac;
        sg_la_round_w(L, &s, &c);
        sg_la_round_w(L + SG_LA_DIGITS, &as, &ac);
        const double AB = as + ac;
        const double T = AB < 0.0 ? NAN : s + c;
        const sg_shard_info &I = info[k];
        const double rel = I.mult * (I.base_rel + T);
        const double absrel = fabs(I.mult) * (fabs(I.base_rel) + AB);
        int e1 = 0;
        const double mant = frexp(I.scale_m * rel, &e1);
        sg_result &r = out[k];
        r.mant = mant;
        r.exp2 = (int64_t)(I.scale_e2 + e1);
        r.value = ldexp(mant, (int)(I.scale_e2 + e1));
        r.cond = sg_ratio(absrel, fabs(rel));
        r.err_est = 0.05 * I.unit_roundoff * r.cond;
        r.points = I.points;
        r.evals = I.evals;
        r.seconds = 0.0;
    }
    return SG_OK;
}
