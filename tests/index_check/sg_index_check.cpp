// Host-side check of the fold kernel's index arithmetic (test infrastructure).
//
// Builds a plan with the library's own planner, then walks every chunk
// sequentially with the same enumeration primitives the CUDA kernel uses
// (sg_fold_logic.h): unranking, runs, tail segments, prefix entries.  Every
// table access is checked against the bounds of the block it must fall in,
// and both lane layouts of a run (the flat one of the FP64 and float-float
// folds, the lane groups of the float fold) are replayed to check that each
// (prefix tuple, tail entry) pair is visited exactly once.  The sums are formed in double so that the tests can also
// compare them with the oracle; this is a check of the enumeration, not a
// second implementation of the method (no CUDA code path calls it).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "../../paper_2210_14313_gb300/csrc/sg_fixed.h"
#include "../../paper_2210_14313_gb300/csrc/sg_xsum.h"
#include "../../paper_2210_14313_gb300/csrc/sg_lacc.h"
#include "../../paper_2210_14313_gb300/csrc/sg_fold_logic.h"
#include "../../paper_2210_14313_gb300/csrc/sg_plan.h"
#include "../../paper_2210_14313_gb300/csrc/sg_rules.h"

namespace {

double phi_dev(int fam, double a, double u, double x) {
    switch (fam) {
    case 0:
    case 1: return a * (x - 0.5);
    case 2: {
        double v = x - u;
        return log1p((0.5 - x) * (0.5 + x - 2.0 * u) / (1.0 / (a * a) + v * v));
    }
    case 3: return -a * a * (x - 0.5) * (x + 0.5 - 2.0 * u);
    case 4: return -a * (x - 0.5) * (x + 0.5 - 2.0 * u);
    }
    return 0;
}

double phi_c(int fam, double a, double u) {
    switch (fam) {
    case 0:
    case 1: return 0.5 * a;
    case 2: return -log(1.0 / (a * a) + (0.5 - u) * (0.5 - u));
    case 3: return -a * a * (0.5 - u) * (0.5 - u);
    case 4: return -a * (0.5 - u) * (0.5 - u);
    }
    return 0;
}

// a merged weight kept to 64 bits, rounded to a double
double w64_value(const SgW64 &w) {
    const double v = ldexp((double)w.m, w.e - 1086);
    return w.neg ? -v : v;
}

void neu(double &s, double &c, double v) {
    double t = s + v;
    if (fabs(s) >= fabs(v)) c += (s - t) + v;
    else c += (v - t) + s;
    s = t;
}

}  // namespace

extern "C" {

// Returns 0 on success; out[0] = forward value relative to exp(log f(c))
// (i.e. base + T times the multiplier), out[1] = log f(c) (exponential
// families), out[2] = number of bound violations, out[3] = pairs visited
// other than exactly once, out[4] = evaluations, out[5] = chunks,
// out[6] = evaluations the plan claims, out[9] = the most runs (subsets
// sharing a prefix) in one chunk, out[8] = lane slots of the point
// loop (32 x warp passes; evaluations / slots is the lane occupancy).  vout receives the adjoint sub-sums
// (nv entries, may be NULL); nv_out their count.
int chk_run(int kind, int fam, const double *params, int d, int L, int form, int grad, int ppc,
            int ctas_per_sm, int warps, double *out, double *vout, long long *nv_out) {
    sg_rule_s rule;
    rule.kind = kind;
    rule.max_level = L + 2 > SG_MAX_LEVEL ? SG_MAX_LEVEL : L + 2;
    std::vector<double> tx(2 * 4097 + 2), tw(2 * 4097 + 2);
    int off = 0;
    for (int bk = 0; bk < 4; bk++)
        for (int k = 1; k < rule.max_level; k++) {
            int n = sg_block(kind, bk, k, tx.data(), tw.data());
            rule.x[bk][k].assign(tx.begin(), tx.begin() + n);
            rule.w[bk][k].assign(tw.begin(), tw.begin() + n);
            rule.off[bk][k] = off;
            off += n;
        }
    std::vector<Req> reqs(1);
    reqs[0] = Req{&rule, fam, d, L, form, 0, grad};
    sg_tuning t{ppc, ctas_per_sm, warps};
    Plan *P = nullptr;
    if (build_plan_host(reqs, 0, t, 152LL * ctas_per_sm * warps, &P) != SG_OK) return 1;

    // table, filled from the host block lists
    std::vector<double2> tab(P->nentries > 0 ? P->nentries : 1);
    std::vector<int> owner(tab.size(), -1);  // block index of every entry
    for (size_t b = 0; b < P->blocks.size() && P->nentries > 0; b++) {
        const SgBlockDev &B = P->blocks[b];
        const BlockRef R = P->block_refs[b];
        const long long begin = b ? P->block_end[b - 1] : 0;
        if (B.off != begin) return 2;
        const std::vector<double> &x = rule.x[R.bk][R.k], &w = rule.w[R.bk][R.k];
        for (int i = 0; i < d; i++)
            for (int j = 0; j < B.m; j++) {
                const long long e = B.off + (long long)i * B.m + j;
                if (e >= P->block_end[b]) return 3;
                tab[e].x = phi_dev(fam, params[i], params[d + i], x[j]);
                tab[e].y = w[j];
                owner[e] = (int)b;
            }
    }
    // centre quantities
    double ls = 0, lc = 0;
    for (int i = 0; i < d; i++) neu(ls, lc, phi_c(fam, params[i], params[d + i]));
    double sth = 0, cth = 1;
    if (fam == 1) {
        const double th = remainder(6.28318530717958647693 * params[d] + (ls + lc), 6.28318530717958647693);
        sth = sin(th);
        cth = cos(th);
    }
    // per-item values (as the prep kernel computes them)
    const int nitems = (int)P->items.size();
    std::vector<SgItemVar> var(nitems);
    for (int it = 0; it < nitems; it++) {
        const SgItemRole &R = P->roles[it];
        double sn = sth, cs = cth;
        if (R.role != SG_ROLE_FORWARD && fam == 1) {
            double tmp = sn;
            sn = cs;
            cs = -tmp;
        }
        double shift = R.role == SG_ROLE_ADJOINT ? phi_dev(fam, params[R.dir], params[d + R.dir], R.x) : 0.0;
        if (fam == 1) {
            var[it].sin_phi = sn * cos(shift) + cs * sin(shift);
            var[it].cos_phi = cs * cos(shift) - sn * sin(shift);
            var[it].base_rel = var[it].cos_phi;
            var[it].mult = 1.0;
        } else {
            var[it].sin_phi = 0;
            var[it].cos_phi = 1;
            var[it].base_rel = 1;
            var[it].mult = exp(shift);
        }
    }
    std::vector<unsigned long long> B((size_t)SG_BINOM_K * (SG_MAX_D + 1));
    sg_fill_binomials(B.data());

    long long violations = 0, badpairs = 0;
    unsigned long long evals = 0;
    long long lane_slots = 0, max_runs = 0;
    std::vector<double> slot(P->nchunks, 0.0);
    int idx[SG_MAX_R];
    for (unsigned long long c = 0; c < P->nchunks; c++) {
        long long lo = 0, hi = (long long)P->pats.size() - 1;
        while (lo < hi) {
            long long mid = (lo + hi + 1) >> 1;
            if (P->pat_chunk0[mid] <= c) lo = mid;
            else hi = mid - 1;
        }
        const SgPatDev *Pp = &P->pats[lo];
        const SgItemDev *I = &P->items[Pp->item];
        if (c < I->chunk0 || c >= I->chunk0 + I->nchunk) violations++;
        const SgItemVar &V = var[Pp->item];
        const long long tbase = I->tab;
        const int dd = I->d, r = Pp->r, skip = I->skip;
        unsigned long long rank, cnt;
        int a_lo, a_hi;
        sg_chunk_span(Pp, c, &rank, &cnt, &a_lo, &a_hi);
        if (a_lo < 0 || a_hi > Pp->A || a_lo >= a_hi) violations++;
        sg_unrank_lex(rank, dd, r, B.data(), idx);
        // replay the kernel's 32-wide unranking rounds; it must agree
        {
            int p = -1;
            unsigned long long rk = rank;
            for (int t = 0; t < r; t++) {
                SgUnrankPos u;
                sg_unrank_begin(&u, rk, dd, r, t, p, B.data());
                for (int rounds = 0;; rounds++) {
                    unsigned mask = 0;
                    for (int j = 0; j < 32; j++)
                        if (sg_unrank_test(&u, sg_unrank_candidate(&u, j), dd, B.data())) mask |= 1u << j;
                    if (!(mask & 1u) || rounds > 3) {
                        violations++;
                        break;
                    }
                    if (sg_unrank_narrow(&u, mask)) break;
                }
                rk -= u.total - sg_binom(B.data(), dd - u.lo, u.k);
                if (u.lo != idx[t]) violations++;
                p = u.lo;
            }
        }
        for (int t = 1; t < r; t++)
            if (idx[t] <= idx[t - 1]) violations++;
        if (idx[r - 1] >= dd) violations++;
        auto check = [&](long long rel, long long blk_off, int m) {
            const long long e = tbase + rel;
            if (e < 0 || e >= P->nentries) {
                violations++;
                return false;
            }
            // must lie inside the intended block of this item's integral
            const SgBlockDev &Bk = P->blocks[owner[e]];
            if (Bk.off != tbase + blk_off || Bk.m != m) violations++;
            return true;
        };
        double acc = 0.0;
        long long runs = 0;
        while (cnt > 0) {
            runs++;
            const int plast = idx[r - 1];
            const int run = (unsigned long long)(dd - plast) < cnt ? dd - plast : (int)cnt;
            const SgTailSegs seg = sg_tail_segments(Pp->toff, Pp->tm, plast, run, skip);
            const int E = seg.E1 + seg.E2;
            if (E != run * Pp->tm) violations++;
            std::vector<double> S(Pp->A), W(Pp->A);
            for (int a = a_lo; a < a_hi; a++) {
                int q = a;
                double s = 0, w = 1;
                for (int tt = r - 2; tt >= 0; tt--) {
                    const int dir = sg_actual_dir(idx[tt], skip);
                    if (dir == skip || dir >= dd + (skip >= 0)) violations++;
                    // the kernels' divide-free digit (magic multiplier) must agree
                    const int q0 = q, mm = Pp->pm[tt];
                    const int qm = sg_div_magic_q(q0, sg_div_magic(mm));
                    const long long rel = sg_prefix_entry(Pp, tt, dir, &q);
                    if (qm != q || Pp->poff[tt] + (long long)dir * mm + (q0 - qm * mm) != rel) violations++;
                    if (check(rel, Pp->poff[tt], Pp->pm[tt])) {
                        s += tab[tbase + rel].x;
                        w *= tab[tbase + rel].y;
                    }
                }
                S[a] = s;
                W[a] = w;
            }
            // replay the lane split of fold_run (one pass per prefix tile)
            for (int ab = a_lo; ab < a_hi; ab += SG_APAD) {
                const int At = a_hi - ab < SG_APAD ? a_hi - ab : SG_APAD;
                std::vector<int> seen((size_t)At * E, 0);
                long long passes = 0;
                for (int lane = 0; lane < 32; lane++) {
                    long long mine = 0;
                    for (SgFlatPos f(lane, E); f.a < At; f.step(), mine++) {
                        const int e = f.e, a = f.a;
                        const long long rel = e < seg.E1 ? seg.base1 + e : seg.base2 + (e - seg.E1);
                        if (!check(rel, Pp->toff, Pp->tm)) continue;
                        const double2 te = tab[tbase + rel];
                        seen[(size_t)a * E + e]++;
                        // merged form: the weight from the pattern's table (its
                        // oscillatory factor -2 included)
                        const bool mw = Pp->woff >= 0;
                        const double Sv = S[ab + a] + te.x;
                        const double Wv = mw ? w64_value(P->wt64[Pp->woff + (long long)(ab + a) * Pp->tm + e % Pp->tm])
                                             : W[ab + a] * te.y;
                        double D;
                        if (I->gk == SG_GK_OSC)
                            D = (mw ? 1.0 : -2.0) * sin(0.5 * Sv) * (V.sin_phi * cos(0.5 * Sv) + V.cos_phi * sin(0.5 * Sv));
                        else D = expm1(Sv);
                        acc += Wv * D;
                        evals++;
                    }
                    if (mine > passes) passes = mine;
                }
                lane_slots += 32 * passes;
                for (int v : seen)
                    if (v != 1) badpairs++;
                // the float fold's lane groups must cover the same pairs once
                std::vector<int> seen2((size_t)At * E, 0);
                for (int lane = 0; lane < 32; lane++) {
                    const SgLaneGroups lg(lane, E);
                    if (!lg.active) continue;
                    for (int e = lg.e0; e < E; e += lg.estep)
                        for (int a = lg.a0; a < At; a += lg.astep) seen2[(size_t)a * E + e]++;
                }
                for (int v : seen2)
                    if (v != 1) badpairs++;
            }
            cnt -= run;
            if (cnt > 0 && !sg_next_prefix(idx, dd, r)) violations++;
        }
        slot[c] = acc * Pp->coef;
        if (runs > max_runs) max_runs = runs;
    }
    // per-item fixed-order reduction and assembly
    std::vector<double> vals(P->nout, 0.0);
    long long nv = P->nv;
    for (int it = 0; it < nitems; it++) {
        const SgItemDev &I = P->items[it];
        double s = 0, cc = 0;
        for (unsigned long long q = 0; q < I.nchunk; q++) neu(s, cc, slot[I.chunk0 + q]);
        const double rel = var[it].mult * (var[it].base_rel + (s + cc));
        if (P->item_integral[it] < 0) {
            if (vout && I.out < nv) vout[I.out] = rel;
        } else {
            vals[I.out] = rel;
        }
    }
    out[0] = vals[0];
    out[1] = ls + lc;
    out[2] = (double)violations;
    out[3] = (double)badpairs;
    out[4] = (double)evals;
    out[5] = (double)P->nchunks;
    out[6] = (double)P->total_evals;
    if (P->nout > 1) out[7] = vals[1];
    out[8] = (double)lane_slots;
    out[9] = (double)max_runs;
    if (nv_out) *nv_out = nv;
    plan_free_host(P);
    return 0;
}

// Compares the kernel's 32-wide unranking rounds with the serial binary
// search for n ranks spread over [0, C(d, r)) (the first, the last and a
// multiplicative sequence in between).  Returns the number of mismatches,
// or -1 if C(d, r) is 0 or does not fit the table.
long long chk_unrank(int d, int r, long long n) {
    std::vector<unsigned long long> B((size_t)SG_BINOM_K * (SG_MAX_D + 1));
    sg_fill_binomials(B.data());
    const unsigned long long total = sg_binom(B.data(), d, r);
    if (total == 0) return -1;
    long long bad = 0;
    unsigned long long x = 0x9E3779B97F4A7C15ull;
    for (long long i = 0; i < n; i++) {
        unsigned long long rank;
        if (i == 0) rank = 0;
        else if (i == 1) rank = total - 1;
        else {
            x = x * 6364136223846793005ull + 1442695040888963407ull;
            rank = (x >> 11) % total;
        }
        int a[SG_MAX_R], b[SG_MAX_R];
        sg_unrank_lex(rank, d, r, B.data(), a);
        int p = -1;
        unsigned long long rk = rank;
        for (int t = 0; t < r; t++) {
            SgUnrankPos u;
            sg_unrank_begin(&u, rk, d, r, t, p, B.data());
            for (int rounds = 0;; rounds++) {
                unsigned mask = 0;
                for (int j = 0; j < 32; j++)
                    if (sg_unrank_test(&u, sg_unrank_candidate(&u, j), d, B.data())) mask |= 1u << j;
                if (!(mask & 1u) || rounds > 3) {
                    bad++;
                    break;
                }
                if (sg_unrank_narrow(&u, mask)) break;
            }
            rk -= u.total - sg_binom(B.data(), d - u.lo, u.k);
            b[t] = u.lo;
            p = u.lo;
        }
        for (int t = 0; t < r; t++)
            if (a[t] != b[t]) {
                bad++;
                break;
            }
    }
    return bad;
}

// The library's level rule and blocks, built on the host (no device needed).
int chk_rule(int kind, int level, double *x, double *w) { return sg_rule_level(kind, level, x, w); }
int chk_block(int kind, int bk, int k, double *x, double *w) { return sg_block(kind, bk, k, x, w); }

// The fixed-point elementary functions of the FP64 fold (sg_fixed.h), built
// for the host: kind 0: expm1(x) for |x| <= ln2/2; kind 1: sin and cos for
// |x| <= 0.7854 (y holds pairs); kind 2: sin(x) sin(phi + x); kind 3:
// w sin(x) sin(phi + x); kind 4: w expm1(x) (w may be NULL for kinds 0-2).
void chk_fixed(int kind, const double *x, const double *w, double *y, long long n, double phi) {
    const SgFxPhase ph = sg_fx_phase(sin(phi), cos(phi));
    for (long long i = 0; i < n; i++) {
        if (kind == 0) {
            y[i] = sg_fx_expm1(x[i]);
        } else if (kind == 1) {
            sg_fx_sincos(x[i], &y[2 * i], &y[2 * i + 1]);
        } else if (kind == 2) {
            y[i] = sg_fx_osc_dev(x[i], ph);
        } else if (kind == 3) {
            y[i] = sg_fx_osc_dev_w(x[i], w[i], ph);
        } else {
            y[i] = sg_fx_expm1_w(x[i], w[i]);
        }
    }
}

// Mismatches of the divide-free q / m (sg_div_magic) for m in [1, mmax] and
// q in a sample of [0, 2^31): every q < 4096, the ends, and a multiplicative
// sequence.
long long chk_divmagic(int mmax) {
    long long bad = 0;
    for (int m = 1; m <= mmax; m++) {
        const SgDivMagic g = sg_div_magic(m);
        for (long long q = 0; q < 4096; q++)
            if (sg_div_magic_q((int)q, g) != (int)(q / m)) bad++;
        for (long long q = 4096; q < 0x7fffffffll; q = q * 9 / 7 + 13)
            if (sg_div_magic_q((int)q, g) != (int)(q / m)) bad++;
        const long long ends[] = {0x7fffffffll, 0x7ffffffell, (0x7fffffffll / m) * m, (0x7fffffffll / m) * m - 1};
        for (long long q : ends)
            if (q >= 0 && sg_div_magic_q((int)q, g) != (int)(q / m)) bad++;
    }
    return bad;
}

// sg_fx_to_double_f(v[i], neg[i] & 1, q[i]) for n values (the fixed-point
// functions' conversion back to double).
void chk_fx_to_double(const unsigned long long *v, const unsigned long long *neg, const int *q, long long n,
                      double *y) {
    for (long long i = 0; i < n; i++) y[i] = sg_fx_to_double_f(v[i], neg[i] & 1ull, q[i]);
}

// The reduction's exact 128-bit window sum (sg_xsum.h) of v[0..n), in the
// order given: out = (s, c).
void chk_xsum(const double *v, long long n, double *out) {
    int E = 1;
    for (long long i = 0; i < n; i++) E = sg_x_exp(v[i]) > E ? sg_x_exp(v[i]) : E;
    SgX a = {0ull, 0ull};
    for (long long i = 0; i < n; i++) sg_x_add(a, v[i], E);
    sg_x_pair(a, E, &out[0], &out[1]);
}

// The setup kernel's scheme: nthreads running sums with adaptive units over
// the terms i = t, t + nthreads, ..., aligned to the largest unit and added.
void chk_xsum_adaptive(const double *v, long long n, int nthreads, double *out) {
    std::vector<SgX> acc(nthreads, SgX{0ull, 0ull});
    std::vector<int> E(nthreads, 1);
    for (int t = 0; t < nthreads; t++)
        for (long long i = t; i < n; i += nthreads) sg_x_add_adaptive(acc[t], E[t], v[i]);
    int Eb = 1;
    for (int t = 0; t < nthreads; t++) Eb = E[t] > Eb ? E[t] : Eb;
    SgX tot = {0ull, 0ull};
    for (int t = 0; t < nthreads; t++) {
        sg_x_shr(acc[t], Eb - E[t]);
        sg_x_plus(tot, acc[t]);
    }
    sg_x_pair(tot, Eb, &out[0], &out[1]);
}

// The limbs of the long accumulator over v[0..n) (the kernels' per-item
// accumulation: each term's digits added into carry-save limbs).
void chk_lacc_limbs(const double *v, long long n, long long *limbs) {
    int ovf = 0;
    for (int k = 0; k < SG_LA_DIGITS; k++) limbs[k] = 0;
    for (long long i = 0; i < n; i++)
        for (int k = 0; k < SG_LA_DIGITS; k++) limbs[k] += sg_la_digit(v[i], k, &ovf);
}

// Every point of the merged form of (kind, d, L) with its weight from the
// library's planner (merged_weights): X[n][d] coordinates on [0,1], Wt[n].
// Returns the point count (only counted when it exceeds cap), -1 on error.
long long chk_merged_points(int kind, int d, int L, double *X, double *Wt, long long cap) {
    sg_rule_s rule;
    rule.kind = kind;
    rule.max_level = L + 2 > SG_MAX_LEVEL ? SG_MAX_LEVEL : L + 2;
    std::vector<double> tx(2 * 4097 + 2), tw(2 * 4097 + 2);
    for (int bk = 0; bk < 4; bk++)
        for (int k = 1; k < rule.max_level; k++) {
            int n = sg_block(kind, bk, k, tx.data(), tw.data());
            rule.x[bk][k].assign(tx.begin(), tx.begin() + n);
            rule.w[bk][k].assign(tw.begin(), tw.begin() + n);
        }
    std::vector<PatSpec> specs;
    gen_patterns(SG_FORM_MERGED, d, L, specs);
    drop_empty_patterns(&rule, specs);
    Plan P;
    if (!merged_weights(&rule, d, L, 1.0, specs, &P)) return -1;
    long long n = 0;
    for (const PatSpec &sp : specs) {
        std::vector<int> ex(sp.r);
        for (int t = 0; t < sp.r - 1; t++) ex[t] = sp.pre[t].k;
        ex[sp.r - 1] = sp.tail.k;
        std::vector<int> dir(sp.r);
        for (int t = 0; t < sp.r; t++) dir[t] = t;
        for (;;) {  // r-subsets in lexicographic order
            // tuples: prefix digits with the last prefix position fastest, then the tail node
            std::vector<int> j(sp.r, 0);
            long long a = 0;
            for (;;) {
                if (n < cap) {
                    for (int i = 0; i < d; i++) X[n * d + i] = 0.5;
                    for (int t = 0; t < sp.r; t++) X[n * d + dir[t]] = rule.x[SG_BLK_NEW][ex[t]][j[t]];
                    Wt[n] = w64_value(P.wt64[sp.woff + a]);
                }
                n++;
                a++;
                int t = sp.r - 1;
                while (t >= 0 && ++j[t] == (int)rule.x[SG_BLK_NEW][ex[t]].size()) j[t--] = 0;
                if (t < 0) break;
            }
            int t = sp.r - 1;
            while (t >= 0 && dir[t] == d - sp.r + t) t--;
            if (t < 0) break;
            dir[t]++;
            for (int u = t + 1; u < sp.r; u++) dir[u] = dir[u - 1] + 1;
        }
    }
    return n;
}

// The single-integral fold's long accumulator (sg_lacc.h): v[0..n) split
// into nparts contiguous parts (one set of limbs each, as the CTAs hold
// them), the parts' limbs added, then rounded: out = (s, c, overflow flag,
// digits outside the three the kernels add).
void chk_lacc(const double *v, long long n, int nparts, double *out) {
    std::vector<long long> tot(SG_LA_DIGITS, 0);
    out[3] = 0;
    int ovf = 0;
    for (int p = 0; p < nparts; p++) {
        std::vector<long long> part(SG_LA_DIGITS, 0);
        const long long i0 = n * p / nparts, i1 = n * (p + 1) / nparts;
        for (long long i = i0; i < i1; i++) {
            // as the kernels add a term: the (at most three) digits from the first
            const int k0 = sg_la_first_digit(v[i], &ovf);
            for (int k = 0; k < SG_LA_DIGITS; k++) {
                const long long dg = sg_la_digit(v[i], k, &ovf);
                if (dg && (k0 < 0 || k < k0 || k > k0 + 2)) out[3] += 1;  // a digit the kernels would miss
                if (k0 >= 0 && k >= k0 && k <= k0 + 2) part[k] += dg;
            }
        }
        for (int k = 0; k < SG_LA_DIGITS; k++) tot[k] += part[k];
    }
    sg_la_round(tot.data(), &out[0], &out[1]);
    out[2] = ovf;
}

// The long accumulator fed as the kernels feed it a chunk's exact sum:
// the terms are cut into nparts chunks, each chunk's terms are added exactly
// in a 128-bit window under its largest term (sg_xsum.h) and the window
// sum enters the limbs digit by digit (sg_la_x_digit) without a rounding
// to doubles.  out = (s, c, overflow, sum of |chunk sums| as s).
void chk_lacc_x(const double *v, long long n, int nparts, double *out) {
    std::vector<long long> tot(SG_LA_DIGITS, 0), mag(SG_LA_DIGITS, 0);
    int ovf = 0;
    for (int p = 0; p < nparts; p++) {
        const long long i0 = n * p / nparts, i1 = n * (p + 1) / nparts;
        int E = 1;
        for (long long i = i0; i < i1; i++) E = sg_x_exp(v[i]) > E ? sg_x_exp(v[i]) : E;
        SgX t = {0ull, 0ull};
        for (long long i = i0; i < i1; i++) sg_x_add(t, v[i], E);
        for (int k = 0; k < SG_LA_DIGITS; k++) {
            long long m = 0;
            tot[k] += sg_la_x_digit(t, E, k, &ovf, &m);
            mag[k] += m;
        }
    }
    double mc = 0.0;
    sg_la_round(tot.data(), &out[0], &out[1]);
    sg_la_round(mag.data(), &out[3], &mc);
    out[2] = ovf;
}

// sg_ratio (the condition number's quotient without an FP64 division) over
// n pairs.
void chk_ratio(const double *a, const double *b, long long n, double *out) {
    for (long long i = 0; i < n; i++) out[i] = sg_ratio(a[i], b[i]);
}

}  // extern "C"
