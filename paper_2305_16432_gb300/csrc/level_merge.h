// Merged-level plan for the triangular solves of "Solve P z = r"
// (Algorithm 1, P = L L^T): the rows of G consecutive levels form one group,
// and substituting the dependencies inside a group expresses each row as
//   y_i = sum_a C_ia r_a - sum_b M_ib y_b,
// with b in earlier groups and a in the row's own group.  With
// D_i the dependencies of row i (coefficient L_ij, diagonal L_ii):
//   M_i = sum_{j in D_i, other group} (L_ij / L_ii) e_j - sum_{j in D_i, same group} (L_ij / L_ii) M_j
//   C_i = e_i / L_ii - sum_{j in D_i, same group} (L_ij / L_ii) C_j
// A group then needs one dependency round instead of G.  The plan is
// symbolic (patterns of M and C and, per entry, the terms that make it) and
// is evaluated numerically for every new factor, in G passes: pass s takes
// the rows whose level is s modulo G, which read only rows of earlier passes
// of their group.  Plain C++ (no CUDA types): the library builds the plan on
// the host; the tests build and evaluate it on the CPU.
#pragma once

#include <algorithm>
#include <cstdint>
#include <vector>

namespace npcg {

struct MergePlan {
    int G = 1;
    int64_t n = 0;
    std::vector<int32_t> grp;            // [n] group of every row (level / G)
    std::vector<int32_t> pass;           // [n] level modulo G
    std::vector<int64_t> diag;           // [n] value index of L_ii
    // patterns, rows ascending within each row
    std::vector<int64_t> mrp, crp;       // [n + 1]
    std::vector<int32_t> mcol, ccol;     // earlier-group rows b / same-group rows a
    // terms of every entry: a term (k, src) adds sign * L[k] / L_ii * (src < 0 ? 1 : X[src]),
    // X the entries of M (for M) or C (for C); sign = +1 for the direct terms
    // (src < 0), -1 for the substituted ones
    std::vector<int64_t> mtp, ctp;       // [nM + 1], [nC + 1]
    std::vector<int64_t> mtk, ctk;       // value index of the L_ij factor (-1: the 1 / L_ii term of C_ii)
    std::vector<int64_t> mts, cts;       // source entry, or -1 for a direct term
};

// dep_rp / dep_row / dep_val: the dependencies of every row (row j and the
// value index of L_ij), diag_val: value index of L_ii, lev: level of every
// row in this solve direction (dependencies sit on lower levels).
inline MergePlan build_merge_plan(int64_t n, const std::vector<int64_t>& dep_rp, const std::vector<int32_t>& dep_row,
                                  const std::vector<int64_t>& dep_val, const std::vector<int64_t>& diag_val,
                                  const std::vector<int32_t>& lev, int G) {
    MergePlan p;
    p.G = G;
    p.n = n;
    p.grp.resize(n);
    p.pass.resize(n);
    p.diag = diag_val;
    for (int64_t i = 0; i < n; ++i) {
        p.grp[i] = lev[i] / G;
        p.pass[i] = lev[i] % G;
    }
    // rows in level order, so that a row's same-group dependencies come first
    std::vector<int64_t> order(n);
    for (int64_t i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return lev[x] < lev[y]; });
    // a term of an entry: L factor k and source entry (row, column), or a direct term (row -1)
    struct Term { int64_t k; int32_t src_row; int32_t src_col; };
    struct Cand { int32_t col; Term t; };
    // per row: its entries' columns (ascending) and, per entry, its terms
    std::vector<std::vector<int32_t>> mcols(n), ccols(n);
    std::vector<std::vector<int64_t>> mtp_r(n), ctp_r(n);          // term offsets per entry (+ end)
    std::vector<std::vector<Term>> mterms(n), cterms(n);
    std::vector<Cand> cm, cc;
    auto emit = [](std::vector<Cand>& cand, std::vector<int32_t>& cols, std::vector<int64_t>& tp,
                   std::vector<Term>& terms) {
        // entries in column order; a column's terms keep their generation order
        std::stable_sort(cand.begin(), cand.end(), [](const Cand& x, const Cand& y) { return x.col < y.col; });
        tp.push_back(0);
        for (size_t a = 0; a < cand.size();) {
            const int32_t col = cand[a].col;
            for (; a < cand.size() && cand[a].col == col; ++a) terms.push_back(cand[a].t);
            cols.push_back(col);
            tp.push_back((int64_t)terms.size());
        }
    };
    for (int64_t oi = 0; oi < n; ++oi) {
        const int64_t i = order[oi];
        cm.clear();
        cc.clear();
        cc.push_back({(int32_t)i, {-1, -1, -1}});                       // e_i / L_ii
        for (int64_t e = dep_rp[i]; e < dep_rp[i + 1]; ++e) {
            const int32_t j = dep_row[e];
            const int64_t k = dep_val[e];
            if (p.grp[j] != p.grp[i]) {
                cm.push_back({j, {k, -1, -1}});                         // + L_ij / L_ii
            } else {
                for (int32_t b : mcols[j]) cm.push_back({b, {k, j, b}});
                for (int32_t a : ccols[j]) cc.push_back({a, {k, j, a}});
            }
        }
        emit(cm, mcols[i], mtp_r[i], mterms[i]);
        emit(cc, ccols[i], ctp_r[i], cterms[i]);
    }
    // flatten: rows ascending, entries ascending, then their terms
    p.mrp.assign(n + 1, 0);
    p.crp.assign(n + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
        p.mrp[i + 1] = p.mrp[i] + (int64_t)mcols[i].size();
        p.crp[i + 1] = p.crp[i] + (int64_t)ccols[i].size();
    }
    p.mcol.reserve(p.mrp[n]);
    p.ccol.reserve(p.crp[n]);
    for (int64_t i = 0; i < n; ++i) {
        p.mcol.insert(p.mcol.end(), mcols[i].begin(), mcols[i].end());
        p.ccol.insert(p.ccol.end(), ccols[i].begin(), ccols[i].end());
    }
    auto entry = [](const std::vector<int64_t>& rp, const std::vector<int32_t>& col, int32_t row, int32_t c) {
        const auto b = col.begin() + rp[row], e = col.begin() + rp[row + 1];
        return (int64_t)(std::lower_bound(b, e, c) - col.begin());
    };
    p.mtp.assign(1, 0);
    p.ctp.assign(1, 0);
    for (int64_t i = 0; i < n; ++i) {
        for (const Term& t : mterms[i]) {
            p.mtk.push_back(t.k);
            p.mts.push_back(t.src_row < 0 ? -1 : entry(p.mrp, p.mcol, t.src_row, t.src_col));
        }
        for (size_t e = 1; e < mtp_r[i].size(); ++e) p.mtp.push_back(p.mtp[p.mtp.size() - 1] + (mtp_r[i][e] - mtp_r[i][e - 1]));
        for (const Term& t : cterms[i]) {
            p.ctk.push_back(t.k);
            p.cts.push_back(t.src_row < 0 ? -1 : entry(p.crp, p.ccol, t.src_row, t.src_col));
        }
        for (size_t e = 1; e < ctp_r[i].size(); ++e) p.ctp.push_back(p.ctp[p.ctp.size() - 1] + (ctp_r[i][e] - ctp_r[i][e - 1]));
        std::vector<Term>().swap(mterms[i]);
        std::vector<Term>().swap(cterms[i]);
    }
    return p;
}

// Numeric evaluation of the plan for factor values Lv (host reference of the
// device passes): M [nM], C [nC].  Within a row the terms are summed in plan
// order.
inline void eval_merge_plan(const MergePlan& p, const double* Lv, std::vector<double>& M, std::vector<double>& C) {
    M.assign(p.mcol.size(), 0.0);
    C.assign(p.ccol.size(), 0.0);
    for (int s = 0; s < p.G; ++s)
        for (int64_t i = 0; i < p.n; ++i) {
            if (p.pass[i] != s) continue;
            const double d = Lv[p.diag[i]];
            for (int64_t e = p.mrp[i]; e < p.mrp[i + 1]; ++e) {
                double v = 0.0;
                for (int64_t t = p.mtp[e]; t < p.mtp[e + 1]; ++t)
                    v += p.mts[t] < 0 ? Lv[p.mtk[t]] / d : -(Lv[p.mtk[t]] / d) * M[p.mts[t]];
                M[e] = v;
            }
            for (int64_t e = p.crp[i]; e < p.crp[i + 1]; ++e) {
                double v = 0.0;
                for (int64_t t = p.ctp[e]; t < p.ctp[e + 1]; ++t)
                    v += p.ctk[t] < 0 ? 1.0 / d : -(Lv[p.ctk[t]] / d) * C[p.cts[t]];
                C[e] = v;
            }
        }
}

// y = solution of the direction's triangular system from the plan (host
// reference of the merged solve): groups in order, every row of a group from
// r and from earlier groups' y.
inline void solve_merge_plan(const MergePlan& p, const std::vector<double>& M, const std::vector<double>& C,
                             const double* r, double* y) {
    int32_t ngroups = 0;
    for (int64_t i = 0; i < p.n; ++i) ngroups = std::max(ngroups, p.grp[i] + 1);
    std::vector<std::vector<int64_t>> rows(ngroups);
    for (int64_t i = 0; i < p.n; ++i) rows[p.grp[i]].push_back(i);
    for (int32_t g = 0; g < ngroups; ++g)
        for (int64_t i : rows[g]) {
            double v = 0.0;
            for (int64_t e = p.crp[i]; e < p.crp[i + 1]; ++e) v += C[e] * r[p.ccol[e]];
            for (int64_t e = p.mrp[i]; e < p.mrp[i + 1]; ++e) v -= M[e] * y[p.mcol[e]];
            y[i] = v;
        }
}

}  // namespace npcg
