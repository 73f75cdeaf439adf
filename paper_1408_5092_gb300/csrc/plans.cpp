// Task-list planner for the block-sparse contractions of the sweep.
#include "plans.h"

#include <algorithm>
#include <map>
#include <tuple>

namespace mpspt {

void GemmPlan::block(double* C, int ldc, int m, int n, int accumulate, int op0) {
    if (m <= 0 || n <= 0) return;
    const int op1 = (int)ops.size();
    for (int o = op0; o < op1; ++o) flops += 2.0 * m * n * ops[o].k;
    for (int r0 = 0; r0 < m; r0 += tm)
        for (int c0 = 0; c0 < n; c0 += tn)
            tasks.push_back({C, ldc, m, n, r0, c0, op0, op1, accumulate, 0});
}

void GemmPlan::upload(cudaStream_t st) {
    if (checks_enabled()) {
        for (const auto& t : tasks) {
            check_range(t.C, ((size_t)(t.m - 1) * t.ldc + t.n) * sizeof(double), "gemm C");
            for (int o = t.op0; o < t.op1; ++o) {
                const GemmOp& op = ops[o];
                const size_t ea = (op.trans & 1) ? (size_t)(op.k - 1) * op.lda + t.m : (size_t)(t.m - 1) * op.lda + op.k;
                const size_t eb = (op.trans & 2) ? (size_t)(t.n - 1) * op.ldb + op.k : (size_t)(op.k - 1) * op.ldb + t.n;
                check_range(op.A, ea * sizeof(double), "gemm A");
                check_range(op.B, eb * sizeof(double), "gemm B");
                if ((op.trans & 1) ? op.lda < t.m : op.lda < op.k) throw Error(MPSPT_ERR_INVALID, "gemm lda");
                if ((op.trans & 2) ? op.ldb < op.k : op.ldb < t.n) throw Error(MPSPT_ERR_INVALID, "gemm ldb");
            }
            if (t.ldc < t.n) throw Error(MPSPT_ERR_INVALID, "gemm ldc");
        }
    }
    mpspt::upload(dtasks, tasks, st);
    mpspt::upload(dops, ops, st);
}

void GemmPlan::run(cudaStream_t st) const {
    if (kind == GEMM_TC) launch_gemm_tc(dtasks.as<GemmTask>(), (int)tasks.size(), dops.as<GemmOp>(), err, st, skip);
    else if (kind == GEMM_F32) launch_gemm_f64in_f32(dtasks.as<GemmTask>(), (int)tasks.size(), dops.as<GemmOp>(), st, skip);
    else launch_gemm_f64(dtasks.as<GemmTask>(), (int)tasks.size(), dops.as<GemmOp>(), st, skip);
}

void Omega::build(const MPO& W, int i) {
    std::map<int, std::vector<const MpoEntry*>> by_b;
    for (const auto& e : W.W[i + 1]) by_b[e.a].push_back(&e);
    std::map<std::tuple<int, int, int, int>, double> acc;
    for (const auto& e1 : W.W[i]) {
        auto it = by_b.find(e1.b);
        if (it == by_b.end()) continue;
        const Mat4& o1 = W.ops[e1.op];
        for (const MpoEntry* e2 : it->second) {
            const Mat4& o2 = W.ops[e2->op];
            const double cc = e1.coef * e2->coef;
            for (int s1 = 0; s1 < 4; ++s1)
                for (int t1 = 0; t1 < 4; ++t1) {
                    const double v1 = o1[s1 * 4 + t1];
                    if (v1 == 0.0) continue;
                    for (int s2 = 0; s2 < 4; ++s2)
                        for (int t2 = 0; t2 < 4; ++t2) {
                            const double v2 = o2[s2 * 4 + t2];
                            if (v2 == 0.0) continue;
                            acc[{s1 * 4 + s2, e1.a, e2->b, t1 * 4 + t2}] += cc * v1 * v2;
                        }
                }
        }
    }
    e.clear();
    first.assign(17, 0);
    for (auto& kv : acc) {
        if (kv.second == 0.0) continue;
        e.push_back({std::get<1>(kv.first), std::get<2>(kv.first), std::get<0>(kv.first),
                     std::get<3>(kv.first), kv.second});
    }
    // entries are sorted by out already (map order); build the index
    int k = 0;
    for (int o = 0; o <= 16; ++o) {
        while (k < (int)e.size() && e[k].out < o) ++k;
        first[o] = k;
    }
}

void TwoSitePlan::build(const Omega& om, const TwoT& bra, const TwoT& ket, const Bond& braL,
                        const Bond& ketL, const Bond& braR, const Bond& ketR, const EnvT& L,
                        const EnvT& R, const std::vector<QN>& dqR, const double* x, double* out,
                        cudaStream_t st) {
    (void)dqR;
    g1.clear();
    g2.clear();
    const int np = (int)ket.panels.size();
    const int nc = (int)(R.idx.size() / (size_t)std::max(1, R.nsk));
    // T panels: one per (c, ket panel) with an R_c block on the panel's sector
    std::vector<long long> toff((size_t)nc * np, -1);
    std::vector<int> tcols((size_t)nc * np, 0);
    std::vector<int> panel_of(ket.blk.size());
    for (int p = 0; p < np; ++p)
        for (int b = ket.panels[p].b0; b < ket.panels[p].b1; ++b) panel_of[b] = p;
    tsize = 0;
    for (int c = 0; c < nc; ++c)
        for (int p = 0; p < np; ++p) {
            int rb = R.find(c, ket.panels[p].sr);
            if (rb < 0) continue;
            int cols = braR.sec[R.blk[rb].sb].dim;
            toff[(size_t)c * np + p] = (long long)tsize;
            tcols[(size_t)c * np + p] = cols;
            tsize += (size_t)ket.panels[p].rows * cols;
        }
    T.ensure((tsize + 1) * sizeof(double), st);
    double* Tp = T.as<double>();
    for (int c = 0; c < nc; ++c)
        for (int p = 0; p < np; ++p) {
            long long o = toff[(size_t)c * np + p];
            if (o < 0) continue;
            const auto& P = ket.panels[p];
            int rb = R.find(c, P.sr);
            int k = ketR.sec[P.sr].dim;
            int m0 = g1.mark();
            g1.op(x + P.off, k, R.ptr(R.blk[rb]), k, k, 2, 1.0);
            g1.block(Tp + o, tcols[(size_t)c * np + p], P.rows, tcols[(size_t)c * np + p], 0, m0);
        }
    // L_a block landing on each bra sector (q_bra = q_ket + dq_a: at most one)
    const int nsb = braL.nsec();
    const int na = (int)(L.idx.size() / (size_t)std::max(1, L.nsk));
    std::vector<int> l_by_sb((size_t)na * nsb, -1);
    for (int b = 0; b < (int)L.blk.size(); ++b) l_by_sb[(size_t)L.blk[b].a * nsb + L.blk[b].sb] = b;
    // output blocks: out = sum L_a [Omega_ac] T_c
    for (const auto& bb : bra.blk) {
        const int o16 = bb.s1 * 4 + bb.s2;
        int m0 = g2.mark();
        for (int q = om.first[o16]; q < om.first[o16 + 1]; ++q) {
            const Omega::E& E = om.e[q];
            const int t1 = E.in / 4, t2 = E.in % 4;
            const int lb = l_by_sb[(size_t)E.a * nsb + bb.sl];
            if (lb < 0) continue;
            const int sk = L.blk[lb].sk;
            const int kb = ket.find(sk, t1, t2);
            if (kb < 0) continue;
            const int p = panel_of[kb];
            const long long o = toff[(size_t)E.c * np + p];
            if (o < 0) continue;
            const int cols = tcols[(size_t)E.c * np + p];
            if (cols != bb.cols) continue;
            const auto& K = ket.blk[kb];
            const size_t row_in_panel = (K.off - ket.panels[p].off) / (size_t)K.cols;
            g2.op(L.ptr(L.blk[lb]), K.rows, Tp + o + row_in_panel * cols, cols, K.rows, 0, E.v);
        }
        g2.block(out + bb.off, bb.cols, bb.rows, bb.cols, 0, m0);
    }
    g1.upload(st);
    g2.upload(st);
}

void DiagPlan::build(const Omega& om, const TwoT& x, const Bond& Lb, const Bond& Rb,
                     const EnvT& Le, const EnvT& Re, const std::vector<QN>& dqL,
                     const std::vector<QN>& dqR, double* out, cudaStream_t st) {
    (void)Lb; (void)Rb;
    tasks.clear();
    terms.clear();
    for (const auto& b : x.blk) {
        const int o16 = b.s1 * 4 + b.s2;
        int t0 = (int)terms.size();
        for (int q = om.first[o16]; q < om.first[o16 + 1]; ++q) {
            const Omega::E& E = om.e[q];
            if (E.in != o16) continue;
            if (!(dqL[E.a] == QN(0, 0)) || !(dqR[E.c] == QN(0, 0))) continue;
            int lb = Le.find(E.a, b.sl), rb = Re.find(E.c, b.sr);
            if (lb < 0 || rb < 0) continue;
            terms.push_back({Le.ptr(Le.blk[lb]), Re.ptr(Re.blk[rb]), b.rows, b.cols, E.v});
        }
        tasks.push_back({out + b.off, b.rows, b.cols, t0, (int)terms.size()});
    }
    if (checks_enabled()) {
        for (const auto& t : tasks) {
            check_range(t.out, (size_t)t.rows * t.cols * sizeof(double), "diag out");
            for (int k = t.t0; k < t.t1; ++k) {
                check_range(terms[k].L, ((size_t)(t.rows - 1) * (terms[k].ldL + 1) + 1) * sizeof(double), "diag L");
                check_range(terms[k].R, ((size_t)(t.cols - 1) * (terms[k].ldR + 1) + 1) * sizeof(double), "diag R");
            }
        }
    }
    upload(dt, tasks, st);
    upload(dterm, terms, st);
}

void DiagPlan::run(cudaStream_t st) const {
    launch_diag(dt.as<DiagTask>(), (int)tasks.size(), dterm.as<DiagTerm>(), st);
}

void plan_product(GemmPlan& g, const TwoT& x, double* xd, const Bond& mid, const SiteT& A,
                  const SiteT& B, const Bond& L) {
    for (const auto& b : x.blk) {
        int m0 = g.mark();
        int sm = mid.find(L.sec[b.sl].q + site_qn(b.s1));
        if (sm >= 0) {
            int ia = A.find(b.sl, b.s1), ib = B.find(sm, b.s2);
            if (ia >= 0 && ib >= 0 && B.blk[ib].sr == b.sr) {
                int k = mid.sec[sm].dim;
                g.op(A.ptr(A.blk[ia]), k, B.ptr(B.blk[ib]), b.cols, k, 0, 1.0);
            }
        }
        g.block(xd + b.off, b.cols, b.rows, b.cols, 0, m0);
    }
}

void EnvPlan::build_left(const MPO& W, int site, const EnvT& L, const SiteT& Abra, const SiteT& Aket,
                         const Bond& braL, const Bond& ketL, const Bond& braR, const Bond& ketR,
                         EnvT& Lnew, cudaStream_t st) {
    g1.clear();
    g2.clear();
    const int na = (int)W.dim[site];
    const int nkb = (int)Aket.blk.size();
    std::vector<long long> yoff((size_t)na * nkb, -1);
    std::vector<int> ysb((size_t)na * nkb, -1);
    size_t ys = 0;
    for (int a = 0; a < na; ++a)
        for (int kb = 0; kb < nkb; ++kb) {
            const auto& K = Aket.blk[kb];
            int lb = L.find(a, K.sl);
            if (lb < 0) continue;
            int sb = L.blk[lb].sb;
            yoff[(size_t)a * nkb + kb] = (long long)ys;
            ysb[(size_t)a * nkb + kb] = sb;
            ys += (size_t)braL.sec[sb].dim * ketR.sec[K.sr].dim;
        }
    Y.ensure((ys + 1) * sizeof(double), st);
    double* Yp = Y.as<double>();
    for (int a = 0; a < na; ++a)
        for (int kb = 0; kb < nkb; ++kb) {
            long long o = yoff[(size_t)a * nkb + kb];
            if (o < 0) continue;
            const auto& K = Aket.blk[kb];
            int lb = L.find(a, K.sl);
            int mb = braL.sec[ysb[(size_t)a * nkb + kb]].dim;
            int kd = ketL.sec[K.sl].dim, nd = ketR.sec[K.sr].dim;
            int m0 = g1.mark();
            g1.op(L.ptr(L.blk[lb]), kd, Aket.ptr(K), nd, kd, 0, 1.0);
            g1.block(Yp + o, nd, mb, nd, 0, m0);
        }
    // group W entries by b
    std::vector<std::vector<const MpoEntry*>> by_b(W.dim[site + 1]);
    for (const auto& e : W.W[site]) by_b[e.b].push_back(&e);
    for (const auto& nb : Lnew.blk) {
        int m0 = g2.mark();
        const int md = braR.sec[nb.sb].dim, nd = ketR.sec[nb.sk].dim;
        for (const MpoEntry* e : by_b[nb.a]) {
            const Mat4& op = W.ops[e->op];
            for (int s = 0; s < 4; ++s)
                for (int t = 0; t < 4; ++t) {
                    const double v = op[s * 4 + t];
                    if (v == 0.0) continue;
                    int slk = ketL.find(ketR.sec[nb.sk].q - site_qn(t));
                    if (slk < 0) continue;
                    int kb = Aket.find(slk, t);
                    if (kb < 0 || Aket.blk[kb].sr != nb.sk) continue;
                    long long o = yoff[(size_t)e->a * nkb + kb];
                    if (o < 0) continue;
                    int slb = ysb[(size_t)e->a * nkb + kb];
                    int bb = Abra.find(slb, s);
                    if (bb < 0 || Abra.blk[bb].sr != nb.sb) continue;
                    int kd = braL.sec[slb].dim;
                    g2.op(Abra.ptr(Abra.blk[bb]), md, Yp + o, nd, kd, 1, e->coef * v);
                }
        }
        g2.block(Lnew.ptr(nb), nd, md, nd, 0, m0);
    }
    g1.upload(st);
    g2.upload(st);
}

void EnvPlan::build_right(const MPO& W, int site, const EnvT& R, const SiteT& Abra, const SiteT& Aket,
                          const Bond& braL, const Bond& ketL, const Bond& braR, const Bond& ketR,
                          EnvT& Rnew, cudaStream_t st) {
    g1.clear();
    g2.clear();
    const int nb_ = (int)W.dim[site + 1];
    const int nkb = (int)Aket.blk.size();
    std::vector<long long> yoff((size_t)nb_ * nkb, -1);
    std::vector<int> ysb((size_t)nb_ * nkb, -1);
    size_t ys = 0;
    for (int b = 0; b < nb_; ++b)
        for (int kb = 0; kb < nkb; ++kb) {
            const auto& K = Aket.blk[kb];
            int rb = R.find(b, K.sr);
            if (rb < 0) continue;
            int sb = R.blk[rb].sb;
            yoff[(size_t)b * nkb + kb] = (long long)ys;
            ysb[(size_t)b * nkb + kb] = sb;
            ys += (size_t)ketL.sec[K.sl].dim * braR.sec[sb].dim;
        }
    Y.ensure((ys + 1) * sizeof(double), st);
    double* Yp = Y.as<double>();
    for (int b = 0; b < nb_; ++b)
        for (int kb = 0; kb < nkb; ++kb) {
            long long o = yoff[(size_t)b * nkb + kb];
            if (o < 0) continue;
            const auto& K = Aket.blk[kb];
            int rb = R.find(b, K.sr);
            int nd = braR.sec[ysb[(size_t)b * nkb + kb]].dim;
            int md = ketL.sec[K.sl].dim, kd = ketR.sec[K.sr].dim;
            int m0 = g1.mark();
            g1.op(Aket.ptr(K), kd, R.ptr(R.blk[rb]), kd, kd, 2, 1.0);
            g1.block(Yp + o, nd, md, nd, 0, m0);
        }
    std::vector<std::vector<const MpoEntry*>> by_a(W.dim[site]);
    for (const auto& e : W.W[site]) by_a[e.a].push_back(&e);
    for (const auto& nbk : Rnew.blk) {
        int m0 = g2.mark();
        const int md = braL.sec[nbk.sb].dim, nd = ketL.sec[nbk.sk].dim;
        for (const MpoEntry* e : by_a[nbk.a]) {
            const Mat4& op = W.ops[e->op];
            for (int s = 0; s < 4; ++s)
                for (int t = 0; t < 4; ++t) {
                    const double v = op[s * 4 + t];
                    if (v == 0.0) continue;
                    int kb = Aket.find(nbk.sk, t);
                    if (kb < 0) continue;
                    long long o = yoff[(size_t)e->b * nkb + kb];
                    if (o < 0) continue;
                    int srb = ysb[(size_t)e->b * nkb + kb];
                    int bb = Abra.find(nbk.sb, s);
                    if (bb < 0 || Abra.blk[bb].sr != srb) continue;
                    int kd = braR.sec[srb].dim;
                    g2.op(Abra.ptr(Abra.blk[bb]), kd, Yp + o, kd, kd, 2, e->coef * v);
                }
        }
        g2.block(Rnew.ptr(nbk), nd, md, nd, 0, m0);
    }
    g1.upload(st);
    g2.upload(st);
}

}  // namespace mpspt
