// Task-list planner for the block-sparse contractions of the sweep.
#include "plans.h"

#include <algorithm>
#include <cstdio>
#include <map>
#include <tuple>

namespace mpspt {

void GemmPlan::block(double* C, int ldc, int m, int n, int accumulate, int op0, long long cmap_off,
                     int cmap_rows) {
    if (m <= 0 || n <= 0) return;
    const int op1 = (int)ops.size();
    for (int o = op0; o < op1; ++o) flops += 2.0 * m * n * ops[o].k;
    blocks.push_back({C, cmap_off, ldc, m, n, accumulate, op0, op1, cmap_rows});
}

int GemmPlan::kchunks(long long m, long long n, long long K) {
    if (K < 1024 || m * n > 128LL * 512) return 1;
    return (int)std::min<long long>(8, K / 512);
}

void GemmPlan::split(int tm_, int tn_, std::vector<GemmTask>& out, std::vector<long long>* cm,
                     std::vector<SplitRed>* rd, std::vector<long long>* rcm, size_t* part_elems) const {
    out.clear();
    if (cm) cm->clear();
    if (rd) rd->clear();
    if (rcm) rcm->clear();
    size_t pe = 0;
    for (const Blk& b : blocks) {
        long long K = 0;
        for (int o = b.op0; o < b.op1; ++o) K += ops[o].k;
        const int S = rd ? kchunks(b.m, b.n, K) : 1;
        const int step = (int)((K + S - 1) / S + 63) / 64 * 64;   // whole K-stages of either kernel
        for (int r0 = 0; r0 < b.m; r0 += tm_)
            for (int c0 = 0; c0 < b.n; c0 += tn_) {
                if (S == 1) {
                    out.push_back({b.C, nullptr, b.ldc, b.m, b.n, r0, c0, b.op0, b.op1, b.accumulate, b.cmap_rows,
                                   nullptr, 0, 1 << 30});
                    if (cm) cm->push_back(b.cmap_off);
                    continue;
                }
                int np = 0;
                for (long long k0 = 0; k0 < K; k0 += step, ++np) {
                    // the partial pointer holds an element offset until upload
                    out.push_back({b.C, nullptr, b.ldc, b.m, b.n, r0, c0, b.op0, b.op1, 0, b.cmap_rows,
                                   reinterpret_cast<double*>((pe + (size_t)np * tm_ * tn_) * sizeof(double) + 8),
                                   (int)k0, (int)std::min<long long>(K, k0 + step)});
                    if (cm) cm->push_back(-1);
                }
                rd->push_back({reinterpret_cast<const double*>(pe * sizeof(double) + 8), b.C, nullptr, np, tm_, tn_,
                               b.ldc, b.m, b.n, r0, c0, b.accumulate, b.cmap_rows});
                if (rcm) rcm->push_back(b.cmap_off);
                pe += (size_t)np * tm_ * tn_;
            }
    }
    if (part_elems) *part_elems = pe;
}

namespace {
// longest K-list first: the persistent kernels hand out tasks in strides of
// the grid, so this order balances the CTAs (each output tile has exactly
// one task, so the order does not change any result)
void order_tasks(std::vector<GemmTask>& tasks, std::vector<long long>* cm, const std::vector<GemmOp>& ops) {
    std::vector<long long> cost(tasks.size());
    for (size_t i = 0; i < tasks.size(); ++i) {
        long long k = 0;
        for (int o = tasks[i].op0; o < tasks[i].op1; ++o) k += ops[o].k;
        cost[i] = k;
    }
    std::vector<size_t> ord(tasks.size());
    for (size_t i = 0; i < ord.size(); ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
    std::vector<GemmTask> t2(tasks.size());
    std::vector<long long> c2(cm ? tasks.size() : 0);
    for (size_t i = 0; i < ord.size(); ++i) {
        t2[i] = tasks[ord[i]];
        if (cm) c2[i] = (*cm)[ord[i]];
    }
    tasks.swap(t2);
    if (cm) cm->swap(c2);
}

int bucket(long long x) {
    int b = 0;
    while (x > 1) { x >>= 1; ++b; }
    return b;
}
}  // namespace

void GemmPlan::upload(cudaStream_t st) {
    mpspt::upload(dops, ops, st);
    if (tuner && !is_tc(kind) && !blocks.empty()) {
        const std::pair<int, int> t = tuner->choose(*this, st);
        tm = t.first;
        tn = t.second;
    }
    size_t pe = 0;
    split(tm, tn, tasks, &task_cmap, &reds, &red_cmap, &pe);
    if (pe) dpart.ensure(pe * sizeof(double) + 16, st);
    double* pbase = dpart.as<double>();
    for (auto& t : tasks)   // partial offsets (stored as byte offsets + 8) become pointers
        if (t.part) t.part = pbase + ((reinterpret_cast<uintptr_t>(t.part) - 8) / sizeof(double));
    for (auto& r : reds) r.part = pbase + ((reinterpret_cast<uintptr_t>(r.part) - 8) / sizeof(double));
    order_tasks(tasks, &task_cmap, ops);
    if (!cmaps.empty()) mpspt::upload(dcmaps, cmaps, st);
    const int* cbase = dcmaps.as<int>();
    for (size_t i = 0; i < tasks.size(); ++i)
        tasks[i].cmap = task_cmap[i] >= 0 ? cbase + task_cmap[i] : nullptr;
    for (size_t i = 0; i < reds.size(); ++i) reds[i].cmap = red_cmap[i] >= 0 ? cbase + red_cmap[i] : nullptr;
    if (!reds.empty()) mpspt::upload(dreds, reds, st);
    if (checks_enabled()) {
        // per planned block (all tiles of a block share its output and its
        // K-list): the output range, or the span of its mapped addresses,
        // and every operand range of its K-list
        for (const Blk& b : blocks) {
            if (b.cmap_off < 0) {
                check_range(b.C, ((size_t)(b.m - 1) * b.ldc + b.n) * sizeof(double), "gemm C");
                if (b.ldc < b.n) throw Error(MPSPT_ERR_INVALID, "gemm ldc");
            } else {
                const long long o = b.cmap_off;
                const int nmap = b.cmap_rows ? b.m : b.n, other = b.cmap_rows ? b.n : b.m;
                require((size_t)(o + 2 * (long long)nmap) <= cmaps.size(), "gemm cmap range");
                long long lo = 0, hi = 0;
                for (int q = 0; q < nmap; ++q) {
                    const long long base = cmaps[o + 2 * q], ld = cmaps[o + 2 * q + 1];
                    require(base >= 0 && ld >= 0, "gemm cmap entry");
                    const long long last = base + (long long)(other - 1) * ld;
                    lo = q ? std::min(lo, base) : base;
                    hi = q ? std::max(hi, last) : last;
                }
                check_range(b.C + lo, (size_t)(hi - lo + 1) * sizeof(double), "gemm cmap dst");
            }
            for (int q = b.op0; q < b.op1; ++q) {
                const GemmOp& op = ops[q];
                const size_t ea = (op.trans & 1) ? (size_t)(op.k - 1) * op.lda + b.m : (size_t)(b.m - 1) * op.lda + op.k;
                const size_t eb = (op.trans & 2) ? (size_t)(b.n - 1) * op.ldb + op.k : (size_t)(op.k - 1) * op.ldb + b.n;
                check_range(op.A, ea * sizeof(double), "gemm A");
                check_range(op.B, eb * sizeof(double), "gemm B");
                if ((op.trans & 1) ? op.lda < b.m : op.lda < op.k) throw Error(MPSPT_ERR_INVALID, "gemm lda");
                if ((op.trans & 2) ? op.ldb < op.k : op.ldb < b.n) throw Error(MPSPT_ERR_INVALID, "gemm ldb");
            }
        }
    }
    mpspt::upload(dtasks, tasks, st);
}

void Autotuner::RawBuf::ensure(size_t bytes) {
    if (bytes <= n) return;
    const size_t want = std::max(bytes, 2 * n);
    if (p) old.push_back(p);
    p = nullptr;
    n = 0;
    MPSPT_CUDA(cudaMalloc(&p, want));
    Registry::get().add(p, want);
    n = want;
}

Autotuner::RawBuf::~RawBuf() {
    old.push_back(p);
    for (void* q : old)
        if (q) {
            Registry::get().remove(q);
            cudaFree(q);
        }
}

Autotuner::~Autotuner() {
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
}

std::pair<int, int> Autotuner::choose(const GemmPlan& g, cudaStream_t st) {
    std::vector<long long> ms, ns, ks;
    size_t cmax = 1;
    for (const auto& b : g.blocks) {
        long long k = 0;
        for (int o = b.op0; o < b.op1; ++o) k += g.ops[o].k;
        ms.push_back(b.m);
        ns.push_back(b.n);
        ks.push_back(k);
        cmax = std::max(cmax, (size_t)b.m * b.n);
    }
    auto med = [](std::vector<long long>& v) {
        std::nth_element(v.begin(), v.begin() + v.size() / 2, v.end());
        return v[v.size() / 2];
    };
    const Key key{g.kind, g.skinny ? 1 : 0, bucket(med(ms)), bucket(med(ns)), bucket(med(ks)),
                  bucket((long long)g.blocks.size())};
    std::lock_guard<std::mutex> lk(mu);
    auto it = best.find(key);
    if (it != best.end()) { ++reused; return it->second; }
    static const int cand_wide[][2] = {{64, 64}, {32, 64}, {64, 32}, {32, 32}};
    static const int cand_skinny[][2] = {{16, 128}, {32, 64}, {32, 32}};
    const int (*cand)[2] = g.skinny ? cand_skinny : cand_wide;
    const int nc = g.skinny ? 3 : 4;
    if (!ev[0]) {
        MPSPT_CUDA(cudaEventCreate(&ev[0]));
        MPSPT_CUDA(cudaEventCreate(&ev[1]));
    }
    scratch.ensure(cmax * sizeof(double) + 16);
    std::pair<int, int> win{cand[0][0], cand[0][1]};
    float tbest = 1e30f;
    std::vector<GemmTask> tt;
    for (int c = 0; c < nc; ++c) {
        g.split(cand[c][0], cand[c][1], tt, nullptr);
        order_tasks(tt, nullptr, g.ops);
        for (auto& t : tt) {   // outputs go to scratch: dense m x n, no map; operands are the plan's
            t.C = static_cast<double*>(scratch.p);
            t.ldc = t.n;
            t.cmap = nullptr;
            t.cmap_rows = 0;
        }
        dtasks.ensure(tt.size() * sizeof(GemmTask) + 16);
        const GemmTask* dt = static_cast<const GemmTask*>(dtasks.p);
        if (!tt.empty()) copy_h2d(dtasks.p, tt.data(), tt.size() * sizeof(GemmTask), st);
        const bool f32 = g.kind == GEMM_F32;
        launch_gemm_tile(cand[c][0], cand[c][1], f32, dt, (int)tt.size(), g.dops.as<GemmOp>(), st);
        MPSPT_CUDA(cudaEventRecord(ev[0], st));
        for (int r = 0; r < 3; ++r)
            launch_gemm_tile(cand[c][0], cand[c][1], f32, dt, (int)tt.size(), g.dops.as<GemmOp>(), st);
        MPSPT_CUDA(cudaEventRecord(ev[1], st));
        MPSPT_CUDA(cudaEventSynchronize(ev[1]));
        float ms_ = 0.f;
        MPSPT_CUDA(cudaEventElapsedTime(&ms_, ev[0], ev[1]));
        if (ms_ < tbest) { tbest = ms_; win = {cand[c][0], cand[c][1]}; }
    }
    ++timed;
    best[key] = win;
    return win;
}

void Autotuner::load(const std::string& path) {
    FILE* f = std::fopen(path.c_str(), "r");
    if (!f) return;
    int a[8];
    std::lock_guard<std::mutex> lk(mu);
    while (std::fscanf(f, "%d %d %d %d %d %d %d %d", &a[0], &a[1], &a[2], &a[3], &a[4], &a[5], &a[6], &a[7]) == 8)
        if (gemm_tile_supported(a[6], a[7])) best[Key{a[0], a[1], a[2], a[3], a[4], a[5]}] = {a[6], a[7]};
    std::fclose(f);
}

void Autotuner::save(const std::string& path) {
    FILE* f = std::fopen(path.c_str(), "w");
    if (!f) return;
    std::lock_guard<std::mutex> lk(mu);
    for (const auto& kv : best) {
        const Key& k = kv.first;
        std::fprintf(f, "%d %d %d %d %d %d %d %d\n", std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k),
                     std::get<4>(k), std::get<5>(k), kv.second.first, kv.second.second);
    }
    std::fclose(f);
}

void GemmPlan::run(cudaStream_t st) const {
    const int nt = (int)tasks.size();
    if (nt == 0) return;
    const GemmTask* t = dtasks.as<GemmTask>();
    const GemmOp* o = dops.as<GemmOp>();
    if (is_tc(kind)) launch_gemm_tc(t, nt, o, err, st, skip, kind == GEMM_TC16);
    else launch_gemm_tile(tm, tn, kind == GEMM_F32, t, nt, o, st, skip);
    if (!reds.empty()) launch_splitk_reduce(dreds.as<SplitRed>(), (int)reds.size(), st, skip);
}

void Omega::build(const MPO& W, int i) {
    std::map<int, std::vector<const MpoEntry*>> by_b;
    for (const auto& e : W.W[i + 1]) by_b[e.a].push_back(&e);
    std::map<std::tuple<int, int, int, int>, double> acc;   // (a, out, c, in)
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
                            acc[{e1.a, s1 * 4 + s2, e2->b, t1 * 4 + t2}] += cc * v1 * v2;
                        }
                }
        }
    }
    Da = W.dim[i];
    e.clear();
    for (auto& kv : acc) {
        if (kv.second == 0.0) continue;
        e.push_back({std::get<0>(kv.first), std::get<2>(kv.first), std::get<1>(kv.first),
                     std::get<3>(kv.first), kv.second});
    }
    first.assign((size_t)Da * 16 + 1, 0);
    size_t k = 0;
    for (int key = 0; key <= Da * 16; ++key) {
        while (k < e.size() && e[k].a * 16 + e[k].out < key) ++k;
        first[key] = (int)k;
    }
}

void TwoSitePlan::build(const Omega& om, const TwoT& bra, const TwoT& ket, const Bond& braL,
                        const Bond& ketL, const Bond& braR, const Bond& ketR, const EnvT& L,
                        const EnvT& R, const std::vector<QN>& dqR, const double* x, double* out,
                        cudaStream_t st) {
    (void)dqR; (void)ketL;
    g1.clear(); g2.clear(); g2s.clear();
    mtasks.clear(); msrc.clear();
    const int np = (int)ket.panels.size();
    const int nc = (int)(R.idx.size() / (size_t)std::max(1, R.nsk));
    const int na = om.Da;
    // ---- Rpack per ket right sector: blocks R_c(sb_c, sk) stacked by c
    std::vector<long long> rp_off(ketR.nsec(), -1);
    std::vector<int> rp_rows(ketR.nsec(), 0);
    std::vector<int> rcol((size_t)nc * ketR.nsec(), -1);   // row offset of c inside Rpack(sk)
    size_t rps = 0;
    std::vector<CopyTask> pk_tasks;
    for (const auto& P : ket.panels) {
        const int sk = P.sr;
        int rows = 0;
        for (int c = 0; c < nc; ++c) {
            int rb = R.find(c, sk);
            if (rb < 0) continue;
            rcol[(size_t)c * ketR.nsec() + sk] = rows;
            rows += braR.sec[R.blk[rb].sb].dim;
        }
        rp_rows[sk] = rows;
        rp_off[sk] = (long long)rps;
        rps += (size_t)rows * ketR.sec[sk].dim;
    }
    // ---- Lpack per bra left sector: blocks L_a(sl, sk_a) side by side
    std::vector<int> lp_cols(braL.nsec(), 0);
    std::vector<long long> lp_off(braL.nsec(), -1);
    std::vector<int> lcol((size_t)na * braL.nsec(), -1);
    std::vector<int> l_blk((size_t)na * braL.nsec(), -1);
    for (int b = 0; b < (int)L.blk.size(); ++b) l_blk[(size_t)L.blk[b].a * braL.nsec() + L.blk[b].sb] = b;
    size_t lps = 0;
    for (int sl = 0; sl < braL.nsec(); ++sl) {
        int cols = 0;
        for (int a = 0; a < na; ++a) {
            int lb = l_blk[(size_t)a * braL.nsec() + sl];
            if (lb < 0) continue;
            lcol[(size_t)a * braL.nsec() + sl] = cols;
            cols += ketL.sec[L.blk[lb].sk].dim;
        }
        lp_cols[sl] = cols;
        lp_off[sl] = (long long)lps;
        lps += (size_t)braL.sec[sl].dim * cols;
    }
    Rp.ensure((rps + 1) * sizeof(double), st);
    Lp.ensure((lps + 1) * sizeof(double), st);
    double* Rpp = Rp.as<double>();
    double* Lpp = Lp.as<double>();
    for (const auto& P : ket.panels) {
        const int sk = P.sr, dk = ketR.sec[sk].dim;
        for (int c = 0; c < nc; ++c) {
            int rb = R.find(c, sk);
            if (rb < 0) continue;
            const int db = braR.sec[R.blk[rb].sb].dim;
            pk_tasks.push_back({R.ptr(R.blk[rb]), Rpp + rp_off[sk] + (size_t)rcol[(size_t)c * ketR.nsec() + sk] * dk,
                                nullptr, db, dk, dk, dk, 0, 0});
        }
    }
    for (int sl = 0; sl < braL.nsec(); ++sl)
        for (int a = 0; a < na; ++a) {
            int lb = l_blk[(size_t)a * braL.nsec() + sl];
            if (lb < 0) continue;
            const int dl = braL.sec[sl].dim, dk = ketL.sec[L.blk[lb].sk].dim;
            pk_tasks.push_back({L.ptr(L.blk[lb]), Lpp + lp_off[sl] + lcol[(size_t)a * braL.nsec() + sl],
                                nullptr, dl, dk, dk, lp_cols[sl], 0, 0});
        }
    if (checks_enabled())
        for (const auto& t : pk_tasks) {
            check_range(t.src, ((size_t)(t.rows - 1) * t.lds + t.cols_n) * sizeof(double), "pack src");
            check_range(t.dst, ((size_t)(t.rows - 1) * t.ldd + t.cols_n) * sizeof(double), "pack dst");
        }
    mpspt::upload(pk, pk_tasks, st);
    launch_copy(pk.as<CopyTask>(), (int)pk_tasks.size(), st);
    // ---- T panels
    std::vector<long long> toff(np, -1);
    std::vector<int> panel_of(ket.blk.size());
    tsize = 0;
    for (int p = 0; p < np; ++p) {
        const auto& P = ket.panels[p];
        for (int b = P.b0; b < P.b1; ++b) panel_of[b] = p;
        if (rp_rows[P.sr] == 0) continue;
        toff[p] = (long long)tsize;
        tsize += (size_t)P.rows * rp_rows[P.sr];
    }
    T.ensure((tsize + 1) * sizeof(double), st);
    double* Tp = T.as<double>();
    for (int p = 0; p < np; ++p) {
        if (toff[p] < 0) continue;
        const auto& P = ket.panels[p];
        const int dk = ketR.sec[P.sr].dim, nr = rp_rows[P.sr];
        int m0 = g1.mark();
        g1.op(x + P.off, dk, Rpp + rp_off[P.sr], dk, dk, 2, 1.0);
        g1.block(Tp + toff[p], nr, P.rows, nr, 0, m0);
    }
    // ---- bra left panels, V stacks and mix tasks
    std::vector<std::vector<int>> left_blocks(braL.nsec());
    for (int b = 0; b < (int)bra.blk.size(); ++b) left_blocks[bra.blk[b].sl].push_back(b);
    std::vector<long long> voff(braL.nsec(), -1);
    std::vector<int> wd(braL.nsec(), 0);
    size_t vs = 0;
    for (int sl = 0; sl < braL.nsec(); ++sl) {
        int w = 0;
        for (int b : left_blocks[sl]) w += bra.blk[b].cols;
        wd[sl] = w;
        if (w == 0 || lp_cols[sl] == 0) continue;
        voff[sl] = (long long)vs;
        vs += (size_t)lp_cols[sl] * w;
    }
    V.ensure((vs + 1) * sizeof(double), st);
    double* Vp = V.as<double>();
    for (int sl = 0; sl < braL.nsec(); ++sl) {
        if (voff[sl] < 0) continue;
        const int W = wd[sl];
        // column map of the bra left panel -> two-site layout
        std::vector<int> cm;
        int wcol = 0;
        for (int bi : left_blocks[sl]) {
            const auto& B = bra.blk[bi];
            for (int r = 0; r < B.cols; ++r) { cm.push_back((int)(B.off + r)); cm.push_back(B.cols); }
            for (int a = 0; a < na; ++a) {
                const int lc = lcol[(size_t)a * braL.nsec() + sl];
                if (lc < 0) continue;
                const int lb = l_blk[(size_t)a * braL.nsec() + sl];
                const int sk = L.blk[lb].sk, dk = ketL.sec[sk].dim;
                MixTask mt{Vp + voff[sl] + (size_t)lc * W + wcol, dk, B.cols, W, (int)msrc.size(), 0, 0};
                const int o16 = B.s1 * 4 + B.s2;
                for (int q = om.begin(a, o16); q < om.end(a, o16); ++q) {
                    const Omega::E& E = om.e[q];
                    const int kb = ket.find(sk, E.in / 4, E.in % 4);
                    if (kb < 0) continue;
                    const int p = panel_of[kb];
                    if (toff[p] < 0) continue;
                    const int srk = ket.panels[p].sr;
                    const int rc = rcol[(size_t)E.c * ketR.nsec() + srk];
                    if (rc < 0) continue;
                    const int rb = R.find(E.c, srk);
                    if (R.blk[rb].sb != B.sr) continue;
                    const auto& K = ket.blk[kb];
                    const size_t rip = (K.off - ket.panels[p].off) / (size_t)K.cols;
                    const int nr = rp_rows[srk];
                    msrc.push_back({Tp + toff[p] + rip * nr + rc, nr, 0, E.v});
                }
                mt.s1 = (int)msrc.size();
                mtasks.push_back(mt);
            }
            wcol += B.cols;
        }
        // g2: out(sl, :) = Lpack(sl) V_stack(sl); TC computes the transpose (rows = panel cols)
        const int dl = braL.sec[sl].dim, K = lp_cols[sl];
        if (is_tc(kind)) {
            const long long co = g2.add_cmap(cm);
            int m0 = g2.mark();
            g2.op(Vp + voff[sl], W, Lpp + lp_off[sl], K, K, 1 | 2, 1.0);
            g2.block(out, 0, W, dl, 0, m0, co, 1);
        } else {
            GemmPlan& g = (dl <= 16) ? g2s : g2;
            const long long co = g.add_cmap(cm);
            int m0 = g.mark();
            g.op(Lpp + lp_off[sl], K, Vp + voff[sl], W, K, 0, 1.0);
            g.block(out, 0, dl, W, 0, m0, co, 0);
        }
    }
    // bra blocks whose left panel has no operator: zero them through the mix path
    for (int sl = 0; sl < braL.nsec(); ++sl) {
        if (voff[sl] >= 0) continue;
        for (int bi : left_blocks[sl]) {
            const auto& B = bra.blk[bi];
            mtasks.push_back({out + B.off, B.rows, B.cols, B.cols, (int)msrc.size(), (int)msrc.size(), 0});
        }
    }
    if (checks_enabled()) {
        for (const auto& t : mtasks) {
            check_range(t.dst, ((size_t)(t.rows - 1) * t.ldd + t.cols) * sizeof(double), "mix dst");
            for (int q = t.s0; q < t.s1; ++q)
                check_range(msrc[q].src, ((size_t)(t.rows - 1) * msrc[q].lds + t.cols) * sizeof(double), "mix src");
        }
    }
    mpspt::upload(dmt, mtasks, st);
    mpspt::upload(dms, msrc, st);
    g1.upload(st);
    g2.upload(st);
    g2s.upload(st);
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
        for (int a = 0; a < om.Da; ++a) {
            if (!(dqL[a] == QN(0, 0))) continue;
            const int lb = Le.find(a, b.sl);
            if (lb < 0) continue;
            for (int q = om.begin(a, o16); q < om.end(a, o16); ++q) {
                const Omega::E& E = om.e[q];
                if (E.in != o16 || !(dqR[E.c] == QN(0, 0))) continue;
                const int rb = Re.find(E.c, b.sr);
                if (rb < 0) continue;
                terms.push_back({Le.ptr(Le.blk[lb]), Re.ptr(Re.blk[rb]), b.rows, b.cols, E.v});
            }
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

void EnvPlan::upload_mix(cudaStream_t st) {
    if (checks_enabled()) {
        for (const auto& t : mt) {
            check_range(t.dst, ((size_t)(t.rows - 1) * t.ldd + t.cols) * sizeof(double), "env mix dst");
            for (int q = t.s0; q < t.s1; ++q)
                check_range(ms[q].src, ((size_t)(t.rows - 1) * ms[q].lds + t.cols) * sizeof(double), "env mix src");
        }
    }
    mpspt::upload(dmt, mt, st);
    mpspt::upload(dms, ms, st);
    g1.upload(st);
    g2.upload(st);
}

// L_new[b](sb', sk') = sum_{s,t} A_bra(sl_b, s)^T [sum_a W_ab(s,t) L_a(sl_b, sl_k)] A_ket(sl_k, t)
void EnvPlan::build_left(const MPO& W, int site, const EnvT& L, const SiteT& Abra, const SiteT& Aket,
                         const Bond& braL, const Bond& ketL, const Bond& braR, const Bond& ketR,
                         EnvT& Lnew, cudaStream_t st) {
    (void)braR;
    g1.clear();
    g2.clear();
    mt.clear();
    ms.clear();
    const int nkb = (int)Aket.blk.size();
    // g1: Y_kb = L_panel(sl_k) A_ket(kb), (panel rows) x dim(sr_k)
    std::vector<long long> yoff(nkb, -1);
    size_t ys = 0;
    for (int kb = 0; kb < nkb; ++kb) {
        const auto& K = Aket.blk[kb];
        if (L.prows[K.sl] == 0) continue;
        yoff[kb] = (long long)ys;
        ys += (size_t)L.prows[K.sl] * ketR.sec[K.sr].dim;
    }
    Y.ensure((ys + 1) * sizeof(double), st);
    double* Yp = Y.as<double>();
    for (int kb = 0; kb < nkb; ++kb) {
        if (yoff[kb] < 0) continue;
        const auto& K = Aket.blk[kb];
        const int kd = ketL.sec[K.sl].dim, nd = ketR.sec[K.sr].dim, P = L.prows[K.sl];
        const int m0 = g1.mark();
        g1.op(L.panel(K.sl), kd, Aket.ptr(K), nd, kd, 0, 1.0);
        g1.block(Yp + yoff[kb], nd, P, nd, 0, m0);
    }
    // mix: Z_(out, s) over the MPO entries e = (a -> b) and t
    const std::vector<MpoEntry>& We = W.W[site];
    const std::vector<int>&in_ptr = W.in_ptr[site], &in_idx = W.in_idx[site];
    struct ZB { int nb, s, bb; size_t off; int rows, cols; };
    std::vector<ZB> zb;
    size_t zs = 0;
    for (int nbi = 0; nbi < (int)Lnew.blk.size(); ++nbi) {
        const auto& nb = Lnew.blk[nbi];
        const int nd = ketR.sec[nb.sk].dim;
        // ket-side lookups depend on t only
        int slk_t[4], kb_t[4];
        for (int t = 0; t < 4; ++t) {
            slk_t[t] = ketL.find(ketR.sec[nb.sk].q - site_qn(t));
            kb_t[t] = slk_t[t] < 0 ? -1 : Aket.find(slk_t[t], t);
            if (kb_t[t] >= 0 && (Aket.blk[kb_t[t]].sr != nb.sk || yoff[kb_t[t]] < 0)) kb_t[t] = -1;
        }
        for (int s = 0; s < 4; ++s) {
            const int slb = braL.find(braR.sec[nb.sb].q - site_qn(s));
            if (slb < 0) continue;
            const int bb = Abra.find(slb, s);
            if (bb < 0 || Abra.blk[bb].sr != nb.sb) continue;
            const int rows = braL.sec[slb].dim;
            const int s0 = (int)ms.size();
            for (int q = in_ptr[nb.a]; q < in_ptr[nb.a + 1]; ++q) {
                const MpoEntry* e = &We[in_idx[q]];
                const Mat4& op = W.ops[e->op];
                for (int t = 0; t < 4; ++t) {
                    const double v = op[s * 4 + t];
                    if (v == 0.0 || kb_t[t] < 0) continue;
                    const int lb = L.find(e->a, slk_t[t]);
                    if (lb < 0 || L.blk[lb].sb != slb) continue;
                    ms.push_back({Yp + yoff[kb_t[t]] + (size_t)L.blk[lb].roff * nd, nd, 0, e->coef * v});
                }
            }
            if ((int)ms.size() == s0) continue;
            zb.push_back({nbi, s, bb, zs, rows, nd});
            mt.push_back({nullptr, rows, nd, nd, s0, (int)ms.size(), 0});
            zs += (size_t)rows * nd;
        }
    }
    Z.ensure((zs + 1) * sizeof(double), st);
    double* Zp = Z.as<double>();
    for (size_t q = 0; q < zb.size(); ++q) mt[q].dst = Zp + zb[q].off;
    // g2: L_new(out) = sum_s A_bra(sl_b, s)^T Z_(out, s)
    size_t z = 0;
    for (int nbi = 0; nbi < (int)Lnew.blk.size(); ++nbi) {
        const auto& nb = Lnew.blk[nbi];
        const int md = braR.sec[nb.sb].dim, nd = ketR.sec[nb.sk].dim;
        const int m0 = g2.mark();
        for (; z < zb.size() && zb[z].nb == nbi; ++z)
            g2.op(Abra.ptr(Abra.blk[zb[z].bb]), md, Zp + zb[z].off, nd, zb[z].rows, 1, 1.0);
        g2.block(Lnew.ptr(nb), nd, md, nd, 0, m0);
    }
    upload_mix(st);
}

void EnvPlan::build_left_run(const RunMap& T, const EnvT& L, const Bond& bra, const Bond& ket, EnvT& Lnew,
                             cudaStream_t st) {
    g1.clear();
    g2.clear();
    mt.clear();
    ms.clear();
    for (const auto& nb : Lnew.blk) {
        const int rows = bra.sec[nb.sb].dim, cols = ket.sec[nb.sk].dim;
        const int s0 = (int)ms.size();
        for (int q = T.ptr[nb.a]; q < T.ptr[nb.a + 1]; ++q) {
            const int lb = L.find(T.col[q], nb.sk);
            if (lb < 0 || L.blk[lb].sb != nb.sb) continue;
            ms.push_back({L.ptr(L.blk[lb]), cols, 0, T.val[q]});
        }
        mt.push_back({Lnew.ptr(nb), rows, cols, cols, s0, (int)ms.size(), 0});
    }
    upload_mix(st);
}

// R_new[a](sb, sk) = sum_{s,t} A_bra(sb, s) [sum_b W_ab(s,t) R_b(sr_b, sr_k)] A_ket(sk, t)^T
void EnvPlan::build_right(const MPO& W, int site, const EnvT& R, const SiteT& Abra, const SiteT& Aket,
                          const Bond& braL, const Bond& ketL, const Bond& braR, const Bond& ketR,
                          EnvT& Rnew, cudaStream_t st) {
    g1.clear();
    g2.clear();
    mt.clear();
    ms.clear();
    const int nkb = (int)Aket.blk.size();
    // g1: Y_kb = A_ket(kb) R_panel(sr_k)^T, dim(sl_k) x (panel rows)
    std::vector<long long> yoff(nkb, -1);
    size_t ys = 0;
    for (int kb = 0; kb < nkb; ++kb) {
        const auto& K = Aket.blk[kb];
        if (R.prows[K.sr] == 0) continue;
        yoff[kb] = (long long)ys;
        ys += (size_t)ketL.sec[K.sl].dim * R.prows[K.sr];
    }
    Y.ensure((ys + 1) * sizeof(double), st);
    double* Yp = Y.as<double>();
    for (int kb = 0; kb < nkb; ++kb) {
        if (yoff[kb] < 0) continue;
        const auto& K = Aket.blk[kb];
        const int md = ketL.sec[K.sl].dim, kd = ketR.sec[K.sr].dim, P = R.prows[K.sr];
        const int m0 = g1.mark();
        g1.op(Aket.ptr(K), kd, R.panel(K.sr), kd, kd, 2, 1.0);
        g1.block(Yp + yoff[kb], P, md, P, 0, m0);
    }
    // mix: Z_(out, s) = sum over e = (a -> b), t of W_ab(s, t) Y_(b, kb(t)), dim(sk) x dim(sr_b)
    const std::vector<MpoEntry>& We = W.W[site];
    const std::vector<int>& out_ptr = W.out_ptr[site];
    struct ZB { int nb, s, bb; size_t off; int rows, cols; };
    std::vector<ZB> zb;
    size_t zs = 0;
    for (int nbi = 0; nbi < (int)Rnew.blk.size(); ++nbi) {
        const auto& nbk = Rnew.blk[nbi];
        const int nd = ketL.sec[nbk.sk].dim;
        int kb_t[4];   // ket-side lookups depend on t only
        for (int t = 0; t < 4; ++t) {
            kb_t[t] = Aket.find(nbk.sk, t);
            if (kb_t[t] >= 0 && yoff[kb_t[t]] < 0) kb_t[t] = -1;
        }
        for (int s = 0; s < 4; ++s) {
            const int bb = Abra.find(nbk.sb, s);
            if (bb < 0) continue;
            const int srb = Abra.blk[bb].sr;
            const int cols = braR.sec[srb].dim;
            const int s0 = (int)ms.size();
            for (int q = out_ptr[nbk.a]; q < out_ptr[nbk.a + 1]; ++q) {
                const MpoEntry* e = &We[q];
                const Mat4& op = W.ops[e->op];
                for (int t = 0; t < 4; ++t) {
                    const double v = op[s * 4 + t];
                    if (v == 0.0) continue;
                    const int kb = kb_t[t];
                    if (kb < 0) continue;
                    const int srk = Aket.blk[kb].sr;
                    const int rb = R.find(e->b, srk);
                    if (rb < 0 || R.blk[rb].sb != srb) continue;
                    ms.push_back({Yp + yoff[kb] + R.blk[rb].roff, R.prows[srk], 0, e->coef * v});
                }
            }
            if ((int)ms.size() == s0) continue;
            zb.push_back({nbi, s, bb, zs, nd, cols});
            mt.push_back({nullptr, nd, cols, cols, s0, (int)ms.size(), 0});
            zs += (size_t)nd * cols;
        }
    }
    Z.ensure((zs + 1) * sizeof(double), st);
    double* Zp = Z.as<double>();
    for (size_t q = 0; q < zb.size(); ++q) mt[q].dst = Zp + zb[q].off;
    // g2: R_new(out) = sum_s A_bra(sb, s) Z_(out, s)^T
    size_t z = 0;
    for (int nbi = 0; nbi < (int)Rnew.blk.size(); ++nbi) {
        const auto& nbk = Rnew.blk[nbi];
        const int md = braL.sec[nbk.sb].dim, nd = ketL.sec[nbk.sk].dim;
        const int m0 = g2.mark();
        for (; z < zb.size() && zb[z].nb == nbi; ++z)
            g2.op(Abra.ptr(Abra.blk[zb[z].bb]), zb[z].cols, Zp + zb[z].off, zb[z].cols, zb[z].cols, 2, 1.0);
        g2.block(Rnew.ptr(nbk), nd, md, nd, 0, m0);
    }
    upload_mix(st);
}

}  // namespace mpspt
