// C ABI of the MPS-PT library: argument checks, exception barrier, handles.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>

#include "eig.h"
#include "engine.h"

struct mpspt_ctx {
    std::unique_ptr<mpspt::Ctx> c;
};

struct mpspt_mlp {
    std::unique_ptr<mpspt::Mlp> m;
    int device = 0;
};

struct mpspt_mps {
    std::unique_ptr<mpspt::MpsD> m;
    cudaStream_t st = 0;
    int device = 0;
};

namespace {

thread_local std::string g_last;

template <class F>
mpspt_status guard(mpspt_ctx* ctx, F&& f) {
    try {
        f();
        return MPSPT_OK;
    } catch (const mpspt::Error& e) {
        g_last = e.what();
        if (ctx && ctx->c) ctx->c->last_error = g_last;
        return e.status;
    } catch (const std::bad_alloc&) {
        g_last = "host allocation failed";
        return MPSPT_ERR_OOM;
    } catch (const std::exception& e) {
        g_last = e.what();
        return MPSPT_ERR_INVALID;
    }
}

}  // namespace

namespace {
void fill_report(mpspt_report* rep, const mpspt::SweepResult& r) {
    std::memset(rep, 0, sizeof(*rep));
    rep->n_sweeps = (int)r.e2_sweep.size();
    for (int s = 0; s < rep->n_sweeps && s < 64; ++s) rep->e2_per_sweep[s] = r.e2_sweep[s];
    rep->max_discarded_weight = r.max_disc;
    rep->cg_iters = r.cg_iters;
    rep->sigma_calls = r.sigma_calls;
    rep->sigma_flops = r.sigma_flops;
    rep->sigma_ms = r.sigma_ms;
    rep->wall_ms = r.wall_ms;
    rep->max_bond_dim = r.max_bond;
    for (int s = 0; s < rep->n_sweeps && s < 64 && s < (int)r.sweep_ms.size(); ++s) rep->sweep_ms[s] = r.sweep_ms[s];
    rep->kernel_launches = r.launches;
    rep->sigma64_calls = r.sigma64_calls;
    rep->sigma64_flops = r.sigma64_flops;
    rep->sigma64_ms = r.sigma64_ms;
    rep->learned_used = r.learned_used;
    rep->learned_rejected = r.learned_rejected;
    rep->converged = r.converged ? 1 : 0;
    for (int s = 0; s < (int)r.disc_sweep.size() && s < 64; ++s) rep->max_discarded_per_sweep[s] = r.disc_sweep[s];
    for (int s = 0; s < (int)r.sigma_cum.size() && s < 64; ++s) rep->sigma_calls_cum[s] = r.sigma_cum[s];
    rep->host_wait_ms = r.host_wait_ms;
}
}  // namespace

extern "C" {

void mpspt_default_options(mpspt_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->device = 0;
    o->stream = nullptr;
    o->prec = MPSPT_FP64;
    o->max_sweeps = 30;
    o->e_tol = 1e-10;
    o->cg_tol = 1e-10;
    o->cg_max_iter = 1000;
    o->seed = 1408;
    o->use_learned = 0;
    o->verbose = 0;
    o->eig_fp64_only = 0;
    o->keep_rel = 1e-10;
    o->autotune = 0;
    o->autotune_cache = nullptr;
    o->cuda_graphs = 0;
}

mpspt_status mpspt_create(mpspt_ctx** ctx, const mpspt_options* opt) {
    if (!ctx) return MPSPT_ERR_INVALID;
    mpspt_options o;
    mpspt_default_options(&o);
    if (opt) o = *opt;
    return guard(nullptr, [&] {
        mpspt::require(o.max_sweeps >= 1 && o.cg_max_iter >= 1 && o.cg_tol > 0 && o.e_tol > 0 &&
                           o.keep_rel >= 0.0 && o.keep_rel < 1.0,
                       "invalid options");
        mpspt::require(o.prec == MPSPT_FP64 || o.prec == MPSPT_FP32 || o.prec == MPSPT_MIXED_BF16 ||
                           o.prec == MPSPT_MIXED_FP16,
                       "unknown precision mode");
        auto* h = new mpspt_ctx;
        try {
            h->c.reset(new mpspt::Ctx(o));
        } catch (...) {
            delete h;
            throw;
        }
        *ctx = h;
    });
}

void mpspt_destroy(mpspt_ctx* ctx) { delete ctx; }

mpspt_status mpspt_set_integrals(mpspt_ctx* ctx, int k_act, int k_virt, int n_elec, const double* h,
                                 const double* L, int n_chol) {
    if (!ctx) return MPSPT_ERR_INVALID;
    return guard(ctx, [&] { mpspt::set_integrals(*ctx->c, k_act, k_virt, n_elec, h, L, n_chol); });
}

mpspt_status mpspt_set_reference_ci(mpspt_ctx* ctx, const double* ci, long long n_ci) {
    if (!ctx) return MPSPT_ERR_INVALID;
    return guard(ctx, [&] {
        MPSPT_CUDA(cudaSetDevice(ctx->c->opt.device));
        mpspt::set_reference(*ctx->c, ci, n_ci);
    });
}

mpspt_status mpspt_set_reference(mpspt_ctx* ctx, int n_sites_act, const int* blk_count, const int* blk_meta,
                                 const double* const* blk_data) {
    if (!ctx || n_sites_act < 1 || !blk_count || !blk_meta || !blk_data) return MPSPT_ERR_INVALID;
    return guard(ctx, [&] {
        auto& c = *ctx->c;
        MPSPT_CUDA(cudaSetDevice(c.opt.device));
        mpspt::require(c.P.have_int, "mpspt_set_integrals must come first", MPSPT_ERR_STATE);
        mpspt::require(n_sites_act == c.P.ka, "n_sites_act must equal k_act");
        const int ns = n_sites_act;
        // bond sectors: QN -> dimension, from both sides of every cut
        std::vector<std::map<mpspt::QN, int>> sec(ns + 1);
        auto note = [&](int cut, mpspt::QN q, int d) {
            mpspt::require(d >= 1, "block dimensions must be >= 1");
            auto it = sec[cut].find(q);
            if (it == sec[cut].end()) sec[cut][q] = d;
            else mpspt::require(it->second == d, "a bond sector has different dimensions in different blocks");
        };
        long long nb = 0;
        for (int st = 0; st < ns; ++st) {
            mpspt::require(blk_count[st] >= 0, "negative block count");
            for (int b = 0; b < blk_count[st]; ++b, ++nb) {
                const int* m = blk_meta + 7 * nb;
                mpspt::require(m[2] >= 0 && m[2] < 4, "local state must be 0..3");
                const mpspt::QN ql(m[0], m[1]), qr(m[3], m[4]);
                mpspt::require(qr == ql + mpspt::site_qn(m[2]), "block QN change does not match its local state");
                mpspt::require(blk_data[nb] != nullptr, "null block data");
                note(st, ql, m[5]);
                note(st + 1, qr, m[6]);
            }
        }
        mpspt::MpsHost h;
        h.nsite = ns;
        h.bond.resize(ns + 1);
        for (int cut = 0; cut <= ns; ++cut) {
            for (auto& kv : sec[cut]) h.bond[cut].sec.push_back({kv.first, kv.second, 0});
            h.bond[cut].finalize();
        }
        h.T.resize(ns);
        for (int st = 0; st < ns; ++st)
            h.T[st].assign((size_t)h.bond[st].total * 4 * h.bond[st + 1].total, 0.0);
        std::vector<std::vector<char>> seen(ns);
        nb = 0;
        for (int st = 0; st < ns; ++st) {
            const mpspt::Bond &L = h.bond[st], &R = h.bond[st + 1];
            seen[st].assign((size_t)L.nsec() * 4, 0);
            for (int b = 0; b < blk_count[st]; ++b, ++nb) {
                const int* m = blk_meta + 7 * nb;
                const int sl = L.find(mpspt::QN(m[0], m[1])), sr = R.find(mpspt::QN(m[3], m[4]));
                char& sn = seen[st][(size_t)sl * 4 + m[2]];
                mpspt::require(!sn, "duplicate reference block");
                sn = 1;
                const double* src = blk_data[nb];
                for (int i = 0; i < m[5]; ++i)
                    for (int j = 0; j < m[6]; ++j)
                        h.T[st][((size_t)(L.sec[sl].off + i) * 4 + m[2]) * R.total + R.sec[sr].off + j] =
                            src[(size_t)i * m[6] + j];
            }
        }
        mpspt::set_reference_mps(c, std::move(h));
    });
}

mpspt_status mpspt_ground_state(mpspt_ctx* ctx, int M0, double s2_penalty, double* e_ref, mpspt_mps** psi0,
                                mpspt_report* rep) {
    if (!ctx || M0 < 1 || !(s2_penalty >= 0.0)) return MPSPT_ERR_INVALID;
    return guard(ctx, [&] {
        auto& c = *ctx->c;
        MPSPT_CUDA(cudaSetDevice(c.opt.device));
        mpspt::SweepResult r;
        std::unique_ptr<mpspt::MpsD> m = mpspt::ground_state(c, M0, s2_penalty, r);
        if (rep) fill_report(rep, r);
        if (e_ref) *e_ref = c.P.e_ref;
        if (psi0) {
            auto* h = new mpspt_mps;
            h->m = std::move(m);
            h->st = c.st;
            h->device = c.opt.device;
            *psi0 = h;
        }
    });
}

mpspt_status mpspt_energies(mpspt_ctx* ctx, mpspt_h0 h0, double* e0, double* e1, double* e_ref) {
    if (!ctx) return MPSPT_ERR_INVALID;
    return guard(ctx, [&] {
        auto& c = *ctx->c;
        mpspt::require(c.P.have_ref, "mpspt_set_reference must come first", MPSPT_ERR_STATE);
        mpspt::require(h0 == MPSPT_H0_FOCK || h0 == MPSPT_H0_DYALL, "unknown H0");
        const double E0 = c.e0(h0);
        if (e0) *e0 = E0;
        if (e1) *e1 = c.P.e_ref - E0;
        if (e_ref) *e_ref = c.P.e_ref;
    });
}


mpspt_status mpspt_minimize_hylleraas(mpspt_ctx* ctx, mpspt_h0 h0, int M, double* e2, mpspt_mps** psi1,
                                      mpspt_report* rep) {
    if (!ctx || !e2) return MPSPT_ERR_INVALID;
    return guard(ctx, [&] {
        auto& c = *ctx->c;
        MPSPT_CUDA(cudaSetDevice(c.opt.device));
        mpspt::SweepResult r;
        std::unique_ptr<mpspt::MpsD> m = mpspt::minimize(c, h0, M, r);
        if (rep) fill_report(rep, r);
        *e2 = r.e2;
        if (psi1) {
            auto* h = new mpspt_mps;
            h->m = std::move(m);
            h->st = c.st;
            h->device = c.opt.device;
            *psi1 = h;
        }
    });
}


mpspt_status mpspt_extrapolate_e2(mpspt_ctx* ctx, mpspt_h0 h0, int n_M, const int* M, double* e2_M, double* w_M,
                                  double* e2_extrap, double* slope) {
    if (!ctx || n_M < 2 || !M || !e2_extrap || !slope) return MPSPT_ERR_INVALID;
    return guard(ctx, [&] {
        auto& c = *ctx->c;
        MPSPT_CUDA(cudaSetDevice(c.opt.device));
        std::vector<double> e(n_M), w(n_M);
        for (int j = 0; j < n_M; ++j) {
            mpspt::require(M[j] >= 1, "bond dimensions must be >= 1");
            mpspt::SweepResult r;
            mpspt::minimize(c, h0, M[j], r);
            e[j] = r.e2;
            w[j] = r.max_disc;
        }
        // least squares line e = a + b w (centred sums, float64)
        double mw = 0.0, me = 0.0;
        for (int j = 0; j < n_M; ++j) { mw += w[j]; me += e[j]; }
        mw /= n_M;
        me /= n_M;
        double sww = 0.0, swe = 0.0;
        for (int j = 0; j < n_M; ++j) { sww += (w[j] - mw) * (w[j] - mw); swe += (w[j] - mw) * (e[j] - me); }
        mpspt::require(sww > 0.0, "the discarded weights are all equal: no line to fit");
        const double b = swe / sww;
        if (e2_M) for (int j = 0; j < n_M; ++j) e2_M[j] = e[j];
        if (w_M) for (int j = 0; j < n_M; ++j) w_M[j] = w[j];
        *slope = b;
        *e2_extrap = me - b * mw;
    });
}

mpspt_status mpspt_minimize_partitioned(mpspt_ctx* ctx, mpspt_h0 h0, int n_part, const int* pair_ab,
                                        const int* M_part, int n_streams, double* e2_total, double* e2_part,
                                        mpspt_report* rep) {
    if (!ctx || !e2_total || n_part < 1 || !pair_ab || !M_part) return MPSPT_ERR_INVALID;
    return guard(ctx, [&] {
        auto& c = *ctx->c;
        MPSPT_CUDA(cudaSetDevice(c.opt.device));
        std::vector<std::pair<int, int>> pairs(n_part);
        std::vector<int> Ms(M_part, M_part + n_part);
        for (int i = 0; i < n_part; ++i) pairs[i] = {pair_ab[2 * i], pair_ab[2 * i + 1]};
        std::vector<double> ep;
        mpspt::SweepResult r;
        const double tot = mpspt::minimize_partitioned(c, h0, pairs, Ms, n_streams > 0 ? n_streams : 8, ep, r);
        if (rep) fill_report(rep, r);
        if (e2_part) for (int i = 0; i < n_part; ++i) e2_part[i] = ep[i];
        *e2_total = tot;
    });
}

mpspt_status mpspt_third_order_partitioned(mpspt_ctx* ctx, mpspt_h0 h0, int n_part, const int* pair_ab,
                                           const int* M_part, int n_streams, double* e2_total,
                                           double* e3_total, double* e3_cross, double* e2_part,
                                           double* e3_part, double* h_pair, mpspt_report* rep) {
    if (!ctx || !e2_total || !e3_total || !e3_cross || n_part < 1 || !pair_ab || !M_part)
        return MPSPT_ERR_INVALID;
    return guard(ctx, [&] {
        auto& c = *ctx->c;
        MPSPT_CUDA(cudaSetDevice(c.opt.device));
        std::vector<std::pair<int, int>> pairs(n_part);
        std::vector<int> Ms(M_part, M_part + n_part);
        for (int i = 0; i < n_part; ++i) pairs[i] = {pair_ab[2 * i], pair_ab[2 * i + 1]};
        mpspt::PartE3 o;
        mpspt::SweepResult r;
        mpspt::third_order_partitioned(c, h0, pairs, Ms, n_streams > 0 ? n_streams : 8, o, r);
        if (rep) {
            fill_report(rep, r);
            rep->e3_ms = o.e3_ms;
            rep->e3_transfers = o.transfers;
            rep->e3_wait_ms = o.wait_ms;
            rep->e3_flops = o.flops;
            rep->e3_plan_bytes = o.plan_bytes;
            rep->e3_setup_ms = o.setup_ms;
        }
        if (e2_part) for (int i = 0; i < n_part; ++i) e2_part[i] = o.e2_part[i];
        if (e3_part) for (int i = 0; i < n_part; ++i) e3_part[i] = o.e3_part[i];
        if (h_pair) std::copy(o.h_pair.begin(), o.h_pair.end(), h_pair);
        *e2_total = o.e2;
        *e3_total = o.e3;
        *e3_cross = o.e3_cross;
    });
}

mpspt_status mpspt_third_order(mpspt_ctx* ctx, mpspt_h0 h0, const mpspt_mps* psi1, double* e3) {
    if (!ctx || !psi1 || !e3) return MPSPT_ERR_INVALID;
    return guard(ctx, [&] {
        auto& c = *ctx->c;
        MPSPT_CUDA(cudaSetDevice(c.opt.device));
        mpspt::require(h0 == MPSPT_H0_FOCK || h0 == MPSPT_H0_DYALL, "unknown H0");
        mpspt::require(psi1->m->nsite == c.P.k, "MPS length differs from the orbital count");
        *e3 = mpspt::third_order(c, h0, *psi1->m);
    });
}

void mpspt_mps_free(mpspt_mps* mps) {
    if (!mps) return;
    cudaSetDevice(mps->device);
    delete mps;
}

mpspt_status mpspt_mps_import(mpspt_ctx* ctx, int nsite, const int* bond_dims, const int* bond_qn,
                              const double* const* tensors, mpspt_mps** out) {
    if (!ctx || !bond_dims || !bond_qn || !tensors || !out || nsite < 1) return MPSPT_ERR_INVALID;
    return guard(ctx, [&] {
        auto& c = *ctx->c;
        MPSPT_CUDA(cudaSetDevice(c.opt.device));
        mpspt::MpsHost h;
        h.nsite = nsite;
        h.bond.resize(nsite + 1);
        const int* q = bond_qn;
        for (int cut = 0; cut <= nsite; ++cut) {
            const int D = bond_dims[cut];
            mpspt::require(D >= 1, "bond dimensions must be >= 1");
            mpspt::Bond& b = h.bond[cut];
            for (int i = 0; i < D; ++i, q += 2) {
                mpspt::QN qq(q[0], q[1]);
                if (b.sec.empty() || !(b.sec.back().q == qq)) {
                    mpspt::require(b.sec.empty() || b.sec.back().q < qq,
                                   "bond QN sectors must be contiguous and ascending");
                    b.sec.push_back({qq, 0, 0});
                }
                b.sec.back().dim++;
            }
            b.finalize();
        }
        h.T.resize(nsite);
        for (int s = 0; s < nsite; ++s) {
            const size_t n = (size_t)bond_dims[s] * 4 * bond_dims[s + 1];
            mpspt::require(tensors[s] != nullptr, "null tensor");
            h.T[s].assign(tensors[s], tensors[s] + n);
            for (double v : h.T[s]) mpspt::require(std::isfinite(v), "non-finite MPS entry");
        }
        auto* m = new mpspt_mps;
        m->m = mpspt::mps_upload(h, c.st);
        m->st = c.st;
        m->device = c.opt.device;
        *out = m;
    });
}

mpspt_status mpspt_mps_shape(const mpspt_mps* mps, int* nsite, int* bond_dims) {
    if (!mps) return MPSPT_ERR_INVALID;
    if (nsite) *nsite = mps->m->nsite;
    if (bond_dims)
        for (int c = 0; c <= mps->m->nsite; ++c) bond_dims[c] = mps->m->bond[c].total;
    return MPSPT_OK;
}

mpspt_status mpspt_mps_export(const mpspt_mps* mps, int* bond_qn, double* const* tensors) {
    if (!mps || !tensors) return MPSPT_ERR_INVALID;
    return guard(nullptr, [&] {
        MPSPT_CUDA(cudaSetDevice(mps->device));
        mpspt::MpsHost h = mpspt::mps_download(*mps->m, mps->st);
        if (bond_qn) {
            int* q = bond_qn;
            for (const auto& b : h.bond)
                for (const auto& s : b.sec)
                    for (int i = 0; i < s.dim; ++i) { *q++ = s.q.n; *q++ = s.q.sz; }
        }
        for (int s = 0; s < h.nsite; ++s) std::memcpy(tensors[s], h.T[s].data(), h.T[s].size() * sizeof(double));
    });
}

mpspt_status mpspt_local_apply(mpspt_ctx* ctx, mpspt_h0 h0, const mpspt_mps* psi1, int i,
                               mpspt_local_op op, const double* x, double* out) {
    if (!ctx || !psi1 || !out) return MPSPT_ERR_INVALID;
    if (op == MPSPT_LOCAL_SIGMA && !x) return MPSPT_ERR_INVALID;
    return guard(ctx, [&] {
        auto& c = *ctx->c;
        MPSPT_CUDA(cudaSetDevice(c.opt.device));
        mpspt::require(h0 == MPSPT_H0_FOCK || h0 == MPSPT_H0_DYALL, "unknown H0");
        mpspt::local_apply(c, h0, *psi1->m, i, op, x, out);
    });
}

mpspt_status mpspt_eigh_batched(int device, void* stream, int batch, const int* n, const double* A,
                                double* V, double* w) {
    if (batch < 1 || !n || !A || !V || !w) return MPSPT_ERR_INVALID;
    return guard(nullptr, [&] {
        MPSPT_CUDA(cudaSetDevice(device));
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        size_t tot = 0, totw = 0;
        for (int i = 0; i < batch; ++i) {
            mpspt::require(n[i] >= 1 && n[i] <= 2048, "matrix size must be in [1, 2048]");
            tot += (size_t)n[i] * n[i];
            totw += (size_t)n[i];
        }
        mpspt::DBuf work(tot * sizeof(double), st), dt;
        MPSPT_CUDA(cudaMemcpyAsync(work.get(), A, tot * sizeof(double), cudaMemcpyDeviceToDevice, st));
        std::vector<mpspt::EigTask> tasks(batch);
        size_t o = 0, ow = 0;
        for (int i = 0; i < batch; ++i) {
            tasks[i] = {work.as<double>() + o, V + o, w + ow, n[i], 0};
            o += (size_t)n[i] * n[i];
            ow += (size_t)n[i];
        }
        mpspt::upload(dt, tasks, st);
        mpspt::launch_eig(dt.as<mpspt::EigTask>(), batch, st);
        MPSPT_CUDA(cudaGetLastError());
    });
}

mpspt_status mpspt_eigh_batched_ex(int device, void* stream, int batch, const int* n, const double* A,
                                   double* V, double* w, int f32_start) {
    if (batch < 1 || !n || !A || !V || !w) return MPSPT_ERR_INVALID;
    return guard(nullptr, [&] {
        MPSPT_CUDA(cudaSetDevice(device));
        mpspt::keep_pool_memory(device);
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        size_t tot = 0, totw = 0;
        for (int i = 0; i < batch; ++i) {
            mpspt::require(n[i] >= 1 && n[i] <= 2048, "matrix size must be in [1, 2048]");
            tot += (size_t)n[i] * n[i];
            totw += (size_t)n[i];
        }
        mpspt::DBuf wa(tot * sizeof(double), st), wv(tot * sizeof(double), st), ww(totw * sizeof(double), st);
        MPSPT_CUDA(cudaMemcpyAsync(wa.get(), A, tot * sizeof(double), cudaMemcpyDeviceToDevice, st));
        std::vector<mpspt::EigTask> tasks(batch);
        size_t o = 0, ow = 0;
        for (int i = 0; i < batch; ++i) {
            tasks[i] = {wa.as<double>() + o, wv.as<double>() + o, ww.as<double>() + ow, n[i], 0};
            o += (size_t)n[i] * n[i];
            ow += (size_t)n[i];
        }
        mpspt::EigSolver es;
        es.run(tasks, f32_start == 0, st);
        MPSPT_CUDA(cudaMemcpyAsync(V, wv.get(), tot * sizeof(double), cudaMemcpyDeviceToDevice, st));
        MPSPT_CUDA(cudaMemcpyAsync(w, ww.get(), totw * sizeof(double), cudaMemcpyDeviceToDevice, st));
        std::vector<int> fl(es.nflags);
        if (es.nflags)
            MPSPT_CUDA(cudaMemcpyAsync(fl.data(), es.flags.get(), es.nflags * sizeof(int), cudaMemcpyDeviceToHost, st));
        MPSPT_CUDA(cudaStreamSynchronize(st));   // the solver's scratch is released on return
        MPSPT_CUDA(cudaGetLastError());
        for (int f : fl)
            mpspt::require(f != 2, "Jacobi sweep cap reached before the convergence test", MPSPT_ERR_NOT_CONVERGED);
    });
}

mpspt_status mpspt_mlp_create(int device, int width, unsigned long long seed, mpspt_mlp** out) {
    if (!out || width < 1) return MPSPT_ERR_INVALID;
    return guard(nullptr, [&] {
        MPSPT_CUDA(cudaSetDevice(device));
        auto* h = new mpspt_mlp;
        h->device = device;
        try {
            h->m.reset(new mpspt::Mlp(mpspt::MLP_NF, width, 2, seed, 0));
        } catch (...) {
            delete h;
            throw;
        }
        *out = h;
    });
}

void mpspt_mlp_free(mpspt_mlp* net) {
    if (!net) return;
    cudaSetDevice(net->device);
    delete net;
}

mpspt_status mpspt_mlp_set_params(mpspt_mlp* net, const float* W1, const float* b1, const float* W2,
                                  const float* b2, const float* W3, const float* b3) {
    if (!net || !W1 || !b1 || !W2 || !b2 || !W3 || !b3) return MPSPT_ERR_INVALID;
    return guard(nullptr, [&] {
        MPSPT_CUDA(cudaSetDevice(net->device));
        const float* W[3] = {W1, W2, W3};
        const float* b[3] = {b1, b2, b3};
        net->m->set_params(W, b);
    });
}

mpspt_status mpspt_mlp_get_params(const mpspt_mlp* net, float* W1, float* b1, float* W2, float* b2,
                                  float* W3, float* b3) {
    if (!net || !W1 || !b1 || !W2 || !b2 || !W3 || !b3) return MPSPT_ERR_INVALID;
    return guard(nullptr, [&] {
        MPSPT_CUDA(cudaSetDevice(net->device));
        float* W[3] = {W1, W2, W3};
        float* b[3] = {b1, b2, b3};
        net->m->get_params(W, b);
    });
}

mpspt_status mpspt_mlp_forward(mpspt_mlp* net, int batch, const float* x, float* y) {
    if (!net || batch < 1 || !x || !y) return MPSPT_ERR_INVALID;
    return guard(nullptr, [&] {
        MPSPT_CUDA(cudaSetDevice(net->device));
        auto& m = *net->m;
        std::vector<float> xs(x, x + (size_t)batch * m.nin);
        mpspt::DBuf X, Y((size_t)batch * m.nout * sizeof(float) + 16, m.st);
        mpspt::upload(X, xs, m.st);
        m.forward(batch, X.as<float>(), Y.as<float>());
        MPSPT_CUDA(cudaMemcpyAsync(y, Y.get(), (size_t)batch * m.nout * sizeof(float), cudaMemcpyDeviceToHost, m.st));
        MPSPT_CUDA(cudaStreamSynchronize(m.st));
    });
}

mpspt_status mpspt_mlp_gradient(mpspt_mlp* net, int batch, const float* x, const float* t, float* loss,
                                float* gW1, float* gb1, float* gW2, float* gb2, float* gW3, float* gb3) {
    if (!net || batch < 1 || !x || !t) return MPSPT_ERR_INVALID;
    return guard(nullptr, [&] {
        MPSPT_CUDA(cudaSetDevice(net->device));
        auto& m = *net->m;
        std::vector<float> xs(x, x + (size_t)batch * m.nin), ts(t, t + (size_t)batch * m.nout);
        mpspt::DBuf X, T;
        mpspt::upload(X, xs, m.st);
        mpspt::upload(T, ts, m.st);
        const float l = m.gradient(batch, X.as<float>(), T.as<float>());
        if (loss) *loss = l;
        float* gw[3] = {gW1, gW2, gW3};
        float* gb[3] = {gb1, gb2, gb3};
        for (int q = 0; q < 3; ++q) {
            if (gw[q]) MPSPT_CUDA(cudaMemcpyAsync(gw[q], m.gW[q].get(), m.wn(q) * sizeof(float), cudaMemcpyDeviceToHost, m.st));
            if (gb[q]) MPSPT_CUDA(cudaMemcpyAsync(gb[q], m.gb[q].get(), m.out_of(q) * sizeof(float), cudaMemcpyDeviceToHost, m.st));
        }
        MPSPT_CUDA(cudaStreamSynchronize(m.st));
    });
}

mpspt_status mpspt_mlp_train(mpspt_mlp* net, int n, const float* x, const float* t, int epochs, int batch,
                             float lr, float* loss) {
    if (!net || n < 1 || !x || !t || epochs < 1 || batch < 1 || !(lr > 0)) return MPSPT_ERR_INVALID;
    return guard(nullptr, [&] {
        MPSPT_CUDA(cudaSetDevice(net->device));
        const float l = net->m->train(n, x, t, epochs, batch, lr);
        if (loss) *loss = l;
    });
}

mpspt_status mpspt_harvest(mpspt_ctx* ctx, mpspt_h0 h0, int M, int max_samples, float* x, float* t,
                           int* n_samples) {
    if (!ctx || max_samples < 1 || !x || !t || !n_samples) return MPSPT_ERR_INVALID;
    return guard(ctx, [&] {
        auto& c = *ctx->c;
        MPSPT_CUDA(cudaSetDevice(c.opt.device));
        c.harvesting = true;
        c.harvest_max = (size_t)max_samples;
        c.harvest_x.clear();
        c.harvest_t.clear();
        mpspt::SweepResult r;
        try {
            mpspt::minimize(c, h0, M, r);
        } catch (...) {
            c.harvesting = false;
            throw;
        }
        c.harvesting = false;
        const int ns = (int)(c.harvest_x.size() / mpspt::MLP_NF);
        std::copy(c.harvest_x.begin(), c.harvest_x.end(), x);
        std::copy(c.harvest_t.begin(), c.harvest_t.end(), t);
        *n_samples = ns;
    });
}

mpspt_status mpspt_train_preconditioner(mpspt_ctx* ctx, mpspt_h0 h0, int M, int max_samples, int epochs,
                                        const char* harvest_path, float* loss) {
    if (!ctx || M < 1 || max_samples < 1 || epochs < 1) return MPSPT_ERR_INVALID;
    return guard(ctx, [&] {
        auto& c = *ctx->c;
        MPSPT_CUDA(cudaSetDevice(c.opt.device));
        std::vector<float> x, t;
        bool loaded = false;
        if (harvest_path) {
            if (FILE* f = std::fopen(harvest_path, "rb")) {
                int n = 0;
                bool ok = std::fread(&n, sizeof(int), 1, f) == 1 && n > 0;
                if (ok) {
                    x.resize((size_t)n * mpspt::MLP_NF);
                    t.resize((size_t)n * 2);
                    ok = std::fread(x.data(), sizeof(float), x.size(), f) == x.size() &&
                         std::fread(t.data(), sizeof(float), t.size(), f) == t.size();
                }
                std::fclose(f);
                mpspt::require(ok, "harvest file is truncated or empty");
                loaded = true;
            }
        }
        if (!loaded) {
            c.harvesting = true;
            c.harvest_max = (size_t)max_samples;
            c.harvest_x.clear();
            c.harvest_t.clear();
            mpspt::SweepResult r;
            try {
                mpspt::minimize(c, h0, M, r);
            } catch (...) {
                c.harvesting = false;
                throw;
            }
            c.harvesting = false;
            x.swap(c.harvest_x);
            t.swap(c.harvest_t);
            mpspt::require(!x.empty(), "the sweep gave no training pairs");
            if (harvest_path) {
                FILE* f = std::fopen(harvest_path, "wb");
                mpspt::require(f != nullptr, "cannot write the harvest file");
                const int n = (int)(x.size() / mpspt::MLP_NF);
                const bool ok = std::fwrite(&n, sizeof(int), 1, f) == 1 &&
                                std::fwrite(x.data(), sizeof(float), x.size(), f) == x.size() &&
                                std::fwrite(t.data(), sizeof(float), t.size(), f) == t.size();
                std::fclose(f);
                mpspt::require(ok, "cannot write the harvest file");
            }
        }
        const int n = (int)(x.size() / mpspt::MLP_NF);
        std::unique_ptr<mpspt::Mlp> net(new mpspt::Mlp(mpspt::MLP_NF, 256, 2, c.opt.seed, 0));
        const float l = net->train(n, x.data(), t.data(), epochs, 256, 1e-3f);
        c.own_net = std::move(net);
        c.net = c.own_net.get();
        if (loss) *loss = l;
    });
}

mpspt_status mpspt_set_preconditioner(mpspt_ctx* ctx, const mpspt_mlp* net) {
    if (!ctx) return MPSPT_ERR_INVALID;
    ctx->c->net = net ? net->m.get() : nullptr;
    return MPSPT_OK;
}

const char* mpspt_status_string(mpspt_status s) {
    switch (s) {
        case MPSPT_OK: return "ok";
        case MPSPT_ERR_INVALID: return g_last.empty() ? "invalid argument" : g_last.c_str();
        case MPSPT_ERR_OOM: return "out of memory";
        case MPSPT_ERR_NOT_SPD: return g_last.empty() ? "H0 - E0 not positive definite on the local space" : g_last.c_str();
        case MPSPT_ERR_NOT_CONVERGED: return g_last.empty() ? "iteration limit reached" : g_last.c_str();
        case MPSPT_ERR_TIMEOUT: return "bounded device wait timed out";
        case MPSPT_ERR_CUDA: return g_last.empty() ? "CUDA error" : g_last.c_str();
        case MPSPT_ERR_STATE: return g_last.empty() ? "call out of order" : g_last.c_str();
    }
    return "unknown status";
}

}  // extern "C"
