// C ABI of the MPS-PT library: argument checks, exception barrier, handles.
#include <cmath>
#include <cstring>

#include "engine.h"

struct mpspt_ctx {
    std::unique_ptr<mpspt::Ctx> c;
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
}

mpspt_status mpspt_create(mpspt_ctx** ctx, const mpspt_options* opt) {
    if (!ctx) return MPSPT_ERR_INVALID;
    mpspt_options o;
    mpspt_default_options(&o);
    if (opt) o = *opt;
    return guard(nullptr, [&] {
        mpspt::require(o.max_sweeps >= 1 && o.cg_max_iter >= 1 && o.cg_tol > 0 && o.e_tol > 0,
                       "invalid options");
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

mpspt_status mpspt_set_reference(mpspt_ctx* ctx, const double* ci, long long n_ci) {
    if (!ctx) return MPSPT_ERR_INVALID;
    return guard(ctx, [&] {
        MPSPT_CUDA(cudaSetDevice(ctx->c->opt.device));
        mpspt::set_reference(*ctx->c, ci, n_ci);
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
        if (rep) {
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
            for (int s = 0; s < rep->n_sweeps && s < 64; ++s) rep->sweep_ms[s] = r.sweep_ms[s];
            rep->kernel_launches = r.launches;
            rep->sigma64_calls = r.sigma64_calls;
            rep->sigma64_flops = r.sigma64_flops;
            rep->sigma64_ms = r.sigma64_ms;
        }
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
}
}  // namespace

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

const char* mpspt_status_string(mpspt_status s) {
    switch (s) {
        case MPSPT_OK: return "ok";
        case MPSPT_ERR_INVALID: return g_last.empty() ? "invalid argument" : g_last.c_str();
        case MPSPT_ERR_OOM: return "out of memory";
        case MPSPT_ERR_NOT_SPD: return "H0 - E0 not positive definite on the local space";
        case MPSPT_ERR_NOT_CONVERGED: return "iteration limit reached";
        case MPSPT_ERR_TIMEOUT: return "bounded device wait timed out";
        case MPSPT_ERR_CUDA: return g_last.empty() ? "CUDA error" : g_last.c_str();
        case MPSPT_ERR_STATE: return g_last.empty() ? "call out of order" : g_last.c_str();
    }
    return "unknown status";
}

}  // extern "C"
