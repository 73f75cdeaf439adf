// MPS-PT engine (host orchestration; device kernels do the contractions).
#include "engine.h"
#include "eig.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>

#include "hostla.h"

#include <nvtx3/nvToolsExt.h>

namespace mpspt {

// ------------------------------------------------------------------ context
Lane::Lane(cudaStream_t s, bool create) : st(s), own_stream(create) {
    if (create) MPSPT_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    red.alloc(4 * 1024 * sizeof(double), st);
    cnt.alloc(64, st);
    MPSPT_CUDA(cudaMemsetAsync(cnt.get(), 0, 64, st));
    cg.alloc(sizeof(CgState), st);
    scal.alloc(16 * sizeof(double), st);
    tcerr.alloc(sizeof(int) * 4, st);
    MPSPT_CUDA(cudaMemsetAsync(tcerr.get(), 0, sizeof(int) * 4, st));
    MPSPT_CUDA(cudaMallocHost(&cg_host, sizeof(CgState)));
    MPSPT_CUDA(cudaMallocHost(&scal_host, 16 * sizeof(double)));
    ring.reset(new PinnedRing((size_t)16 << 20, st));
    MPSPT_CUDA(cudaStreamSynchronize(st));
}

void* Lane::readback(size_t bytes) {
    if (bytes > rb_bytes) {
        MPSPT_CUDA(cudaStreamSynchronize(st));
        if (rb) cudaFreeHost(rb);
        rb = nullptr;
        rb_bytes = 0;
        const size_t nb = std::max(bytes, (size_t)1 << 20);
        MPSPT_CUDA(cudaMallocHost(&rb, nb));
        rb_bytes = nb;
    }
    return rb;
}

Lane::~Lane() {
    cudaStreamSynchronize(st);
    ring.reset();
    if (rb) cudaFreeHost(rb);
    red.release(); cnt.release(); cg.release(); scal.release(); tcerr.release();
    cudaStreamSynchronize(st);
    if (cg_host) cudaFreeHost(cg_host);
    if (scal_host) cudaFreeHost(scal_host);
    if (own_stream) cudaStreamDestroy(st);
}

Ctx::Ctx(const mpspt_options& o) : opt(o) {
    MPSPT_CUDA(cudaSetDevice(o.device));
    keep_pool_memory(o.device);
    st = static_cast<cudaStream_t>(o.stream);
    lane0.reset(new Lane(st));
    red.alloc(4 * 1024 * sizeof(double), st);
    cnt.alloc(64, st);
    MPSPT_CUDA(cudaMemsetAsync(cnt.get(), 0, 64, st));
    cg.alloc(sizeof(CgState), st);
    scal.alloc(16 * sizeof(double), st);
    tcerr.alloc(sizeof(int) * 4, st);
    MPSPT_CUDA(cudaMemsetAsync(tcerr.get(), 0, sizeof(int) * 4, st));
    MPSPT_CUDA(cudaMallocHost(&cg_host, sizeof(CgState)));
    MPSPT_CUDA(cudaMallocHost(&scal_host, 16 * sizeof(double)));
    if (o.autotune) {
        tuner.reset(new Autotuner);
        if (o.autotune_cache) {
            tuner_path = o.autotune_cache;
            tuner->load(tuner_path);
        }
    }
}

Ctx::~Ctx() {
    cudaStreamSynchronize(st);
    if (tuner && !tuner_path.empty()) tuner->save(tuner_path);
    if (cg_host) cudaFreeHost(cg_host);
    if (scal_host) cudaFreeHost(scal_host);
}

double Ctx::e0(int h0) const {
    if (h0 == MPSPT_H0_DYALL) return P.e_ref;
    double s = 0.0;
    for (int t = 0; t < P.ka; ++t)
        for (int u = 0; u < P.ka; ++u) s += P.f[(size_t)t * P.k + u] * P.gamma[(size_t)t * P.ka + u];
    return s;
}

const MPO& Ctx::A_mpo(int h0) {
    auto it = mpoA.find(h0);
    if (it != mpoA.end()) return it->second;
    std::vector<Term> t;
    const int k = P.k, ka = P.ka;
    if (h0 == MPSPT_H0_DYALL) {
        add_one_body(t, P.h, k, 0, ka, 0, ka);
        add_two_body(t, P.eri, k, 0, ka, 0, ka, -1);
    } else {
        add_one_body(t, P.f, k, 0, ka, 0, ka);
    }
    add_number(t, P.eps, ka, k);
    Term c{-e0(h0), 0, {}};
    t.push_back(c);
    return mpoA[h0] = build_mpo(t, k, ka);
}

const MPO& Ctx::V_mpo() {
    auto it = mpoV.find(0);
    if (it != mpoV.end()) return it->second;
    std::vector<Term> t;
    const int k = P.k, ka = P.ka;
    add_one_body(t, P.h, k, ka, k, 0, ka);          // c+_a c_t
    add_two_body(t, P.eri, k, 0, k, 0, ka, ka);     // >= 1 virtual creator, active annihilators
    return mpoV[0] = build_mpo(t, k, ka);
}

const MPO& Ctx::H_mpo() {
    if (!mpoH) {
        std::vector<Term> t;
        add_one_body(t, P.h, P.k, 0, P.k, 0, P.k);
        add_two_body(t, P.eri, P.k, 0, P.k, 0, P.k, -1);
        mpoH.reset(new MPO(build_mpo(t, P.k, P.ka)));
    }
    return *mpoH;
}

const MPO& Ctx::I_mpo() {
    if (!mpoI) {
        std::vector<Term> t;
        t.push_back(Term{1.0, 0, {}});
        mpoI.reset(new MPO(build_mpo(t, P.k, P.ka)));
    }
    return *mpoI;
}

// ------------------------------------------------------------- integrals
void set_integrals(Ctx& c, int ka, int kv, int nel, const double* h, const double* L, int nq) {
    require(ka >= 1 && kv >= 0 && nq >= 1, "bad orbital / Cholesky dimensions");
    require(nel >= 2 && nel % 2 == 0 && nel <= 2 * ka, "n_elec must be even, 2 <= n_elec <= 2 k_act");
    require(ka <= 14, "k_act > 14 not supported by the dense reference input");
    require(h && L, "null integral array");
    const int k = ka + kv;
    Problem& P = c.P;
    P = Problem();
    P.k = k; P.ka = ka; P.kv = kv; P.nel = nel; P.nq = nq;
    P.h_in.assign(h, h + (size_t)k * k);
    P.L_in.assign(L, L + (size_t)nq * k * k);
    for (double v : P.h_in) require(std::isfinite(v), "non-finite one-electron integral");
    for (double v : P.L_in) require(std::isfinite(v), "non-finite Cholesky vector");
    for (int p = 0; p < k; ++p)
        for (int q = 0; q < p; ++q)
            require(std::fabs(P.h_in[(size_t)p * k + q] - P.h_in[(size_t)q * k + p]) < 1e-12,
                    "h must be symmetric");
    P.have_int = true;
    c.mpoA.clear(); c.mpoV.clear(); c.mpoH.reset(); c.mpoI.reset();
}

namespace {

// Occupation-string helpers on the 4^ka active space (site 0 most significant).
inline int code_at(long long idx, int p, int ka) { return (int)((idx >> (2 * (ka - 1 - p))) & 3); }

// c_j or c+_j (j = 2p + s) on a string; returns -1 if it vanishes.
inline long long apply1(long long idx, int j, bool dag, int ka, int& sign) {
    const int p = j / 2, s = j % 2;
    const int code = code_at(idx, p, ka);
    const int bit = 1 << s;
    if (dag == ((code & bit) != 0)) return -1;
    int below = 0;
    for (int q = 0; q < p; ++q) below += __builtin_popcount(code_at(idx, q, ka));
    if (s == 1) below += code & 1;
    if (below & 1) sign = -sign;
    const int nc = code ^ bit;
    const int sh = 2 * (ka - 1 - p);
    return (idx & ~(3LL << sh)) | ((long long)nc << sh);
}

void one_rdm_and_energy(Problem& P) {
    const int ka = P.ka, k = P.k;
    const long long n = 1LL << (2 * ka);
    std::vector<long long> nz;
    for (long long i = 0; i < n; ++i) if (P.ci[i] != 0.0) nz.push_back(i);
    P.gamma.assign((size_t)ka * ka, 0.0);
    double e1 = 0.0, e2 = 0.0;
    for (long long d : nz) {
        const double cd = P.ci[d];
        for (int s = 0; s < 2; ++s)
            for (int u = 0; u < ka; ++u) {
                int sg1 = 1;
                long long d1 = apply1(d, 2 * u + s, false, ka, sg1);
                if (d1 < 0) continue;
                for (int t = 0; t < ka; ++t) {
                    int sg2 = sg1;
                    long long d2 = apply1(d1, 2 * t + s, true, ka, sg2);
                    if (d2 < 0) continue;
                    P.gamma[(size_t)t * ka + u] += P.ci[d2] * cd * sg2;
                }
                // two-body: 1/2 (tu|vw) c+_ts c+_vr c_wr c_us
                for (int r = 0; r < 2; ++r)
                    for (int w = 0; w < ka; ++w) {
                        int sg2 = sg1;
                        long long d2 = apply1(d1, 2 * w + r, false, ka, sg2);
                        if (d2 < 0) continue;
                        for (int v = 0; v < ka; ++v) {
                            int sg3 = sg2;
                            long long d3 = apply1(d2, 2 * v + r, true, ka, sg3);
                            if (d3 < 0) continue;
                            for (int t = 0; t < ka; ++t) {
                                int sg4 = sg3;
                                long long d4 = apply1(d3, 2 * t + s, true, ka, sg4);
                                if (d4 < 0) continue;
                                const double g = P.eri[(((size_t)t * k + u) * k + v) * k + w];
                                e2 += 0.5 * g * P.ci[d4] * cd * sg4;
                            }
                        }
                    }
            }
    }
    for (int t = 0; t < ka; ++t)
        for (int u = 0; u < ka; ++u) e1 += P.h[(size_t)t * k + u] * P.gamma[(size_t)t * ka + u];
    P.e_ref = e1 + e2;
}

void build_eri(Problem& P) {
    const int k = P.k;
    P.eri.assign((size_t)k * k * k * k, 0.0);
    for (int Q = 0; Q < P.nq; ++Q) {
        const double* Lq = &P.L[(size_t)Q * k * k];
        for (size_t pq = 0; pq < (size_t)k * k; ++pq) {
            const double a = Lq[pq];
            if (a == 0.0) continue;
            double* row = &P.eri[pq * k * k];
            for (size_t rs = 0; rs < (size_t)k * k; ++rs) row[rs] += a * Lq[rs];
        }
    }
}

// Exact QN-blocked MPS of a dense active-space vector (density-matrix form
// of the left-to-right SVD); keeps eigenvalues above keep_rel * max.
void ci_to_mps(const Problem& P, MpsHost& out) {
    const int ka = P.ka;
    out.nsite = ka;
    out.bond.assign(ka + 1, Bond());
    out.T.assign(ka, {});
    out.bond[0].sec.push_back({QN(0, 0), 1, 0});
    out.bond[0].finalize();
    std::vector<double> T(P.ci);      // Dl x R
    long long R = (long long)T.size();
    for (int c = 0; c < ka - 1; ++c) {
        const Bond& bl = out.bond[c];
        const int Dl = bl.total;
        const long long Rn = R / 4;
        // row (l, s) of X = T[l][s * Rn + rest]
        std::vector<QN> rq(Dl * 4);
        for (const auto& sec : bl.sec)
            for (int i = 0; i < sec.dim; ++i)
                for (int s = 0; s < 4; ++s) rq[(sec.off + i) * 4 + s] = sec.q + site_qn(s);
        std::map<QN, std::vector<int>> groups;
        for (int r = 0; r < Dl * 4; ++r) groups[rq[r]].push_back(r);
        struct Kept { QN q; std::vector<double> U; int nr; int nk; std::vector<int> rows; };
        std::vector<Kept> kept;
        for (auto& g : groups) {
            const auto& rows = g.second;
            const int nr = (int)rows.size();
            std::vector<double> rho((size_t)nr * nr, 0.0);
            for (int a = 0; a < nr; ++a) {
                const double* xa = &T[(size_t)(rows[a] / 4) * R + (size_t)(rows[a] % 4) * Rn];
                for (int b = a; b < nr; ++b) {
                    const double* xb = &T[(size_t)(rows[b] / 4) * R + (size_t)(rows[b] % 4) * Rn];
                    double s = 0.0;
                    for (long long z = 0; z < Rn; ++z) s += xa[z] * xb[z];
                    rho[(size_t)a * nr + b] = rho[(size_t)b * nr + a] = s;
                }
            }
            std::vector<double> w, V;
            jacobi_eigh(nr, rho, w, V);
            double wmax = 0.0;
            for (double v : w) wmax = std::max(wmax, v);
            Kept kp{g.first, {}, nr, 0, rows};
            for (int j = nr - 1; j >= 0; --j) {
                if (!(w[j] > 1e-14 * wmax) || w[j] <= 0.0) continue;
                for (int a = 0; a < nr; ++a) kp.U.push_back(V[(size_t)a * nr + j]);  // column-major store
                kp.nk++;
            }
            if (kp.nk) kept.push_back(std::move(kp));
        }
        Bond nb;
        for (auto& kp : kept) nb.sec.push_back({kp.q, kp.nk, 0});
        nb.finalize();
        std::vector<double> A((size_t)Dl * 4 * nb.total, 0.0);
        std::vector<double> Tn((size_t)nb.total * Rn, 0.0);
        for (size_t si = 0; si < kept.size(); ++si) {
            const auto& kp = kept[si];
            const int off = nb.sec[si].off;
            for (int j = 0; j < kp.nk; ++j) {
                for (int a = 0; a < kp.nr; ++a) {
                    const double u = kp.U[(size_t)j * kp.nr + a];
                    const int row = kp.rows[a];
                    A[(size_t)row * nb.total + off + j] = u;
                    const double* xa = &T[(size_t)(row / 4) * R + (size_t)(row % 4) * Rn];
                    double* tn = &Tn[(size_t)(off + j) * Rn];
                    for (long long z = 0; z < Rn; ++z) tn[z] += u * xa[z];
                }
            }
        }
        out.T[c] = std::move(A);
        out.bond[c + 1] = nb;
        T.swap(Tn);
        R = Rn;
    }
    // last site
    const Bond& bl = out.bond[ka - 1];
    const QN tot(P.nel, 0);
    Bond last;
    last.sec.push_back({tot, 1, 0});
    last.finalize();
    std::vector<double> A((size_t)bl.total * 4, 0.0);
    for (const auto& sec : bl.sec)
        for (int i = 0; i < sec.dim; ++i)
            for (int s = 0; s < 4; ++s)
                if (sec.q + site_qn(s) == tot) A[(size_t)(sec.off + i) * 4 + s] = T[(size_t)(sec.off + i) * 4 + s];
    out.T[ka - 1] = std::move(A);
    out.bond[ka] = last;
}

}  // namespace

void set_reference(Ctx& c, const double* ci, long long n) {
    Problem& P = c.P;
    require(P.have_int, "mpspt_set_integrals must come first", MPSPT_ERR_STATE);
    require(ci != nullptr && n == (1LL << (2 * P.ka)), "n_ci must equal 4^k_act");
    P.ci.assign(ci, ci + n);
    double nrm = 0.0;
    for (double v : P.ci) { require(std::isfinite(v), "non-finite CI coefficient"); nrm += v * v; }
    require(nrm > 0.0, "zero reference vector");
    nrm = std::sqrt(nrm);
    for (double& v : P.ci) v /= nrm;
    // QN check: every nonzero string has N = n_elec, Sz = 0
    for (long long i = 0; i < n; ++i) {
        if (P.ci[i] == 0.0) continue;
        int nn = 0, sz = 0;
        for (int p = 0; p < P.ka; ++p) { int cd = code_at(i, p, P.ka); nn += __builtin_popcount(cd); sz += (cd & 1) - ((cd >> 1) & 1); }
        require(nn == P.nel && sz == 0, "reference has components outside (N, Sz = 0)");
    }
    P.h = P.h_in;
    P.L = P.L_in;
    build_eri(P);
    one_rdm_and_energy(P);      // gamma, E_ref (active block, untouched by the rotation)
    MpsHost act;
    ci_to_mps(P, act);
    finish_reference(c, act);
}

namespace {
// H_act on the k_act active sites (orbital index = site index): the terms of
// H with all indices active, from the integrals in the input basis.
std::vector<Term> active_hamiltonian_terms(const Problem& P) {
    const int k = P.k, ka = P.ka;
    std::vector<double> ha((size_t)ka * ka), ea((size_t)ka * ka * ka * ka);
    for (int p = 0; p < ka; ++p)
        for (int q = 0; q < ka; ++q) {
            ha[(size_t)p * ka + q] = P.h_in[(size_t)p * k + q];
            for (int r = 0; r < ka; ++r)
                for (int t = 0; t < ka; ++t) {
                    double v = 0.0;
                    for (int Q = 0; Q < P.nq; ++Q)
                        v += P.L_in[((size_t)Q * k + p) * k + q] * P.L_in[((size_t)Q * k + r) * k + t];
                    ea[(((size_t)p * ka + q) * ka + r) * ka + t] = v;
                }
        }
    std::vector<Term> th;
    add_one_body(th, ha, ka, 0, ka, 0, ka);
    add_two_body(th, ea, ka, 0, ka, 0, ka, -1);
    return th;
}

// Structure checks of an active-space reference MPS.
void check_reference_mps(const Problem& P, const MpsHost& act) {
    require(act.nsite == P.ka, "reference MPS must have k_act sites");
    require((int)act.bond.size() == P.ka + 1 && (int)act.T.size() == P.ka, "reference MPS: bond / tensor count");
    const Bond &b0 = act.bond[0], &b1 = act.bond[P.ka];
    require(b0.nsec() == 1 && b0.sec[0].q == QN(0, 0) && b0.total == 1, "reference MPS: first bond must be (0, 0), dim 1");
    require(b1.nsec() == 1 && b1.sec[0].q == QN(P.nel, 0) && b1.total == 1,
            "reference MPS: last bond must be (n_elec, 0), dim 1");
    for (int s = 0; s < P.ka; ++s) {
        require(act.T[s].size() == (size_t)act.bond[s].total * 4 * act.bond[s + 1].total, "reference MPS: tensor size");
        for (double v : act.T[s]) require(std::isfinite(v), "non-finite reference MPS entry");
    }
}
}  // namespace

void set_reference_mps(Ctx& c, MpsHost act) {
    Problem& P = c.P;
    require(P.have_int, "mpspt_set_integrals must come first", MPSPT_ERR_STATE);
    check_reference_mps(P, act);
    const int ka = P.ka;
    P.ci.clear();
    P.h = P.h_in;
    P.L = P.L_in;
    build_eri(P);
    std::unique_ptr<MpsD> d = mps_upload(act, c.st);   // entries that break QN conservation are dropped here
    std::vector<Term> ti{Term{1.0, 0, {}}};
    const double nrm = expectation(c, build_mpo(ti, ka, ka), *d, *d);
    require(std::isfinite(nrm) && nrm > 0.0, "reference MPS has zero norm");
    // gamma_tu = <c+_t c_u> (spin summed); real wavefunction: symmetric
    P.gamma.assign((size_t)ka * ka, 0.0);
    std::vector<double> unit((size_t)ka * ka, 0.0);
    for (int t = 0; t < ka; ++t)
        for (int u = t; u < ka; ++u) {
            unit[(size_t)t * ka + u] = 1.0;
            std::vector<Term> tt;
            add_one_body(tt, unit, ka, t, t + 1, u, u + 1);
            unit[(size_t)t * ka + u] = 0.0;
            const double g = expectation(c, build_mpo(tt, ka, ka), *d, *d) / nrm;
            P.gamma[(size_t)t * ka + u] = P.gamma[(size_t)u * ka + t] = g;
        }
    P.e_ref = expectation(c, build_mpo(active_hamiltonian_terms(P), ka, ka), *d, *d) / nrm;
    const double sc = 1.0 / std::sqrt(nrm);
    for (double& v : act.T[0]) v *= sc;
    finish_reference(c, act);
}

namespace {
// Shared tail of both reference forms, with gamma and E_ref set and the
// integrals in the input basis: generalised Fock matrix, semicanonical
// virtual orbitals, eps, and Psi0 on the full chain (empty virtual sites).
void finish_reference_impl(Ctx& c, MpsHost& act) {
    Problem& P = c.P;
    const int k = P.k, ka = P.ka, kv = P.kv;
    // f in the original basis (needs only (pq|tu), (pu|tq) with t,u active)
    std::vector<double> f((size_t)k * k);
    for (int p = 0; p < k; ++p)
        for (int q = 0; q < k; ++q) {
            double s = P.h[(size_t)p * k + q];
            for (int t = 0; t < ka; ++t)
                for (int u = 0; u < ka; ++u) {
                    const double g = P.gamma[(size_t)t * ka + u];
                    if (g == 0.0) continue;
                    s += g * (P.eri[(((size_t)p * k + q) * k + t) * k + u] -
                              0.5 * P.eri[(((size_t)p * k + u) * k + t) * k + q]);
                }
            f[(size_t)p * k + q] = s;
        }
    // semicanonical virtuals: rotate by the eigenvectors of f_vv (ascending)
    if (kv > 0) {
        std::vector<double> fvv((size_t)kv * kv), w, U;
        for (int a = 0; a < kv; ++a)
            for (int b = 0; b < kv; ++b) fvv[(size_t)a * kv + b] = f[(size_t)(ka + a) * k + ka + b];
        jacobi_eigh(kv, fvv, w, U);
        // sign convention: largest-magnitude coefficient of each orbital positive
        for (int j = 0; j < kv; ++j) {
            int im = 0;
            for (int i = 1; i < kv; ++i)
                if (std::fabs(U[(size_t)i * kv + j]) > std::fabs(U[(size_t)im * kv + j])) im = i;
            if (U[(size_t)im * kv + j] < 0)
                for (int i = 0; i < kv; ++i) U[(size_t)i * kv + j] = -U[(size_t)i * kv + j];
        }
        std::vector<double> C((size_t)k * k, 0.0);
        for (int t = 0; t < ka; ++t) C[(size_t)t * k + t] = 1.0;
        for (int a = 0; a < kv; ++a)
            for (int b = 0; b < kv; ++b) C[(size_t)(ka + a) * k + ka + b] = U[(size_t)a * kv + b];
        auto rotate = [&](const double* M, double* out) {
            std::vector<double> tmp((size_t)k * k, 0.0);
            for (int p = 0; p < k; ++p)
                for (int j = 0; j < k; ++j) {
                    double s = 0.0;
                    for (int q = 0; q < k; ++q) s += M[(size_t)p * k + q] * C[(size_t)q * k + j];
                    tmp[(size_t)p * k + j] = s;
                }
            for (int i = 0; i < k; ++i)
                for (int j = 0; j < k; ++j) {
                    double s = 0.0;
                    for (int p = 0; p < k; ++p) s += C[(size_t)p * k + i] * tmp[(size_t)p * k + j];
                    out[(size_t)i * k + j] = s;
                }
        };
        std::vector<double> hr((size_t)k * k), fr((size_t)k * k);
        rotate(P.h.data(), hr.data());
        rotate(f.data(), fr.data());
        P.h.swap(hr);
        f.swap(fr);
        for (int Q = 0; Q < P.nq; ++Q) rotate(&P.L_in[(size_t)Q * k * k], &P.L[(size_t)Q * k * k]);
        build_eri(P);
    }
    P.f = f;
    P.eps.resize(k);
    for (int p = 0; p < k; ++p) P.eps[p] = f[(size_t)p * k + p];
    // Psi0 on the full chain: the active MPS, then empty virtual sites
    MpsHost h0 = act;
    const QN tot(P.nel, 0);
    for (int a = 0; a < kv; ++a) {
        Bond b;
        b.sec.push_back({tot, 1, 0});
        b.finalize();
        h0.bond.push_back(b);
        std::vector<double> T(4, 0.0);
        T[0] = 1.0;
        h0.T.push_back(T);
    }
    h0.nsite = k;
    c.psi0 = std::move(*mps_upload(h0, c.st));
    P.have_ref = true;
    c.mpoA.clear(); c.mpoV.clear(); c.mpoH.reset(); c.mpoI.reset();
    c.sync();
}
}  // namespace

void finish_reference(Ctx& c, MpsHost& act) { finish_reference_impl(c, act); }

// ---------------------------------------------------------------- MPS I/O
std::unique_ptr<MpsD> mps_upload(const MpsHost& h, cudaStream_t st) {
    std::unique_ptr<MpsD> m(new MpsD);
    m->nsite = h.nsite;
    m->bond = h.bond;
    m->A.resize(h.nsite);
    for (int c = 0; c < h.nsite; ++c) {
        SiteT& A = m->A[c];
        const Bond &L = h.bond[c], &R = h.bond[c + 1];
        A.build(L, R, st);
        std::vector<double> buf(A.n);
        const int Dr = R.total;
        for (const auto& b : A.blk) {
            const int rl = L.sec[b.sl].dim, rr = R.sec[b.sr].dim;
            for (int i = 0; i < rl; ++i)
                for (int j = 0; j < rr; ++j)
                    buf[b.off + (size_t)i * rr + j] =
                        h.T[c][((size_t)(L.sec[b.sl].off + i) * 4 + b.s) * Dr + R.sec[b.sr].off + j];
        }
        if (A.n) MPSPT_CUDA(cudaMemcpyAsync(A.d.get(), buf.data(), A.n * sizeof(double),
                                            cudaMemcpyHostToDevice, st));
        MPSPT_CUDA(cudaStreamSynchronize(st));
    }
    return m;
}

MpsHost mps_download(const MpsD& m, cudaStream_t st) {
    MpsHost h;
    h.nsite = m.nsite;
    h.bond = m.bond;
    h.T.resize(m.nsite);
    for (int c = 0; c < m.nsite; ++c) {
        const SiteT& A = m.A[c];
        const Bond &L = m.bond[c], &R = m.bond[c + 1];
        std::vector<double> buf(A.n);
        if (A.n) MPSPT_CUDA(cudaMemcpyAsync(buf.data(), A.d.get(), A.n * sizeof(double),
                                            cudaMemcpyDeviceToHost, st));
        MPSPT_CUDA(cudaStreamSynchronize(st));
        h.T[c].assign((size_t)L.total * 4 * R.total, 0.0);
        for (const auto& b : A.blk) {
            const int rl = L.sec[b.sl].dim, rr = R.sec[b.sr].dim;
            for (int i = 0; i < rl; ++i)
                for (int j = 0; j < rr; ++j)
                    h.T[c][((size_t)(L.sec[b.sl].off + i) * 4 + b.s) * R.total + R.sec[b.sr].off + j] =
                        buf[b.off + (size_t)i * rr + j];
        }
    }
    return h;
}

// ----------------------------------------------------------- initial Psi1
namespace {

inline uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

inline double init_value(uint64_t seed, int c, int s, int l, int r) {
    uint64_t x = (seed << 48) + ((uint64_t)(4 * c + s) << 38) + ((uint64_t)l << 19) + (uint64_t)r;
    return (double)(splitmix64(x) >> 11) * (1.0 / 9007199254740992.0) - 0.5;
}

// Allowed-N filter per cut (empty = no filter).
std::vector<std::vector<int>> cut_filters(const Problem& P) {
    std::vector<std::vector<int>> f(P.k + 1);
    if (P.kv > 0) f[P.ka] = {P.nel - 1, P.nel - 2};
    return f;
}

// Initial bond sectors: w_q = min(nL, nR, M); proportional cap to M.
std::vector<Bond> initial_bonds(int nsite, QN target, const std::vector<std::vector<int>>& filt, int M) {
    const long long CAP = 1LL << 40;
    std::vector<std::map<QN, long long>> nL(nsite + 1), nR(nsite + 1);
    auto pass = [&](int cut, const QN& q) {
        if (filt[cut].empty()) return true;
        for (int v : filt[cut]) if (v == q.n) return true;
        return false;
    };
    nL[0][QN(0, 0)] = 1;
    for (int c = 0; c < nsite; ++c) {
        for (auto& kv : nL[c])
            for (int s = 0; s < 4; ++s) {
                QN q = kv.first + site_qn(s);
                long long& v = nL[c + 1][q];
                v = std::min(CAP, v + kv.second);
            }
        for (auto it = nL[c + 1].begin(); it != nL[c + 1].end();)
            it = pass(c + 1, it->first) ? std::next(it) : nL[c + 1].erase(it);
    }
    nR[nsite][target] = 1;
    for (int c = nsite - 1; c >= 0; --c) {
        for (auto& kv : nR[c + 1])
            for (int s = 0; s < 4; ++s) {
                QN q = kv.first - site_qn(s);
                long long& v = nR[c][q];
                v = std::min(CAP, v + kv.second);
            }
        for (auto it = nR[c].begin(); it != nR[c].end();)
            it = pass(c, it->first) ? std::next(it) : nR[c].erase(it);
    }
    std::vector<Bond> out(nsite + 1);
    for (int c = 0; c <= nsite; ++c) {
        std::vector<std::pair<QN, long long>> w;
        long long tot = 0;
        for (auto& kv : nL[c]) {
            auto it = nR[c].find(kv.first);
            if (it == nR[c].end()) continue;
            long long v = std::min(std::min(kv.second, it->second), (long long)M);
            if (v > 0) { w.push_back({kv.first, v}); tot += v; }
        }
        for (auto& e : w) {
            long long d = e.second;
            if (tot > M) d = std::min(d, std::max(1LL, ((long long)M * e.second) / tot));
            out[c].sec.push_back({e.first, (int)d, 0});
        }
        out[c].finalize();
    }
    return out;
}

}  // namespace

// ------------------------------------------------------------------ sweep
namespace {

struct Work {
    DBuf x, g, b, r, z, p, Ap, minv, x0, d, ri, zero, xw, dg;
    size_t nzero = 0;
    void ensure(size_t n, size_t n0, cudaStream_t st) {
        const size_t by = (n + 1) * sizeof(double);
        x.ensure(by, st); g.ensure(by, st); b.ensure(by, st); r.ensure(by, st); z.ensure(by, st);
        p.ensure(by, st); Ap.ensure(by, st); minv.ensure(by, st);
        d.ensure(by, st); ri.ensure(by, st); xw.ensure(by, st); dg.ensure(by, st);
        if (zero.bytes() < by || nzero < n) {
            zero.ensure(by, st);
            MPSPT_CUDA(cudaMemsetAsync(zero.get(), 0, zero.bytes(), st));
            nzero = zero.bytes() / sizeof(double);
        }
        x0.ensure((n0 + 1) * sizeof(double), st);
    }
};

struct Env {
    EnvT LA, LV, RA, RV;
};

// Composite sector of a two-site split.
struct Comp {
    QN q;
    struct Mem { int a, b; int roff; int dim; };   // (sl,s1) or (s2,sr)
    std::vector<Mem> mem;
    int dim = 0;
    size_t rho_off = 0;
};

// Truncation keeps density-matrix eigenvectors with eigenvalue above
// kKeepRel * tr(rho) (at most M of them).  At 1e-10 the smallest kept states
// are separated from the rounding level of a float64 eigensolver
// (~1e-16 |rho|) by six decades, so the kept subspace is fixed by the
// mathematics and not by how an eigensolver rounds.
constexpr double kKeepRel = 1e-10;

// Validates copy tasks (column indices are read back from the host copy).
void check_copies(const std::vector<CopyTask>& ct, const std::vector<int>& colv, const int* colp) {
    if (!checks_enabled()) return;
    for (const auto& t : ct) {
        check_range(t.dst, ((size_t)(t.rows - 1) * t.ldd + t.cols_n) * sizeof(double), "copy dst");
        int maxc = (t.trans ? t.rows : t.cols_n) - 1;
        if (t.cols) {
            const size_t base = (size_t)(t.cols - colp);
            const int nsel = t.trans ? t.rows : t.cols_n;
            require(base + nsel <= colv.size(), "copy column list out of range");
            maxc = 0;
            for (int q = 0; q < nsel; ++q) maxc = std::max(maxc, colv[base + q]);
        }
        const int nrow = t.trans ? t.cols_n : t.rows;
        check_range(t.src, ((size_t)(nrow - 1) * t.lds + maxc + 1) * sizeof(double), "copy src");
    }
}

struct Sweeper {
    Ctx& c;
    Lane& ln;
    const Chain& ch;
    int M;
    const MPO& WA;
    const MPO& WV;
    MpsD& psi;
    const MpsD& psi0;
    std::vector<std::vector<int>> filt;
    std::vector<EnvT> LA, LV, RA, RV;
    Work w;
    TwoT X, X0;
    Omega omA, omV;
    std::vector<std::unique_ptr<Omega>> omA_c, omV_c;   // per bond: the MPO is fixed during the run
    const Omega& omega(std::vector<std::unique_ptr<Omega>>& cache, const MPO& W, int i) {
        if ((int)cache.size() <= i) cache.resize(i + 1);
        if (!cache[i]) { cache[i].reset(new Omega); cache[i]->build(W, i); }
        return *cache[i];
    }
    TwoSitePlan sig, sig_lo, rhs;   // sig: float64; sig_lo: inner operator when prec != FP64
    DiagPlan dia;
    int lo_kind = GEMM_F64;
    GemmPlan prod, prod0, gr, gc;
    EnvPlan envp;
    DBuf rho, V, wv, ctasks, cols, etasks;
    EigSolver eig;
    SweepResult* res = nullptr;
    double keep_rel = kKeepRel;
    cudaEvent_t ev0, ev1;

    Sweeper(Ctx& c_, Lane& ln_, const Chain& ch_, int M_, MpsD& psi_)
        : c(c_), ln(ln_), ch(ch_), M(M_), WA(*ch_.WA), WV(*ch_.WV), psi(psi_), psi0(ch_.psi0) {
        filt = ch.filt;
        const int k = ch.nsite;
        LA.resize(k + 1); LV.resize(k + 1); RA.resize(k + 1); RV.resize(k + 1);
        if (c.opt.keep_rel > 0.0) keep_rel = c.opt.keep_rel;
        if (c.opt.prec == MPSPT_MIXED_BF16) lo_kind = GEMM_TC;
        else if (c.opt.prec == MPSPT_MIXED_FP16) lo_kind = GEMM_TC16;
        else if (c.opt.prec == MPSPT_FP32) lo_kind = GEMM_F32;
        sig_lo.set_kind(lo_kind, ln.tcerr.as<int>());
        sig.set_kind(GEMM_F64, nullptr);
        rhs.set_kind(GEMM_F64, nullptr);
        if (c.tuner) {
            Autotuner* t = c.tuner.get();
            sig.set_tuner(t); sig_lo.set_tuner(t); rhs.set_tuner(t); envp.set_tuner(t);
            prod.tuner = t; prod0.tuner = t; gr.tuner = t; gc.tuner = t; eig.ge.tuner = t;
        }
        MPSPT_CUDA(cudaEventCreate(&ev0));
        MPSPT_CUDA(cudaEventCreate(&ev1));
        for (auto& e : evs) MPSPT_CUDA(cudaEventCreate(&e));
        for (auto& e : sev) MPSPT_CUDA(cudaEventCreate(&e));
        for (auto& e : pev) MPSPT_CUDA(cudaEventCreate(&e));
        eig.stats = c.opt.verbose >= 3;
    }
    ~Sweeper() {
        if (dsc_host) { cudaStreamSynchronize(ln.st); cudaFreeHost(dsc_host); }
        if (gexec) { cudaStreamSynchronize(ln.st); cudaGraphExecDestroy(gexec); }
        cudaEventDestroy(ev0); cudaEventDestroy(ev1);
        for (auto& e : evs) cudaEventDestroy(e);
        for (auto& e : sev) cudaEventDestroy(e);
        for (auto& e : pev) cudaEventDestroy(e);
    }

    void boundary_envs() {
        const int k = ch.nsite;
        auto one = [&](EnvT& E, const std::vector<QN>& dq, const Bond& b, const Bond& k0) {
            E.build(dq, b, k0, ln.st);
            const double v = 1.0;
            MPSPT_CUDA(cudaMemcpyAsync(E.d.get(), &v, sizeof(double), cudaMemcpyHostToDevice, ln.st));
            wait();
        };
        one(LA[0], WA.dq[0], psi.bond[0], psi.bond[0]);
        one(RA[k], WA.dq[k], psi.bond[k], psi.bond[k]);
        if (ch.ground) return;
        one(LV[0], WV.dq[0], psi.bond[0], psi0.bond[0]);
        one(RV[k], WV.dq[k], psi.bond[k], psi0.bond[k]);
    }

    double env_flops = 0.0;     // flops of the last environment update
    void update_left(int i) {   // L[i+1] from L[i] and site i
        LA[i + 1].build(WA.dq[i + 1], psi.bond[i + 1], psi.bond[i + 1], ln.st);
        envp.build_left(WA, i, LA[i], psi.A[i], psi.A[i], psi.bond[i], psi.bond[i], psi.bond[i + 1],
                        psi.bond[i + 1], LA[i + 1], ln.st);
        envp.run(ln.st);
        env_flops = envp.flops();
        if (ch.ground) return;
        LV[i + 1].build(WV.dq[i + 1], psi.bond[i + 1], psi0.bond[i + 1], ln.st);
        envp.build_left(WV, i, LV[i], psi.A[i], psi0.A[i], psi.bond[i], psi0.bond[i], psi.bond[i + 1],
                        psi0.bond[i + 1], LV[i + 1], ln.st);
        envp.run(ln.st);
        env_flops += envp.flops();
    }

    void update_right(int i) {  // R[i] from R[i+1] and site i
        RA[i].build(WA.dq[i], psi.bond[i], psi.bond[i], ln.st);
        envp.build_right(WA, i, RA[i + 1], psi.A[i], psi.A[i], psi.bond[i], psi.bond[i], psi.bond[i + 1],
                         psi.bond[i + 1], RA[i], ln.st);
        envp.run(ln.st);
        env_flops = envp.flops();
        if (ch.ground) return;
        RV[i].build(WV.dq[i], psi.bond[i], psi0.bond[i], ln.st);
        envp.build_right(WV, i, RV[i + 1], psi.A[i], psi0.A[i], psi.bond[i], psi0.bond[i], psi.bond[i + 1],
                         psi0.bond[i + 1], RV[i], ln.st);
        envp.run(ln.st);
        env_flops += envp.flops();
    }

    // x (device, X layout) -> new A_i, A_{i+1}, bond i+1.  dir 0: left-to-right.
    double split(int i, int dir, int Mkeep, const TwoT& Xl, const double* xd) {
        const Bond &bL = psi.bond[i], &bR = psi.bond[i + 2];
        const std::vector<int>& fm = filt[i + 1];
        std::map<QN, Comp> comps;
        // members that appear in the layout
        for (const auto& b : Xl.blk) {
            QN q;
            int ma, mb, dim;
            if (dir == 0) { q = bL.sec[b.sl].q + site_qn(b.s1); ma = b.sl; mb = b.s1; dim = b.rows; }
            else { q = bR.sec[b.sr].q - site_qn(b.s2); ma = b.s2; mb = b.sr; dim = b.cols; }
            Comp& cp = comps[q];
            cp.q = q;
            bool have = false;
            for (auto& m : cp.mem) if (m.a == ma && m.b == mb) { have = true; break; }
            if (!have) { cp.mem.push_back({ma, mb, cp.dim, dim}); cp.dim += dim; }
        }
        std::vector<Comp> cl;
        size_t rs = 0;
        for (auto& kv : comps) {
            if (!fm.empty() && std::find(fm.begin(), fm.end(), kv.first.n) == fm.end()) continue;
            kv.second.rho_off = rs;
            rs += (size_t)kv.second.dim * kv.second.dim;
            cl.push_back(kv.second);
        }
        rho.ensure((rs + 1) * sizeof(double), ln.st);
        V.ensure((rs + 1) * sizeof(double), ln.st);
        size_t wsz = 0;
        for (auto& cp : cl) wsz += cp.dim;
        wv.ensure((wsz + 1) * sizeof(double), ln.st);
        double* rhop = rho.as<double>();
        // rho blocks
        gr.clear();
        auto member_index = [&](const Comp& cp, int a, int b) {
            for (int t = 0; t < (int)cp.mem.size(); ++t) if (cp.mem[t].a == a && cp.mem[t].b == b) return t;
            return -1;
        };
        (void)member_index;
        for (auto& cp : cl) {
            for (auto& m1 : cp.mem)
                for (auto& m2 : cp.mem) {
                    int m0 = gr.mark();
                    if (dir == 0) {
                        for (int s2 = 0; s2 < 4; ++s2) {
                            int b1 = Xl.find(m1.a, m1.b, s2), b2 = Xl.find(m2.a, m2.b, s2);
                            if (b1 < 0 || b2 < 0) continue;
                            const auto &B1 = Xl.blk[b1], &B2 = Xl.blk[b2];
                            gr.op(xd + B1.off, B1.cols, xd + B2.off, B2.cols, B1.cols, 2, 1.0);
                        }
                    } else {
                        for (int sl = 0; sl < bL.nsec(); ++sl)
                            for (int s1 = 0; s1 < 4; ++s1) {
                                int b1 = Xl.find(sl, s1, m1.a), b2 = Xl.find(sl, s1, m2.a);
                                if (b1 < 0 || b2 < 0) continue;
                                const auto &B1 = Xl.blk[b1], &B2 = Xl.blk[b2];
                                if (B1.sr != m1.b || B2.sr != m2.b) continue;
                                gr.op(xd + B1.off, B1.cols, xd + B2.off, B2.cols, B1.rows, 1, 1.0);
                            }
                    }
                    gr.block(rhop + cp.rho_off + (size_t)m1.roff * cp.dim + m2.roff, cp.dim, m1.dim, m2.dim, 0, m0);
                }
        }
        gr.upload(ln.st);
        if (c.opt.verbose >= 3) MPSPT_CUDA(cudaEventRecord(sev[0], ln.st));
        gr.run(ln.st);
        if (c.opt.verbose >= 3) MPSPT_CUDA(cudaEventRecord(sev[1], ln.st));
        // eigen-decomposition per composite sector
        std::vector<EigTask> et;
        size_t wo = 0;
        std::vector<size_t> woff;
        for (auto& cp : cl) {
            et.push_back({rhop + cp.rho_off, V.as<double>() + cp.rho_off, wv.as<double>() + wo, cp.dim, 0});
            woff.push_back(wo);
            wo += cp.dim;
        }
        eig.run(et, c.opt.eig_fp64_only != 0, ln.st);
        if (c.opt.verbose >= 3) {
            MPSPT_CUDA(cudaEventRecord(sev[2], ln.st));
            double n3 = 0; int nmax = 0;
            for (const auto& t : et) { n3 += (double)t.n * t.n * t.n; nmax = std::max(nmax, t.n); }
            eig_n3 += n3; eig_nmax = std::max(eig_nmax, nmax); eig_calls += (int)et.size();
        }
        // eigenvalues and convergence flags back through the lane's
        // page-locked buffer (one asynchronous copy each, one sync)
        const size_t wbytes = (wsz * sizeof(double) + 15) & ~(size_t)15;
        unsigned char* hb = static_cast<unsigned char*>(ln.readback(wbytes + eig.nflags * sizeof(int) + 16));
        if (wsz) MPSPT_CUDA(cudaMemcpyAsync(hb, wv.get(), wsz * sizeof(double), cudaMemcpyDeviceToHost, ln.st));
        if (eig.nflags)
            MPSPT_CUDA(cudaMemcpyAsync(hb + wbytes, eig.flags.get(), eig.nflags * sizeof(int), cudaMemcpyDeviceToHost,
                                       ln.st));
        auto ts = clk::now();
        wait();
        split_wait += since(ts);
        std::vector<double> wh(reinterpret_cast<double*>(hb), reinterpret_cast<double*>(hb) + wsz);
        std::vector<int> eflag(reinterpret_cast<int*>(hb + wbytes), reinterpret_cast<int*>(hb + wbytes) + eig.nflags);
        for (int f : eflag)
            require(f != 2, "truncation eigensolver: sweep cap reached before the convergence test",
                    MPSPT_ERR_NOT_CONVERGED);
        // selection: keep the Mkeep largest (ties at the cut dropped as a group)
        struct Cand { double lam; int ci; int rank; int col; };
        std::vector<Cand> cand;
        double tr = 0.0;
        std::vector<std::vector<int>> order(cl.size());
        for (size_t ci = 0; ci < cl.size(); ++ci) {
            const int n = cl[ci].dim;
            std::vector<int> ord(n);
            std::iota(ord.begin(), ord.end(), 0);
            const double* w_ = wh.data() + woff[ci];
            std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return w_[a] > w_[b]; });
            order[ci] = ord;
            for (int j = 0; j < n; ++j) tr += w_[j];
        }
        for (size_t ci = 0; ci < cl.size(); ++ci) {
            const double* w_ = wh.data() + woff[ci];
            for (int r = 0; r < cl[ci].dim; ++r) {
                const double lam = w_[order[ci][r]];
                if (lam > keep_rel * tr) cand.push_back({lam, (int)ci, r, order[ci][r]});
            }
        }
        std::sort(cand.begin(), cand.end(), [&](const Cand& a, const Cand& b) {
            if (a.lam != b.lam) return a.lam > b.lam;
            if (!(cl[a.ci].q == cl[b.ci].q)) return cl[a.ci].q < cl[b.ci].q;
            return a.rank < b.rank;
        });
        int m = std::min<int>(Mkeep, (int)cand.size());
        if (m < (int)cand.size()) {
            int m0 = m;
            while (m > 0 && cand[m - 1].lam <= cand[m].lam * (1.0 + 1e-8)) --m;
            if (m == 0) m = m0;
        }
        require(m > 0, "truncation kept no state (zero two-site tensor)", MPSPT_ERR_NOT_CONVERGED);
        double kept_w = 0.0;
        std::vector<std::vector<int>> kcols(cl.size());
        std::vector<std::pair<int, int>> krank;   // (ci, rank) sorted later
        for (int t = 0; t < m; ++t) { kept_w += cand[t].lam; krank.push_back({cand[t].ci, cand[t].rank}); }
        std::sort(krank.begin(), krank.end());
        for (auto& kr : krank) kcols[kr.first].push_back(order[kr.first][kr.second]);
        // new bond at cut i+1
        Bond nb;
        std::vector<int> nsec_of(cl.size(), -1);
        for (size_t ci = 0; ci < cl.size(); ++ci)
            if (!kcols[ci].empty()) { nsec_of[ci] = nb.nsec(); nb.sec.push_back({cl[ci].q, (int)kcols[ci].size(), 0}); }
        nb.finalize();
        std::vector<int> colv;
        std::vector<size_t> coff(cl.size(), 0);
        for (size_t ci = 0; ci < cl.size(); ++ci) { coff[ci] = colv.size(); colv.insert(colv.end(), kcols[ci].begin(), kcols[ci].end()); }
        upload(cols, colv, ln.st);
        const int* colp = cols.as<int>();
        psi.bond[i + 1] = nb;
        SiteT An, Bn;
        An.build(bL, nb, ln.st);
        Bn.build(nb, bR, ln.st);
        std::vector<CopyTask> ct;
        gc.clear();
        if (dir == 0) {
            if (An.n) MPSPT_CUDA(cudaMemsetAsync(An.d.get(), 0, An.n * sizeof(double), ln.st));
            for (const auto& b : An.blk) {
                const int ci = std::find_if(cl.begin(), cl.end(), [&](const Comp& cp) { return cp.q == nb.sec[b.sr].q; }) - cl.begin();
                const Comp& cp = cl[ci];
                for (const auto& mm : cp.mem)
                    if (mm.a == b.sl && mm.b == b.s)
                        ct.push_back({V.as<double>() + cp.rho_off + (size_t)mm.roff * cp.dim, An.ptr(b),
                                      colp + coff[ci], mm.dim, nb.sec[b.sr].dim, cp.dim, nb.sec[b.sr].dim, 0, 0});
            }
            check_copies(ct, colv, colp);
            upload(ctasks, ct, ln.st);
            launch_copy(ctasks.as<CopyTask>(), (int)ct.size(), ln.st);
            // carry: B(Q, s2, sr) = sum_(sl,s1) A(sl,s1,Q)^T x(sl,s1,s2)
            for (const auto& b : Bn.blk) {
                int m0 = gc.mark();
                const Comp* cp = nullptr;
                for (auto& cc : cl) if (cc.q == nb.sec[b.sl].q) cp = &cc;
                const int kq = nb.sec[b.sl].dim;
                for (const auto& mm : cp->mem) {
                    int xb = Xl.find(mm.a, mm.b, b.s);
                    int ab = An.find(mm.a, mm.b);
                    if (xb < 0 || ab < 0 || Xl.blk[xb].sr != b.sr) continue;
                    const auto& XB = Xl.blk[xb];
                    gc.op(An.ptr(An.blk[ab]), kq, xd + XB.off, XB.cols, XB.rows, 1, 1.0);
                }
                gc.block(Bn.ptr(b), bR.sec[b.sr].dim, kq, bR.sec[b.sr].dim, 0, m0);
            }
        } else {
            if (Bn.n) MPSPT_CUDA(cudaMemsetAsync(Bn.d.get(), 0, Bn.n * sizeof(double), ln.st));
            for (const auto& b : Bn.blk) {
                const int ci = std::find_if(cl.begin(), cl.end(), [&](const Comp& cp) { return cp.q == nb.sec[b.sl].q; }) - cl.begin();
                const Comp& cp = cl[ci];
                for (const auto& mm : cp.mem)
                    if (mm.a == b.s && mm.b == b.sr)
                        ct.push_back({V.as<double>() + cp.rho_off + (size_t)mm.roff * cp.dim, Bn.ptr(b),
                                      colp + coff[ci], nb.sec[b.sl].dim, mm.dim, cp.dim, mm.dim, 1, 0});
            }
            check_copies(ct, colv, colp);
            upload(ctasks, ct, ln.st);
            launch_copy(ctasks.as<CopyTask>(), (int)ct.size(), ln.st);
            // carry: A(sl, s1, Q) = sum_(s2,sr) x(sl,s1,s2,sr) B(Q,s2,sr)^T
            for (const auto& b : An.blk) {
                int m0 = gc.mark();
                const Comp* cp = nullptr;
                for (auto& cc : cl) if (cc.q == nb.sec[b.sr].q) cp = &cc;
                const int kq = nb.sec[b.sr].dim;
                for (const auto& mm : cp->mem) {
                    int xb = Xl.find(b.sl, b.s, mm.a);
                    int bb = Bn.find(b.sr, mm.a);
                    if (xb < 0 || bb < 0 || Xl.blk[xb].sr != mm.b || Bn.blk[bb].sr != mm.b) continue;
                    const auto& XB = Xl.blk[xb];
                    gc.op(xd + XB.off, XB.cols, Bn.ptr(Bn.blk[bb]), XB.cols, XB.cols, 2, 1.0);
                }
                gc.block(An.ptr(b), kq, bL.sec[b.sl].dim, kq, 0, m0);
            }
        }
        gc.upload(ln.st);
        gc.run(ln.st);
        if (c.opt.verbose >= 3) {
            MPSPT_CUDA(cudaEventRecord(sev[3], ln.st));
            MPSPT_CUDA(cudaEventSynchronize(sev[3]));
            float a = 0, b = 0, d = 0;
            cudaEventElapsedTime(&a, sev[0], sev[1]);
            cudaEventElapsedTime(&b, sev[1], sev[2]);
            cudaEventElapsedTime(&d, sev[2], sev[3]);
            t_rho += a; t_eig += b; t_post += d;
        }
        psi.A[i] = std::move(An);
        psi.A[i + 1] = std::move(Bn);
        return tr > 0 ? std::max(0.0, (tr - kept_w) / tr) : 0.0;
    }

    // x0 = A_i A_{i+1} on layout Xl into xd
    void product(GemmPlan& g, const MpsD& m, int i, const TwoT& Xl, double* xd) {
        g.clear();
        plan_product(g, Xl, xd, m.bond[i + 1], m.A[i], m.A[i + 1], m.bond[i]);
        g.upload(ln.st);
        g.run(ln.st);
    }

    void right_canonicalize() {
        for (int i = ch.nsite - 2; i >= 0; --i) {
            X.build(psi.bond[i], psi.bond[i + 2], filt[i + 1]);
            w.ensure(X.n, 1, ln.st);
            product(prod, psi, i, X, w.x.as<double>());
            split(i, 1, 1 << 30, X, w.x.as<double>());
        }
    }

    double dot(const double* a, const double* b, size_t n, int slot) {
        vec_dot(a, b, n, ln.scal.as<double>() + slot, ln.red.as<double>(), ln.cnt.as<unsigned>(), ln.st);
        return 0.0;
    }

    // every sigma launch pair is bracketed by its own events (ring of 64
    // pairs); elapsed times are collected at the next host sync
    static constexpr int NEV = 64;
    cudaEvent_t evs[2 * NEV];
    bool ev_is64[NEV];
    int nev = 0;
    void ev_begin() {
        if (nev == NEV) add_time();
        MPSPT_CUDA(cudaEventRecord(evs[2 * nev], ln.st));
    }
    void ev_end(bool is64) {
        MPSPT_CUDA(cudaEventRecord(evs[2 * nev + 1], ln.st));
        ev_is64[nev++] = is64;
    }
    void sigma64() {
        ev_begin();
        sig.run(ln.st);
        ev_end(true);
        res->sigma64_calls++;
        res->sigma64_flops += sig.flops();
    }
    void sigma_lo() {
        ev_begin();
        sig_lo.run(ln.st);
        ev_end(false);
        res->sigma_calls++;
        res->sigma_flops += sig_lo.flops();
    }
    void add_time() {
        if (nev == 0) return;
        MPSPT_CUDA(cudaEventSynchronize(evs[2 * nev - 1]));
        for (int q = 0; q < nev; ++q) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, evs[2 * q], evs[2 * q + 1]) != cudaSuccess) continue;
            if (ev_is64[q]) res->sigma64_ms += ms;
            else res->sigma_ms += ms;
        }
        nev = 0;
    }
    // ---- CUDA graphs of CG chunks (opt.cuda_graphs) ---------------------------
    // A chunk of kChunk CG iterations (sigma + the fused vector updates, no
    // host work in between) is captured once per local solve and replayed
    // until the device convergence flag is set: one graph launch instead of
    // ~7 kernel launches per iteration.  The sigma time of a graph chunk is
    // its CUDA-event time (it includes the chunk's CG vector kernels).
    static constexpr int kChunk = 8;
    cudaGraphExec_t gexec = nullptr;
    bool lo_warm = false;
    void capture(cudaGraphExec_t& ex, const std::function<void()>& body) {
        cudaGraph_t g = nullptr;
        MPSPT_CUDA(cudaStreamBeginCapture(ln.st, cudaStreamCaptureModeThreadLocal));
        const long long l0 = launch_count_thread();
        try {
            body();
        } catch (...) {
            cudaStreamEndCapture(ln.st, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        MPSPT_CUDA(cudaStreamEndCapture(ln.st, &g));
        uncount_launches(launch_count_thread() - l0);   // replays are counted, not the capture
        if (ex) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(ex, g, &info) != cudaSuccess) {
                cudaGetLastError();
                cudaGraphExecDestroy(ex);
                ex = nullptr;
            }
        }
        if (!ex) {
            const cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            MPSPT_CUDA(e);
        } else {
            cudaGraphDestroy(g);
        }
    }
    void launch_graph(cudaGraphExec_t ex, bool is64, double flops_per_iter) {
        ev_begin();
        MPSPT_CUDA(cudaGraphLaunch(ex, ln.st));
        count_launch();
        ev_end(is64);
        if (is64) { res->sigma64_calls += kChunk; res->sigma64_flops += kChunk * flops_per_iter; }
        else { res->sigma_calls += kChunk; res->sigma_flops += kChunk * flops_per_iter; }
    }

    // host time blocked on the lane's stream (the device is behind the host)
    void wait() {
        const auto t = clk::now();
        MPSPT_CUDA(cudaStreamSynchronize(ln.st));
        res->host_wait_ms += since(t);
    }

    void sync_state() {
        MPSPT_CUDA(cudaMemcpyAsync(ln.cg_host, ln.cg.as<CgState>(), sizeof(CgState), cudaMemcpyDeviceToHost, ln.st));
        wait();
        add_time();
    }
    void check_tc() {
        if (!is_tc(lo_kind)) return;
        int e = 0;
        MPSPT_CUDA(cudaMemcpyAsync(&e, ln.tcerr.get(), sizeof(int), cudaMemcpyDeviceToHost, ln.st));
        wait();
        require(e == 0, "tensor-core GEMM: bounded mbarrier wait gave up", MPSPT_ERR_TIMEOUT);
    }

    // Hylleraas value x.Ax + 2 x.g, Ax already in w.Ap (float64)
    double hylleraas(size_t n) {
        double* x = w.x.as<double>();
        dot(x, w.Ap.as<double>(), n, 0);
        dot(x, w.g.as<double>(), n, 1);
        MPSPT_CUDA(cudaMemcpyAsync(ln.scal_host, ln.scal.get(), 2 * sizeof(double), cudaMemcpyDeviceToHost, ln.st));
        wait();
        return ln.scal_host[0] + 2.0 * ln.scal_host[1];
    }

    // Plain float64 Jacobi-PCG on A x = b from the warm start x.
    double solve_plain(size_t n) {
        double* x = w.x.as<double>();
        CgState* S = ln.cg.as<CgState>();
        MPSPT_CUDA(cudaMemcpyAsync(w.p.get(), x, n * sizeof(double), cudaMemcpyDeviceToDevice, ln.st));
        sigma64();
        cg_init(w.r.as<double>(), w.z.as<double>(), w.p.as<double>(), w.b.as<double>(), w.Ap.as<double>(),
                w.minv.as<double>(), n, S, c.opt.cg_tol, ln.red.as<double>(), ln.cnt.as<unsigned>(), ln.st);
        sync_state();
        int launched = 0;
        sig.set_skip(&S->done);
        if (c.opt.cuda_graphs && ln.st != nullptr && !ln.cg_host->done) {
            capture(gexec, [&] {
                for (int q = 0; q < kChunk; ++q) {
                    sig.run(ln.st);
                    cg_step(x, w.r.as<double>(), w.z.as<double>(), w.p.as<double>(), w.Ap.as<double>(),
                            w.minv.as<double>(), n, S, ln.red.as<double>(), ln.cnt.as<unsigned>(), ln.st);
                }
            });
            while (!ln.cg_host->done && launched < c.opt.cg_max_iter) {
                launch_graph(gexec, true, sig.flops());
                launched += kChunk;
                sync_state();
            }
        }
        while (!ln.cg_host->done && launched < c.opt.cg_max_iter) {
            const int chunk = std::min(c.opt.cg_max_iter - launched, launched < 8 ? 4 : 8);
            for (int q = 0; q < chunk; ++q) {
                sigma64();
                cg_step(x, w.r.as<double>(), w.z.as<double>(), w.p.as<double>(), w.Ap.as<double>(),
                        w.minv.as<double>(), n, S, ln.red.as<double>(), ln.cnt.as<unsigned>(), ln.st);
            }
            launched += chunk;
            sync_state();
        }
        sig.set_skip(nullptr);
        require(!ln.cg_host->not_spd, "CG: p^T A p <= 0 (H0 - E0 not positive on the local space)",
                MPSPT_ERR_NOT_SPD);
        require(ln.cg_host->done != 0, "local CG reached cg_max_iter before the residual test",
                MPSPT_ERR_NOT_CONVERGED);
        res->cg_iters += ln.cg_host->iters;
        res->sigma64_calls -= launched - ln.cg_host->iters;   // skipped launches did no work
        res->sigma64_flops -= (launched - ln.cg_host->iters) * sig.flops();
        MPSPT_CUDA(cudaMemcpyAsync(w.p.get(), x, n * sizeof(double), cudaMemcpyDeviceToDevice, ln.st));
        sigma64();
        wait();
        add_time();
        return hylleraas(n);
    }

    // Iterative refinement: float64 residual r = b - A x, inner PCG on
    // A d = r with the low-precision operator, x += d, until the float64
    // residual meets cg_tol.  The last float64 A x gives the Hylleraas value.
    double solve_refined(size_t n) {
        double* x = w.x.as<double>();
        CgState* S = ln.cg.as<CgState>();
        const int max_outer = 12;
        const double tol_in = 1e-4;
        dot(w.b.as<double>(), w.b.as<double>(), n, 2);
        for (int outer = 0;; ++outer) {
            MPSPT_CUDA(cudaMemcpyAsync(w.p.get(), x, n * sizeof(double), cudaMemcpyDeviceToDevice, ln.st));
            sigma64();
            MPSPT_CUDA(cudaMemcpyAsync(w.r.get(), w.b.get(), n * sizeof(double), cudaMemcpyDeviceToDevice, ln.st));
            vec_axpy(w.r.as<double>(), w.Ap.as<double>(), -1.0, n, ln.st);
            dot(w.r.as<double>(), w.r.as<double>(), n, 3);
            MPSPT_CUDA(cudaMemcpyAsync(ln.scal_host, ln.scal.get(), 4 * sizeof(double), cudaMemcpyDeviceToHost, ln.st));
            wait();
            add_time();
            const double bb = ln.scal_host[2], rr = ln.scal_host[3];
            if (rr <= c.opt.cg_tol * c.opt.cg_tol * bb || bb == 0.0) break;
            require(outer < max_outer, "float64 refinement: 12 rounds without meeting cg_tol",
                    MPSPT_ERR_NOT_CONVERGED);
            // float16 terms have a narrow exponent range: the inner solve runs
            // on the residual scaled to unit norm (A is linear, d scales back)
            const double sc = (lo_kind == GEMM_TC16 && rr > 0.0) ? 1.0 / std::sqrt(rr) : 1.0;
            if (sc != 1.0) vec_scale_mask(w.r.as<double>(), w.r.as<double>(), sc, n, ln.st);
            // inner solve from d = 0 (the Ap buffer is reused by the inner operator)
            MPSPT_CUDA(cudaMemsetAsync(w.d.get(), 0, n * sizeof(double), ln.st));
            cg_init(w.ri.as<double>(), w.z.as<double>(), w.p.as<double>(), w.r.as<double>(),
                    w.zero.as<double>(), w.minv.as<double>(), n, S, tol_in, ln.red.as<double>(),
                    ln.cnt.as<unsigned>(), ln.st);
            MPSPT_CUDA(cudaMemcpyAsync(ln.cg_host, S, sizeof(CgState), cudaMemcpyDeviceToHost, ln.st));
            wait();
            int launched = 0;
            sig_lo.set_skip(&S->done);
            if (c.opt.cuda_graphs && ln.st != nullptr && !ln.cg_host->done) {
                // the first launch of each kernel sets its attributes and
                // occupancy cache; make it outside the capture (the product
                // lands in Ap, which the first CG iteration overwrites)
                if (!lo_warm) { sig_lo.run(ln.st); lo_warm = true; }
                capture(gexec, [&] {
                    for (int q = 0; q < kChunk; ++q) {
                        sig_lo.run(ln.st);
                        cg_step(w.d.as<double>(), w.ri.as<double>(), w.z.as<double>(), w.p.as<double>(),
                                w.Ap.as<double>(), w.minv.as<double>(), n, S, ln.red.as<double>(),
                                ln.cnt.as<unsigned>(), ln.st);
                    }
                });
                while (!ln.cg_host->done && launched < c.opt.cg_max_iter) {
                    launch_graph(gexec, false, sig_lo.flops());
                    launched += kChunk;
                    sync_state();
                }
            }
            while (!ln.cg_host->done && launched < c.opt.cg_max_iter) {
                const int chunk = std::min(c.opt.cg_max_iter - launched, launched < 8 ? 4 : 8);
                for (int q = 0; q < chunk; ++q) {
                    sigma_lo();
                    cg_step(w.d.as<double>(), w.ri.as<double>(), w.z.as<double>(), w.p.as<double>(),
                            w.Ap.as<double>(), w.minv.as<double>(), n, S, ln.red.as<double>(),
                            ln.cnt.as<unsigned>(), ln.st);
                }
                launched += chunk;
                sync_state();
            }
            sig_lo.set_skip(nullptr);
            require(!ln.cg_host->not_spd, "CG: p^T A p <= 0 (H0 - E0 not positive on the local space)",
                    MPSPT_ERR_NOT_SPD);
            res->cg_iters += ln.cg_host->iters;
            res->sigma_calls -= launched - ln.cg_host->iters;
            res->sigma_flops -= (launched - ln.cg_host->iters) * sig_lo.flops();
            vec_axpy(x, w.d.as<double>(), 1.0 / sc, n, ln.st);
        }
        return hylleraas(n);   // w.Ap holds the float64 A x of the final x
    }

    // ---- learned preconditioner -------------------------------------------
    DBuf dblocks, dmeta, dfeat, dcoef, dfit;
    std::vector<BlockRef> hblocks;
    std::vector<float> hmeta;

    // block list + QN metadata and the feature vectors of the current step
    void block_prepare(int i) {
        const Bond &bL = psi.bond[i], &bR = psi.bond[i + 2];
        hblocks.clear();
        hmeta.clear();
        const int N = ch.target.n;
        for (const auto& b : X.blk) {
            hblocks.push_back({b.off, b.rows * b.cols, 0});
            const QN ql = bL.sec[b.sl].q, qr = bR.sec[b.sr].q;
            const float m[8] = {(float)(ql.n - N) / 4.f, (float)ql.sz / 4.f, (float)(qr.n - N) / 4.f,
                                (float)qr.sz / 4.f, (float)b.s1 / 3.f, (float)b.s2 / 3.f,
                                (float)std::log2((double)b.rows) / 8.f, (float)std::log2((double)b.cols) / 8.f};
            hmeta.insert(hmeta.end(), m, m + 8);
        }
        upload(dblocks, hblocks, ln.st);
        upload(dmeta, hmeta, ln.st);
        dfeat.ensure(hblocks.size() * MLP_NF * sizeof(float) + 16, ln.st);
        block_features(dblocks.as<BlockRef>(), (int)hblocks.size(), w.dg.as<double>(), w.g.as<double>(),
                       w.x.as<double>(), dmeta.as<float>(), dfeat.as<float>(), ln.st);
    }

    // residual norm^2 of b - A v (float64 sigma)
    double resid2(const double* v, size_t n) {
        MPSPT_CUDA(cudaMemcpyAsync(w.p.get(), v, n * sizeof(double), cudaMemcpyDeviceToDevice, ln.st));
        sigma64();
        MPSPT_CUDA(cudaMemcpyAsync(w.r.get(), w.b.get(), n * sizeof(double), cudaMemcpyDeviceToDevice, ln.st));
        vec_axpy(w.r.as<double>(), w.Ap.as<double>(), -1.0, n, ln.st);
        dot(w.r.as<double>(), w.r.as<double>(), n, 4);
        MPSPT_CUDA(cudaMemcpyAsync(ln.scal_host, ln.scal.get(), 5 * sizeof(double), cudaMemcpyDeviceToHost, ln.st));
        wait();
        add_time();
        return ln.scal_host[4];
    }

    // x <- learned initial guess if its float64 residual beats the warm start
    void learned_guess(size_t n) {
        Mlp& net = *const_cast<Mlp*>(c.net);
        const int nb = (int)hblocks.size();
        dcoef.ensure((size_t)nb * 2 * sizeof(float) + 16, ln.st);
        net.forward(nb, dfeat.as<float>(), dcoef.as<float>());
        block_combine(dblocks.as<BlockRef>(), nb, dcoef.as<float>(), w.x.as<double>(), w.minv.as<double>(),
                      w.b.as<double>(), w.d.as<double>(), ln.st);
        const double r_warm = resid2(w.x.as<double>(), n);
        const double r_learn = resid2(w.d.as<double>(), n);
        if (r_learn < r_warm) {
            MPSPT_CUDA(cudaMemcpyAsync(w.x.get(), w.d.get(), n * sizeof(double), cudaMemcpyDeviceToDevice, ln.st));
            res->learned_used++;
        } else {
            res->learned_rejected++;
        }
    }

    // training pair per block: features -> least-squares (gamma, delta) of x*
    void harvest(size_t) {
        const int nb = (int)hblocks.size();
        dfit.ensure((size_t)nb * 5 * sizeof(double) + 16, ln.st);
        block_fit(dblocks.as<BlockRef>(), nb, w.xw.as<double>(), w.minv.as<double>(), w.b.as<double>(),
                  w.x.as<double>(), dfit.as<double>(), ln.st);
        std::vector<double> fit((size_t)nb * 5);
        std::vector<float> feat((size_t)nb * MLP_NF);
        MPSPT_CUDA(cudaMemcpyAsync(fit.data(), dfit.get(), fit.size() * sizeof(double), cudaMemcpyDeviceToHost, ln.st));
        MPSPT_CUDA(cudaMemcpyAsync(feat.data(), dfeat.get(), feat.size() * sizeof(float), cudaMemcpyDeviceToHost, ln.st));
        wait();
        for (int q = 0; q < nb; ++q) {
            if (c.harvest_x.size() / MLP_NF >= c.harvest_max) return;
            const double* f = &fit[(size_t)q * 5];
            const double a = f[0], b_ = f[1], cc = f[2], d = f[3], e = f[4];
            const double det = a * cc - b_ * b_;
            double ga, de;
            if (cc <= 0.0) continue;
            if (a > 0.0 && det > 1e-10 * a * cc) { ga = (d * cc - e * b_) / det; de = (a * e - b_ * d) / det; }
            else { ga = 0.0; de = e / cc; }
            if (!std::isfinite(ga) || !std::isfinite(de)) continue;
            ga = std::max(-4.0, std::min(4.0, ga));
            de = std::max(-4.0, std::min(4.0, de));
            c.harvest_x.insert(c.harvest_x.end(), &feat[(size_t)q * MLP_NF], &feat[(size_t)q * MLP_NF] + MLP_NF);
            c.harvest_t.push_back((float)ga);
            c.harvest_t.push_back((float)de);
        }
    }

    // ---- ground-state DMRG (reference Psi0) ---------------------------------
    DBuf dvec, davec, dsc;
    double* dsc_host = nullptr;

    // Lowest eigenpair of A_loc by Davidson with the Jacobi (diagonal)
    // correction, started from x (the current two-site product); restarts
    // from the Ritz vector when the basis reaches kmax.  Inner products run
    // on the device; the kmax x kmax Rayleigh quotient is diagonalised on
    // the host.  Returns the Ritz value; x holds the unit Ritz vector.
    double davidson(size_t n) {
        constexpr int kmax = 16;
        const int maxit = std::max(8, c.opt.cg_max_iter);
        dvec.ensure((size_t)kmax * n * sizeof(double) + 16, ln.st);
        davec.ensure((size_t)kmax * n * sizeof(double) + 16, ln.st);
        dsc.ensure(64 * sizeof(double), ln.st);
        if (!dsc_host) MPSPT_CUDA(cudaMallocHost(&dsc_host, 64 * sizeof(double)));
        double* Vb = dvec.as<double>();
        double* AVb = davec.as<double>();
        double* x = w.x.as<double>();
        auto V = [&](int j) { return Vb + (size_t)j * n; };
        auto AV = [&](int j) { return AVb + (size_t)j * n; };
        auto dots = [&](int cnt, const double* const* a, const double* const* b) {
            for (int q = 0; q < cnt; ++q)
                vec_dot(a[q], b[q], n, dsc.as<double>() + q, ln.red.as<double>(), ln.cnt.as<unsigned>(), ln.st);
            MPSPT_CUDA(cudaMemcpyAsync(dsc_host, dsc.get(), cnt * sizeof(double), cudaMemcpyDeviceToHost, ln.st));
            wait();
        };
        {   // v0 = x / |x|
            const double* a[1] = {x};
            dots(1, a, a);
            const double nx = std::sqrt(dsc_host[0]);
            require(nx > 0.0 && std::isfinite(nx), "Davidson: zero start vector");
            vec_scale_mask(V(0), x, 1.0 / nx, n, ln.st);
        }
        std::vector<double> H((size_t)kmax * kmax, 0.0);
        int m = 1;
        bool need_av = true;
        double theta = 0.0;
        const double tol = c.opt.cg_tol;
        for (int it = 0; it < maxit; ++it) {
            if (need_av) {   // AV[m-1] = A V[m-1] and the new column of H
                MPSPT_CUDA(cudaMemcpyAsync(w.p.get(), V(m - 1), n * sizeof(double), cudaMemcpyDeviceToDevice, ln.st));
                sigma64();
                MPSPT_CUDA(cudaMemcpyAsync(AV(m - 1), w.Ap.get(), n * sizeof(double), cudaMemcpyDeviceToDevice, ln.st));
                std::vector<const double*> a(m), b(m, AV(m - 1));
                for (int j = 0; j < m; ++j) a[j] = V(j);
                dots(m, a.data(), b.data());
                for (int j = 0; j < m; ++j) H[(size_t)j * kmax + m - 1] = H[(size_t)(m - 1) * kmax + j] = dsc_host[j];
            }
            // Rayleigh-Ritz on span V
            std::vector<double> Hm((size_t)m * m), ev, U;
            for (int i2 = 0; i2 < m; ++i2)
                for (int j = 0; j < m; ++j) Hm[(size_t)i2 * m + j] = H[(size_t)i2 * kmax + j];
            jacobi_eigh(m, Hm, ev, U);
            int lo = 0;
            for (int j = 1; j < m; ++j) if (ev[j] < ev[lo]) lo = j;
            theta = ev[lo];
            // u = V y -> x, A u = AV y -> w.r, residual r = A u - theta u -> w.z
            vec_zero(x, n, ln.st);
            vec_zero(w.r.as<double>(), n, ln.st);
            for (int j = 0; j < m; ++j) {
                const double y = U[(size_t)j * m + lo];
                vec_axpy(x, V(j), y, n, ln.st);
                vec_axpy(w.r.as<double>(), AV(j), y, n, ln.st);
            }
            MPSPT_CUDA(cudaMemcpyAsync(w.z.get(), w.r.get(), n * sizeof(double), cudaMemcpyDeviceToDevice, ln.st));
            vec_axpy(w.z.as<double>(), x, -theta, n, ln.st);
            {
                const double* a[1] = {w.z.as<double>()};
                dots(1, a, a);
            }
            const double rn = std::sqrt(dsc_host[0]);
            if (rn <= tol * std::max(1.0, std::fabs(theta))) return theta;
            if (m == kmax) {   // restart from the Ritz vector
                MPSPT_CUDA(cudaMemcpyAsync(V(0), x, n * sizeof(double), cudaMemcpyDeviceToDevice, ln.st));
                MPSPT_CUDA(cudaMemcpyAsync(AV(0), w.r.get(), n * sizeof(double), cudaMemcpyDeviceToDevice, ln.st));
                std::fill(H.begin(), H.end(), 0.0);
                H[0] = theta;
                m = 1;
            }
            // correction t = r / (theta - diag) on the masked entries, then
            // orthogonalised against V twice and normalised
            double* t = V(m);
            davidson_correction(t, w.z.as<double>(), w.dg.as<double>(), theta, n, ln.st);
            for (int pass = 0; pass < 2; ++pass) {
                std::vector<const double*> a(m), b(m, t);
                for (int j = 0; j < m; ++j) a[j] = V(j);
                dots(m, a.data(), b.data());
                for (int j = 0; j < m; ++j) vec_axpy(t, V(j), -dsc_host[j], n, ln.st);
            }
            {
                const double* a[1] = {t};
                dots(1, a, a);
            }
            const double tn = std::sqrt(dsc_host[0]);
            require(tn > 1e-300, "Davidson: correction vanished before convergence", MPSPT_ERR_NOT_CONVERGED);
            vec_scale_mask(t, t, 1.0 / tn, n, ln.st);
            ++m;
            need_av = true;
        }
        throw Error(MPSPT_ERR_NOT_CONVERGED, "Davidson reached its iteration cap (cg_max_iter)");
    }

    double step_ground(int i, int dir) {
        const Bond &bL = psi.bond[i], &bR = psi.bond[i + 2];
        X.build(bL, bR, filt[i + 1]);
        const size_t n = X.n;
        w.ensure(n, 1, ln.st);
        double* x = w.x.as<double>();
        product(prod, psi, i, X, x);
        const Omega& oA = omega(omA_c, WA, i);
        sig.build(oA, X, X, bL, bL, bR, bR, LA[i], RA[i + 2], WA.dq[i + 2], w.p.as<double>(),
                  w.Ap.as<double>(), ln.st);
        dia.build(oA, X, bL, bR, LA[i], RA[i + 2], WA.dq[i], WA.dq[i + 2], w.dg.as<double>(), ln.st);
        dia.run(ln.st);
        const double e = davidson(n);
        const double disc = split(i, dir, M, X, x);
        res->max_disc = std::max(res->max_disc, disc);
        res->max_bond = std::max(res->max_bond, psi.bond[i + 1].total);
        if (dir == 0) update_left(i);
        else update_right(i + 1);
        return e;
    }

    // one bond step; returns h_loc
    // host-side phase timers (printed with verbose >= 2)
    double t_plan = 0, t_rhs = 0, t_solve = 0, t_split = 0, t_env = 0;
    double t_rho = 0, t_eig = 0, t_post = 0, eig_n3 = 0;   // device ms (verbose >= 3)
    int eig_nmax = 0, eig_calls = 0;
    cudaEvent_t sev[4], pev[4];
    double t_rhs_dev = 0, t_env_dev = 0, rhs_gf = 0, env_gf = 0;   // verbose >= 3
    double h_prod = 0, h_rhs = 0, h_sig = 0, h_split = 0, h_env = 0;   // host-only ms
    double split_wait = 0;
    using clk = std::chrono::steady_clock;
    static double since(clk::time_point t) { return std::chrono::duration<double, std::milli>(clk::now() - t).count(); }

    double step(int i, int dir) {
        if (ch.ground) return step_ground(i, dir);
        auto t0 = clk::now();
        const Bond &bL = psi.bond[i], &bR = psi.bond[i + 2];
        auto th = clk::now();
        X.build(bL, bR, filt[i + 1]);
        X0.build(psi0.bond[i], psi0.bond[i + 2], {});
        const size_t n = X.n;
        w.ensure(n, X0.n, ln.st);
        double* x = w.x.as<double>();
        product(prod, psi, i, X, x);
        product(prod0, psi0, i, X0, w.x0.as<double>());
        h_prod += since(th); th = clk::now();
        const Omega& oA = omega(omA_c, WA, i);
        const Omega& oV = omega(omV_c, WV, i);
        rhs.build(oV, X, X0, bL, psi0.bond[i], bR, psi0.bond[i + 2], LV[i], RV[i + 2], WV.dq[i + 2],
                  w.x0.as<double>(), w.g.as<double>(), ln.st);
        h_rhs += since(th);
        if (c.opt.verbose >= 3) MPSPT_CUDA(cudaEventRecord(pev[0], ln.st));
        rhs.run(ln.st);
        if (c.opt.verbose >= 3) { MPSPT_CUDA(cudaEventRecord(pev[1], ln.st)); rhs_gf += rhs.flops() * 1e-9; }
        if (c.opt.verbose >= 2) { MPSPT_CUDA(cudaStreamSynchronize(ln.st)); t_rhs += since(t0); t0 = clk::now(); }
        if (c.opt.verbose >= 3) { float a; cudaEventElapsedTime(&a, pev[0], pev[1]); t_rhs_dev += a; }
        th = clk::now();
        sig.build(oA, X, X, bL, bL, bR, bR, LA[i], RA[i + 2], WA.dq[i + 2], w.p.as<double>(),
                  w.Ap.as<double>(), ln.st);
        dia.build(oA, X, bL, bR, LA[i], RA[i + 2], WA.dq[i], WA.dq[i + 2], w.dg.as<double>(), ln.st);
        dia.run(ln.st);
        make_minv(w.minv.as<double>(), w.dg.as<double>(), n, ln.st);
        vec_scale_mask(w.b.as<double>(), w.g.as<double>(), -1.0, n, ln.st);
        // the network and the harvest are the context's, on its own stream:
        // only a solve on the context's lane uses them (partition lanes, which
        // run concurrently on their own streams, keep the plain start)
        const bool main_lane = &ln == c.lane0.get();
        const bool use_net = main_lane && c.net != nullptr && c.opt.use_learned && !c.harvesting;
        const bool harvest_here = main_lane && c.harvesting;
        const bool learn = use_net || harvest_here;
        if (learn) block_prepare(i);
        if (harvest_here)
            MPSPT_CUDA(cudaMemcpyAsync(w.xw.get(), x, n * sizeof(double), cudaMemcpyDeviceToDevice, ln.st));
        if (lo_kind != GEMM_F64)
            sig_lo.build(oA, X, X, bL, bL, bR, bR, LA[i], RA[i + 2], WA.dq[i + 2], w.p.as<double>(),
                         w.Ap.as<double>(), ln.st);
        h_sig += since(th);
        if (c.opt.verbose >= 2) { MPSPT_CUDA(cudaStreamSynchronize(ln.st)); t_plan += since(t0); t0 = clk::now(); }
        if (use_net) learned_guess(n);
        const double h = (lo_kind == GEMM_F64) ? solve_plain(n) : solve_refined(n);
        check_tc();
        if (harvest_here) harvest(n);
        if (c.opt.verbose >= 2) { t_solve += since(t0); t0 = clk::now(); }
        th = clk::now();
        const double w0 = split_wait;
        const double disc = split(i, dir, M, X, x);
        h_split += since(th) - (split_wait - w0);
        res->max_disc = std::max(res->max_disc, disc);
        res->max_bond = std::max(res->max_bond, psi.bond[i + 1].total);
        if (c.opt.verbose >= 2) { t_split += since(t0); t0 = clk::now(); }
        if (c.opt.verbose >= 3) MPSPT_CUDA(cudaEventRecord(pev[2], ln.st));
        th = clk::now();
        if (dir == 0) update_left(i);
        else update_right(i + 1);
        h_env += since(th);
        if (c.opt.verbose >= 3) { MPSPT_CUDA(cudaEventRecord(pev[3], ln.st)); env_gf += env_flops * 1e-9; }
        if (c.opt.verbose >= 2) { MPSPT_CUDA(cudaStreamSynchronize(ln.st)); t_env += since(t0); }
        if (c.opt.verbose >= 3) { float a; cudaEventElapsedTime(&a, pev[2], pev[3]); t_env_dev += a; }
        return h;
    }
};

}  // namespace

namespace {
// Initial MPS of a sweep (reading R8): sector dimensions from the counting
// rule, entries from SplitMix64 keyed by (seed, site, state, row, column).
MpsHost initial_mps(const Ctx& c, const Chain& ch, int M) {
    const int nsite = ch.nsite;
    MpsHost ih;
    ih.nsite = nsite;
    ih.bond = initial_bonds(nsite, ch.target, ch.filt, M);
    ih.T.resize(nsite);
    for (int s = 0; s < nsite; ++s) {
        const Bond &L = ih.bond[s], &R = ih.bond[s + 1];
        ih.T[s].assign((size_t)L.total * 4 * R.total, 0.0);
        for (const auto& sl : L.sec)
            for (int t = 0; t < 4; ++t) {
                int sr = R.find(sl.q + site_qn(t));
                if (sr < 0) continue;
                const auto& rs = R.sec[sr];
                for (int a = 0; a < sl.dim; ++a)
                    for (int b = 0; b < rs.dim; ++b)
                        ih.T[s][((size_t)(sl.off + a) * 4 + t) * R.total + rs.off + b] =
                            init_value(c.opt.seed, s, t, sl.off + a, rs.off + b);
            }
    }
    return ih;
}
}  // namespace

std::unique_ptr<MpsD> minimize(Ctx& c, const Chain& ch, int M, SweepResult& res, Lane* lane) {
    Lane& ln = lane ? *lane : *c.lane0;
    RingScope rs(ln.ring.get());
    require(c.P.have_ref, "mpspt_set_reference must come first", MPSPT_ERR_STATE);
    require(M >= 1, "bond dimension M must be >= 1");
    require(c.opt.prec == MPSPT_FP64 || c.opt.prec == MPSPT_FP32 || c.opt.prec == MPSPT_MIXED_BF16 ||
                c.opt.prec == MPSPT_MIXED_FP16,
            "unknown precision mode");
    const auto t0 = std::chrono::steady_clock::now();
    const long long l0 = launch_count();
    // device timeline: an event at entry and one at the end of every sweep
    cudaEvent_t e_start;
    std::vector<cudaEvent_t> e_sweep;
    MPSPT_CUDA(cudaEventCreate(&e_start));
    MPSPT_CUDA(cudaEventRecord(e_start, ln.st));
    const int nsite = ch.nsite;
    MpsHost ih = initial_mps(c, ch, M);
    std::unique_ptr<MpsD> psi = mps_upload(ih, ln.st);
    Sweeper sw(c, ln, ch, M, *psi);
    sw.res = &res;
    sw.right_canonicalize();
    sw.boundary_envs();
    for (int i = nsite - 1; i >= 1; --i) sw.update_right(i);
    double prev = 0.0;
    const int maxs = std::min(64, std::max(1, c.opt.max_sweeps));
    for (int s = 0; s < maxs; ++s) {
        res.max_disc = 0.0;
        double e = 0.0;
        for (int i = 0; i <= nsite - 2; ++i) e = sw.step(i, 0);
        for (int i = nsite - 2; i >= 0; --i) e = sw.step(i, 1);
        res.e2_sweep.push_back(e);
        res.disc_sweep.push_back(res.max_disc);
        res.sigma_cum.push_back(res.sigma_calls + res.sigma64_calls);
        cudaEvent_t ev;
        MPSPT_CUDA(cudaEventCreate(&ev));
        MPSPT_CUDA(cudaEventRecord(ev, ln.st));
        e_sweep.push_back(ev);
        if (c.opt.verbose)
            fprintf(stderr, "[mpspt] sweep %d  E2 = %.12f  max discarded %.3e  cg %lld\n", s, e,
                    res.max_disc, res.cg_iters);
        if (c.opt.verbose >= 2)
            fprintf(stderr, "[mpspt]   host ms: rhs %.1f plan %.1f solve %.1f split %.1f env %.1f | sigma dev ms %.1f (64: %.1f)\n",
                    sw.t_rhs, sw.t_plan, sw.t_solve, sw.t_split, sw.t_env, res.sigma_ms, res.sigma64_ms);
        if (c.opt.verbose >= 3) {
            fprintf(stderr, "[mpspt]   split dev ms: rho %.1f eig %.1f post %.1f | eig tasks %d nmax %d sum n^3 %.3g\n",
                    sw.t_rho, sw.t_eig, sw.t_post, sw.eig_calls, sw.eig_nmax, sw.eig_n3);
            fprintf(stderr, "[mpspt]   rhs dev ms %.1f (%.1f GF) env dev ms %.1f (%.1f GF)\n", sw.t_rhs_dev, sw.rhs_gf,
                    sw.t_env_dev, sw.env_gf);
            const auto& E = sw.eig;
            fprintf(stderr, "[mpspt]   jacobi sweeps (mean/max): float32 %.2f/%lld polish %.2f/%lld float64 %.2f/%lld\n",
                    E.sweeps32[1] ? (double)E.sweeps32[0] / E.sweeps32[1] : 0.0, E.sweeps32[2],
                    E.sweeps_polish[1] ? (double)E.sweeps_polish[0] / E.sweeps_polish[1] : 0.0, E.sweeps_polish[2],
                    E.sweeps64[1] ? (double)E.sweeps64[0] / E.sweeps64[1] : 0.0, E.sweeps64[2]);
        }
        if (c.opt.verbose == 1)
            fprintf(stderr, "[mpspt]   host-only ms: layouts+products %.1f rhs-plan %.1f sigma-plans %.1f split-host %.1f env-plans %.1f\n",
                    sw.h_prod, sw.h_rhs, sw.h_sig, sw.h_split, sw.h_env);
        if (s > 0 && std::fabs(e - prev) < c.opt.e_tol) { res.converged = true; break; }
        prev = e;
    }
    res.e2 = res.e2_sweep.back();
    res.launches = launch_count() - l0;
    if (c.opt.prec == MPSPT_FP64) {   // all applications are float64: report them as sigma
        res.sigma_calls = res.sigma64_calls; res.sigma_flops = res.sigma64_flops; res.sigma_ms = res.sigma64_ms;
    }
    MPSPT_CUDA(cudaStreamSynchronize(ln.st));
    for (cudaEvent_t ev : e_sweep) {
        float ms = 0.f;
        MPSPT_CUDA(cudaEventElapsedTime(&ms, e_start, ev));
        res.sweep_ms.push_back(ms);
        cudaEventDestroy(ev);
    }
    cudaEventDestroy(e_start);
    res.wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return psi;
}

std::unique_ptr<MpsD> ground_state(Ctx& c, int M0, double s2_penalty, SweepResult& res) {
    Problem& P = c.P;
    require(P.have_int, "mpspt_set_integrals must come first", MPSPT_ERR_STATE);
    require(M0 >= 1, "bond dimension M0 must be >= 1");
    require(P.ka >= 2, "ground-state DMRG needs k_act >= 2");
    Lane& ln = *c.lane0;
    RingScope rs(ln.ring.get());
    const auto t0 = std::chrono::steady_clock::now();
    const long long l0 = launch_count();
    const int ka = P.ka;
    require(s2_penalty >= 0.0 && std::isfinite(s2_penalty), "spin penalty must be >= 0");
    std::vector<Term> th = active_hamiltonian_terms(P);
    // lambda S^2 = lambda S- S+ on Sz = 0 (S+ = sum_p c+_pa c_pb): lifts every
    // state with S > 0 by at least 2 lambda, so the sweep finds the lowest singlet
    if (s2_penalty > 0.0)
        for (int q = 0; q < ka; ++q)
            for (int p = 0; p < ka; ++p)
                th.push_back(Term{s2_penalty, 4, {FOp{2 * q + 1, true}, FOp{2 * q, false}, FOp{2 * p, true},
                                                  FOp{2 * p + 1, false}}});
    const MPO W = build_mpo(th, ka, ka);
    Chain ch;
    ch.nsite = ka;
    ch.ka = ka;
    ch.target = QN(P.nel, 0);
    ch.filt.assign(ka + 1, {});
    ch.WA = &W;
    ch.WV = &W;
    ch.ground = true;
    MpsHost ih = initial_mps(c, ch, M0);
    std::unique_ptr<MpsD> psi = mps_upload(ih, ln.st);
    {
        Sweeper sw(c, ln, ch, M0, *psi);
        sw.res = &res;
        sw.right_canonicalize();
        sw.boundary_envs();
        for (int i = ka - 1; i >= 1; --i) sw.update_right(i);
        double prev = 0.0;
        const int maxs = std::min(64, std::max(1, c.opt.max_sweeps));
        for (int s = 0; s < maxs; ++s) {
            res.max_disc = 0.0;
            double e = 0.0;
            for (int i = 0; i <= ka - 2; ++i) e = sw.step(i, 0);
            for (int i = ka - 2; i >= 0; --i) e = sw.step(i, 1);
            res.e2_sweep.push_back(e);
            res.disc_sweep.push_back(res.max_disc);
            if (c.opt.verbose)
                fprintf(stderr, "[mpspt] DMRG sweep %d  E = %.12f  max discarded %.3e\n", s, e, res.max_disc);
            if (s > 0 && std::fabs(e - prev) < c.opt.e_tol) { res.converged = true; break; }
            prev = e;
        }
        res.e2 = res.e2_sweep.back();
    }
    MPSPT_CUDA(cudaStreamSynchronize(ln.st));
    set_reference_mps(c, mps_download(*psi, ln.st));
    res.launches = launch_count() - l0;
    res.wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return psi;
}

std::unique_ptr<MpsD> minimize(Ctx& c, int h0, int M, SweepResult& res) {
    require(h0 == MPSPT_H0_FOCK || h0 == MPSPT_H0_DYALL, "unknown H0");
    require(c.P.have_ref, "mpspt_set_reference must come first", MPSPT_ERR_STATE);
    Chain ch = full_chain(c, h0);
    return minimize(c, ch, M, res);
}

namespace {
// Views of the context's reference MPS: site map s -> full-chain site.
void view_psi0(const Ctx& c, const std::vector<int>& sites, MpsD& out) {
    out.nsite = (int)sites.size();
    out.bond.clear();
    out.A.clear();
    out.A.resize(sites.size());
    out.bond.push_back(c.psi0.bond[sites[0]]);
    for (size_t s = 0; s < sites.size(); ++s) {
        const SiteT& src = c.psi0.A[sites[s]];
        SiteT& dst = out.A[s];
        dst.blk = src.blk;
        dst.idx = src.idx;
        dst.n = src.n;
        dst.d.make_view(src.d.get(), src.n * sizeof(double));
        out.bond.push_back(c.psi0.bond[sites[s] + 1]);
    }
}
}  // namespace

Chain full_chain(Ctx& c, int h0) {
    Chain ch;
    const Problem& P = c.P;
    ch.nsite = P.k;
    ch.ka = P.ka;
    ch.target = QN(P.nel, 0);
    ch.filt = cut_filters(P);
    ch.WA = &c.A_mpo(h0);
    ch.WV = &c.V_mpo();
    std::vector<int> sites(P.k);
    for (int s = 0; s < P.k; ++s) sites[s] = s;
    ch.orbs = sites;
    view_psi0(c, sites, ch.psi0);
    return ch;
}

Chain partition_chain(Ctx& c, int h0, int a, int b, PartOps& ops) {
    const Problem& P = c.P;
    require(a >= 0 && b >= a && b < P.kv, "partition pair out of range (need 0 <= a <= b < k_virt)");
    Chain ch;
    const int ka = P.ka, N = P.nel;
    std::vector<int> orbs;
    for (int t = 0; t < ka; ++t) orbs.push_back(t);
    orbs.push_back(ka + a);
    if (b != a) orbs.push_back(ka + b);
    const int ks = (int)orbs.size();
    ch.nsite = ks;
    ch.ka = ka;
    ch.target = QN(N, 0);
    ch.orbs = orbs;
    ch.filt.assign(ks + 1, {});
    if (a == b) ch.filt[ka] = {N - 1, N - 2};
    else { ch.filt[ka] = {N - 2}; ch.filt[ka + 1] = {N - 1}; }
    // integrals restricted to the chain's orbitals, in chain order
    const int k = P.k;
    std::vector<double> h((size_t)ks * ks), f((size_t)ks * ks), eps(ks), eri((size_t)ks * ks * ks * ks);
    for (int p = 0; p < ks; ++p) {
        eps[p] = P.eps[orbs[p]];
        for (int q = 0; q < ks; ++q) {
            h[(size_t)p * ks + q] = P.h[(size_t)orbs[p] * k + orbs[q]];
            f[(size_t)p * ks + q] = P.f[(size_t)orbs[p] * k + orbs[q]];
            for (int r = 0; r < ks; ++r)
                for (int s2 = 0; s2 < ks; ++s2)
                    eri[(((size_t)p * ks + q) * ks + r) * ks + s2] =
                        P.eri[(((size_t)orbs[p] * k + orbs[q]) * k + orbs[r]) * k + orbs[s2]];
        }
    }
    std::vector<Term> tA, tV;
    if (h0 == MPSPT_H0_DYALL) {
        add_one_body(tA, h, ks, 0, ka, 0, ka);
        add_two_body(tA, eri, ks, 0, ka, 0, ka, -1);
    } else {
        add_one_body(tA, f, ks, 0, ka, 0, ka);
    }
    add_number(tA, eps, ka, ks);
    tA.push_back(Term{-c.e0(h0), 0, {}});
    add_one_body(tV, h, ks, ka, ks, 0, ka);
    add_two_body(tV, eri, ks, 0, ks, 0, ka, ka);
    ops.A = build_mpo(tA, ks, ka);
    ops.V = build_mpo(tV, ks, ka);
    ch.WA = &ops.A;
    ch.WV = &ops.V;
    std::vector<int> sites;
    for (int t = 0; t < ka; ++t) sites.push_back(t);
    for (int s = ka; s < ks; ++s) sites.push_back(ka);   // empty virtual site of the reference
    view_psi0(c, sites, ch.psi0);
    return ch;
}

namespace {
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

void check_pairs(Ctx& c, int h0, const std::vector<std::pair<int, int>>& pairs, const std::vector<int>& Ms) {
    require(c.P.have_ref, "mpspt_set_reference must come first", MPSPT_ERR_STATE);
    require(h0 == MPSPT_H0_FOCK || h0 == MPSPT_H0_DYALL, "unknown H0");
    require(pairs.size() == Ms.size(), "one bond dimension per partition");
    for (size_t i = 0; i < pairs.size(); ++i) {
        require(pairs[i].first >= 0 && pairs[i].first <= pairs[i].second && pairs[i].second < c.P.kv,
                "partition pair out of range (need 0 <= a <= b < k_virt)");
        require(Ms[i] >= 1, "bond dimension must be >= 1");
    }
}

// Runs fn(lane, worker index) on every lane, one host thread per lane; the
// first error of any lane is rethrown after all threads have joined (a lane
// that fails sets stop so that the others leave their loops).
template <class F>
void on_lanes(Ctx& c, std::vector<std::unique_ptr<Lane>>& lanes, std::atomic<bool>& stop, F fn) {
    const int n_lanes = (int)lanes.size();
    std::vector<std::pair<mpspt_status, std::string>> errs(n_lanes, {MPSPT_OK, ""});
    auto work = [&](int l) {
        try {
            MPSPT_CUDA(cudaSetDevice(c.opt.device));
            fn(*lanes[l], l);
        } catch (const Error& e) {
            errs[l] = {e.status, e.what()};
            stop.store(true);
        } catch (const std::exception& e) {
            errs[l] = {MPSPT_ERR_INVALID, e.what()};
            stop.store(true);
        }
    };
    std::vector<std::thread> th;
    for (int l = 1; l < n_lanes; ++l) th.emplace_back(work, l);
    work(0);
    for (auto& t : th) t.join();
    for (auto& e : errs)
        if (e.first != MPSPT_OK) throw Error(e.first, e.second);
}

// The listed partitions solved concurrently on the lanes, longest first
// (cost grows like M^3); keep (if given) receives every partition's Psi1 on
// its own chain, its device memory ordered on the lane that made it.
double solve_partitions(Ctx& c, int h0, const std::vector<std::pair<int, int>>& pairs,
                        const std::vector<int>& Ms, std::vector<std::unique_ptr<Lane>>& lanes,
                        std::vector<double>& e2_part, SweepResult& res,
                        std::vector<std::unique_ptr<MpsD>>* keep) {
    const auto t0 = std::chrono::steady_clock::now();
    const long long l0 = launch_count();
    const int n = (int)pairs.size();
    e2_part.assign(n, 0.0);
    if (keep) {
        keep->clear();
        keep->resize(n);
    }
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return Ms[x] > Ms[y]; });
    std::atomic<int> next{0};
    std::atomic<bool> stop{false};
    std::vector<SweepResult> rs(n);
    on_lanes(c, lanes, stop, [&](Lane& ln, int) {
        for (int j; !stop.load() && (j = next.fetch_add(1)) < n;) {
            const int idx = order[j];
            PartOps ops;
            Chain ch = partition_chain(c, h0, pairs[idx].first, pairs[idx].second, ops);
            std::unique_ptr<MpsD> psi = minimize(c, ch, Ms[idx], rs[idx], &ln);
            e2_part[idx] = rs[idx].e2;
            if (keep) (*keep)[idx] = std::move(psi);
        }
    });
    double tot = 0.0;
    for (int i = 0; i < n; ++i) tot += e2_part[i];   // fixed (pair) order
    res = SweepResult();
    res.e2 = tot;
    res.converged = true;
    for (const auto& r : rs) {
        res.converged = res.converged && r.converged;
        res.host_wait_ms += r.host_wait_ms;
        res.cg_iters += r.cg_iters;
        res.sigma_calls += r.sigma_calls;
        res.sigma_flops += r.sigma_flops;
        res.sigma_ms += r.sigma_ms;
        res.sigma64_calls += r.sigma64_calls;
        res.sigma64_flops += r.sigma64_flops;
        res.sigma64_ms += r.sigma64_ms;
        res.max_disc = std::max(res.max_disc, r.max_disc);
        res.max_bond = std::max(res.max_bond, r.max_bond);
        if (r.e2_sweep.size() > res.e2_sweep.size()) res.e2_sweep.resize(r.e2_sweep.size(), 0.0);
    }
    res.launches = launch_count() - l0;
    res.wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    res.sweep_ms.assign(res.e2_sweep.size(), res.wall_ms);
    return tot;
}

std::vector<std::unique_ptr<Lane>> make_lanes(int n_lanes, int n) {
    n_lanes = std::max(1, std::min(n_lanes, n));
    std::vector<std::unique_ptr<Lane>> lanes;
    for (int l = 0; l < n_lanes; ++l) lanes.emplace_back(new Lane(nullptr, true));
    return lanes;
}
}  // namespace

double minimize_partitioned(Ctx& c, int h0, const std::vector<std::pair<int, int>>& pairs,
                            const std::vector<int>& Ms, int n_lanes, std::vector<double>& e2_part,
                            SweepResult& res) {
    check_pairs(c, h0, pairs, Ms);
    std::vector<std::unique_ptr<Lane>> lanes = make_lanes(n_lanes, (int)pairs.size());
    return solve_partitions(c, h0, pairs, Ms, lanes, e2_part, res, nullptr);
}

double expectation(Ctx& c, const MPO& W, const MpsD& bra, const MpsD& ket) {
    return expectation(c, W, bra, ket, c.st);
}

double expectation(Ctx& c, const MPO& W, const MpsD& bra, const MpsD& ket, cudaStream_t st) {
    (void)c;
    require(bra.nsite == ket.nsite && bra.nsite == W.nsite, "bra, ket and operator lengths differ");
    EnvT L, Ln;
    L.build(W.dq[0], bra.bond[0], ket.bond[0], st);
    const double one = 1.0;
    MPSPT_CUDA(cudaMemcpyAsync(L.d.get(), &one, sizeof(double), cudaMemcpyHostToDevice, st));
    EnvPlan ep;
    for (int i = 0; i < bra.nsite; ++i) {
        Ln.build(W.dq[i + 1], bra.bond[i + 1], ket.bond[i + 1], st);
        ep.build_left(W, i, L, bra.A[i], ket.A[i], bra.bond[i], ket.bond[i], bra.bond[i + 1],
                      ket.bond[i + 1], Ln, st);
        ep.run(st);
        MPSPT_CUDA(cudaStreamSynchronize(st));
        std::swap(L, Ln);
    }
    double v = 0.0;
    if (!L.blk.empty())
        MPSPT_CUDA(cudaMemcpyAsync(&v, L.d.get(), sizeof(double), cudaMemcpyDeviceToHost, st));
    MPSPT_CUDA(cudaStreamSynchronize(st));
    return v;
}

// <bra|W|ket> where the sites flagged in `empty` are identity sites (local
// state |0>) in both bra and ket: each maximal run of them is one sparse map
// of MPO states (one mix launch), the other sites the full transfer.  Only
// MPO states on some path from the left boundary to the right one are
// carried: a state that needs an operator on an empty site dies there, and
// a complementary operator that still needs one is never started.  On the
// medium chain that keeps about 1/6 of the states deep in the virtual region
// and 1/8 to 2/3 of them in the active region.
// Buffers of the transfers one lane runs in turn: environments, plan task
// lists and scratch keep their device memory from one transfer to the next
// (all on the lane's stream), so a transfer makes no allocation once they
// have grown.
struct XferWs {
    EnvT L, Ln;
    EnvPlan ep;
};

double expectation_runs(XferWs& ws, const MPO& W, RunMaps& rm, const MpsD& bra, const MpsD& ket,
                        const std::vector<char>& empty, cudaStream_t st, double* wait_ms, double* flops,
                        double* plan_bytes) {
    const int ns = bra.nsite;
    require(ket.nsite == ns && W.nsite == ns && (int)empty.size() == ns,
            "bra, ket, operator and site mask lengths differ");
    // segments: single sites and maximal runs of empty sites
    struct Seg { int i, j; const RunMap* T; };
    std::vector<Seg> seg;
    for (int i = 0; i < ns;) {
        int j = i + 1;
        if (empty[i]) {
            while (j < ns && empty[j]) ++j;
            seg.push_back({i, j, &rm.get(i, j)});
        } else {
            seg.push_back({i, j, nullptr});
        }
        i = j;
    }
    // states that can still reach the right boundary, at every segment's right cut
    const int ng = (int)seg.size();
    std::vector<std::vector<char>> back(ng + 1);
    back[ng].assign(W.dim[ns], 1);
    for (int g = ng - 1; g >= 0; --g) {
        const Seg& S = seg[g];
        back[g].assign(W.dim[S.i], 0);
        if (S.T) {
            for (int b = 0; b < W.dim[S.j]; ++b)
                if (back[g + 1][b])
                    for (int q = S.T->ptr[b]; q < S.T->ptr[b + 1]; ++q) back[g][S.T->col[q]] = 1;
        } else {
            const auto &ip = W.in_ptr[S.i], &ix = W.in_idx[S.i];
            for (int b = 0; b < W.dim[S.j]; ++b)
                if (back[g + 1][b])
                    for (int q = ip[b]; q < ip[b + 1]; ++q) back[g][W.W[S.i][ix[q]].a] = 1;
        }
    }
    EnvT &L = ws.L, &Ln = ws.Ln;
    EnvPlan& ep = ws.ep;
    std::vector<char> live = back[0], nlive;
    L.build(W.dq[0], bra.bond[0], ket.bond[0], st, &live, true);
    const double one = 1.0;
    if (!L.blk.empty())
        MPSPT_CUDA(cudaMemcpyAsync(L.d.get(), &one, sizeof(double), cudaMemcpyHostToDevice, st));
    for (int g = 0; g < ng; ++g) {
        const Seg& S = seg[g];
        const std::vector<char>& bk = back[g + 1];
        nlive.assign(W.dim[S.j], 0);
        if (S.T) {
            for (int b = 0; b < W.dim[S.j]; ++b)
                if (bk[b])
                    for (int q = S.T->ptr[b]; q < S.T->ptr[b + 1] && !nlive[b]; ++q) nlive[b] = live[S.T->col[q]];
            Ln.build(W.dq[S.j], bra.bond[S.j], ket.bond[S.j], st, &nlive, true);
            ep.build_left_run(*S.T, L, bra.bond[S.i], ket.bond[S.i], Ln, st);
        } else {
            const auto& op = W.out_ptr[S.i];
            for (int a = 0; a < W.dim[S.i]; ++a)
                if (live[a])
                    for (int q = op[a]; q < op[a + 1]; ++q) {
                        const int b = W.W[S.i][q].b;
                        if (bk[b]) nlive[b] = 1;
                    }
            Ln.build(W.dq[S.j], bra.bond[S.j], ket.bond[S.j], st, &nlive, true);
            ep.build_left(W, S.i, L, bra.A[S.i], ket.A[S.i], bra.bond[S.i], ket.bond[S.i], bra.bond[S.j],
                          ket.bond[S.j], Ln, st);
        }
        live.swap(nlive);
        if (flops) *flops += ep.flops();
        if (plan_bytes) *plan_bytes += (double)ep.plan_bytes();
        // no host wait between segments: every buffer the next plan replaces
        // is released stream-ordered, so the host plans the next segment
        // while the device still runs this one
        ep.run(st);
        std::swap(L, Ln);
    }
    double v = 0.0;
    if (!L.blk.empty())
        MPSPT_CUDA(cudaMemcpyAsync(&v, L.d.get(), sizeof(double), cudaMemcpyDeviceToHost, st));
    const auto tw = std::chrono::steady_clock::now();
    MPSPT_CUDA(cudaStreamSynchronize(st));
    if (wait_ms) *wait_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tw).count();
    return v;
}

double third_order(Ctx& c, int h0, const MpsD& psi1) {
    require(c.P.have_ref, "mpspt_set_reference must come first", MPSPT_ERR_STATE);
    const double n2 = expectation(c, c.I_mpo(), psi1, psi1);
    const double eh = expectation(c, c.H_mpo(), psi1, psi1);
    const double ea = expectation(c, c.A_mpo(h0), psi1, psi1);
    return eh - ea - c.P.e_ref * n2;   // <H> - <A> - (E0 + E1) <1>
}

namespace {
// A site that carries every bond state through an empty orbital: identity on
// each sector of B with local state |0> (the only non-zero blocks).
void identity_site(const Bond& B, SiteT& A, cudaStream_t st) {
    A.blk.clear();
    A.idx.assign((size_t)B.nsec() * 4, -1);
    A.n = 0;
    for (int s = 0; s < B.nsec(); ++s) {
        A.idx[(size_t)s * 4] = (int)A.blk.size();
        A.blk.push_back({s, 0, s, A.n});
        A.n += (size_t)B.sec[s].dim * B.sec[s].dim;
    }
    A.d.alloc(A.n * sizeof(double), st);
    std::vector<double> h(A.n, 0.0);
    for (const auto& b : A.blk) {
        const int d = B.sec[b.sl].dim;
        for (int i = 0; i < d; ++i) h[b.off + (size_t)i * d + i] = 1.0;
    }
    if (A.n) MPSPT_CUDA(cudaMemcpyAsync(A.d.get(), h.data(), A.n * sizeof(double), cudaMemcpyHostToDevice, st));
    MPSPT_CUDA(cudaStreamSynchronize(st));
}

void view_site(const SiteT& src, SiteT& dst) {
    dst.blk = src.blk;
    dst.idx = src.idx;
    dst.n = src.n;
    dst.d.make_view(src.d.get(), src.n * sizeof(double));
}
}  // namespace

// Psi1 of partition (a, b), given on its chain (active sites, then a, then b
// if b != a), written on the full chain.  The active sites and the
// partition's virtual sites are views of its tensors; every other virtual
// orbital is an empty site that passes the bond through.  The chain keeps the
// orbitals' relative order and an empty site has even parity, so the state is
// the same vector of the full determinant space.
void embed_partition(const Problem& P, const MpsD& part, int a, int b, MpsD& out, cudaStream_t st) {
    require(part.nsite == P.ka + (a == b ? 1 : 2), "partition MPS length differs from its chain");
    out.nsite = P.k;
    out.bond.assign(part.bond.begin(), part.bond.begin() + P.ka + 1);
    out.A.clear();
    out.A.resize(P.k);
    for (int s = 0; s < P.ka; ++s) view_site(part.A[s], out.A[s]);
    int j = P.ka;   // next site of the partition chain
    for (int v = 0; v < P.kv; ++v) {
        const int want = (j == P.ka) ? a : b;
        if (j < part.nsite && v == want) {
            view_site(part.A[j], out.A[P.ka + v]);
            out.bond.push_back(part.bond[j + 1]);
            ++j;
        } else {
            const Bond B = out.bond.back();
            identity_site(B, out.A[P.ka + v], st);
            out.bond.push_back(B);
        }
    }
    require(j == part.nsite, "partition sites not all placed");
}

double third_order_partitioned(Ctx& c, int h0, const std::vector<std::pair<int, int>>& pairs,
                               const std::vector<int>& Ms, int n_lanes, PartE3& out, SweepResult& res) {
    check_pairs(c, h0, pairs, Ms);
    const int n = (int)pairs.size();
    std::vector<std::unique_ptr<Lane>> lanes = make_lanes(n_lanes, std::max(n, n * (n - 1) / 2));
    std::vector<std::unique_ptr<MpsD>> psi;   // destroyed before the lanes it was made on
    out.e2 = solve_partitions(c, h0, pairs, Ms, lanes, out.e2_part, res, &psi);
    for (auto& l : lanes) MPSPT_CUDA(cudaStreamSynchronize(l->st));
    // operators of the E3 phase, built here before the lanes share them (the
    // full H MPO is built once per context: seconds on the medium chain)
    const auto ts = std::chrono::steady_clock::now();
    const MPO& WH = c.H_mpo();
    const MPO& WA = c.A_mpo(h0);
    const MPO& WI = c.I_mpo();
    RunMaps rmH(WH), rmA(WA), rmI(WI);
    const auto t0 = std::chrono::steady_clock::now();
    out.setup_ms = std::chrono::duration<double, std::milli>(t0 - ts).count();
    const long long l0 = launch_count();
    std::vector<MpsD> emb(n);
    for (int i = 0; i < n; ++i) embed_partition(c.P, *psi[i], pairs[i].first, pairs[i].second, emb[i], c.st);
    MPSPT_CUDA(cudaStreamSynchronize(c.st));
    // sites that are empty in both partitions of a term
    auto empty_mask = [&](int i, int j) {
        std::vector<char> m(c.P.k, 0);
        for (int v = 0; v < c.P.kv; ++v) m[c.P.ka + v] = 1;
        for (int q : {i, j}) {
            m[c.P.ka + pairs[q].first] = 0;
            m[c.P.ka + pairs[q].second] = 0;
        }
        return m;
    };
    // tasks: (i, i) = E3 of partition i (three transfers), (i, j) i < j =
    // <Psi1^i|H|Psi1^j> (one transfer); the costliest (largest M_i M_j) first
    struct Task { int i, j; long long w; };
    std::vector<Task> tasks;
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) tasks.push_back({i, j, (long long)Ms[i] * Ms[j] * (i == j ? 3 : 1)});
    std::stable_sort(tasks.begin(), tasks.end(), [](const Task& x, const Task& y) { return x.w > y.w; });
    std::vector<double> val(tasks.size(), 0.0);
    std::atomic<int> next{0};
    std::atomic<bool> stop{false};
    std::vector<double> wait(lanes.size(), 0.0), fl(lanes.size(), 0.0), pb(lanes.size(), 0.0);
    on_lanes(c, lanes, stop, [&](Lane& ln, int l) {
        RingScope rs(ln.ring.get());
        NvtxRange nr("mpspt_e3_transfers");   // lets a profiler select this phase's kernels
        XferWs ws;
        ws.ep.set_tuner(c.tuner.get());
        double* w = &wait[l];
        double* f = &fl[l];
        double* b = &pb[l];
        for (int t; !stop.load() && (t = next.fetch_add(1)) < (int)tasks.size();) {
            const Task& k = tasks[t];
            const std::vector<char> m = empty_mask(k.i, k.j);
            if (k.i == k.j) {
                const MpsD& x = emb[k.i];
                const double n2 = expectation_runs(ws, WI, rmI, x, x, m, ln.st, w, f, b);
                const double eh = expectation_runs(ws, WH, rmH, x, x, m, ln.st, w, f, b);
                const double ea = expectation_runs(ws, WA, rmA, x, x, m, ln.st, w, f, b);
                val[t] = eh - ea - c.P.e_ref * n2;   // <H> - <A> - (E0 + E1) <1>
            } else {
                val[t] = expectation_runs(ws, WH, rmH, emb[k.i], emb[k.j], m, ln.st, w, f, b);
            }
        }
        MPSPT_CUDA(cudaStreamSynchronize(ln.st));
    });
    out.wait_ms = out.flops = out.plan_bytes = 0.0;
    for (size_t l = 0; l < lanes.size(); ++l) {
        out.wait_ms += wait[l];
        out.flops += fl[l];
        out.plan_bytes += pb[l];
    }
    out.e3_part.assign(n, 0.0);
    out.h_pair.assign((size_t)n * n, 0.0);
    for (size_t t = 0; t < tasks.size(); ++t) {
        const Task& k = tasks[t];
        if (k.i == k.j) out.e3_part[k.i] = val[t];
        else out.h_pair[(size_t)k.i * n + k.j] = out.h_pair[(size_t)k.j * n + k.i] = val[t];
    }
    // sums in a fixed order: partitions, then pairs (i < j) row by row
    out.e3_cross = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) out.e3_cross += 2.0 * out.h_pair[(size_t)i * n + j];
    double diag = 0.0;
    for (int i = 0; i < n; ++i) diag += out.e3_part[i];
    out.e3 = diag + out.e3_cross;
    out.transfers = 3LL * n + (long long)n * (n - 1) / 2;
    out.e3_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    res.launches += launch_count() - l0;
    emb.clear();
    MPSPT_CUDA(cudaStreamSynchronize(c.st));
    return out.e3;
}

void local_apply(Ctx& c, int h0, const MpsD& psi1_in, int i, int op, const double* xh, double* out) {
    require(c.P.have_ref, "mpspt_set_reference must come first", MPSPT_ERR_STATE);
    require(psi1_in.nsite == c.P.k, "MPS length differs from the orbital count");
    require(i >= 0 && i + 1 < c.P.k, "bond index out of range");
    MpsD& psi1 = const_cast<MpsD&>(psi1_in);
    SweepResult res;
    require(h0 == MPSPT_H0_FOCK || h0 == MPSPT_H0_DYALL, "unknown H0");
    Chain ch = full_chain(c, h0);
    Sweeper sw(c, *c.lane0, ch, 1 << 30, psi1);
    sw.res = &res;
    sw.boundary_envs();
    for (int s = 0; s < i; ++s) sw.update_left(s);
    for (int s = c.P.k - 1; s >= i + 2; --s) sw.update_right(s);
    const Bond &bL = psi1.bond[i], &bR = psi1.bond[i + 2];
    TwoT X;
    X.build(bL, bR, sw.filt[i + 1]);
    const size_t n = X.n;
    std::vector<double> xb(n, 0.0), ob(n, 0.0);
    const int DL = bL.total, DR = bR.total;
    auto dense_index = [&](const TwoT::B& b, int r, int q) {
        return (((size_t)(bL.sec[b.sl].off + r) * 4 + b.s1) * 4 + b.s2) * DR + bR.sec[b.sr].off + q;
    };
    if (xh)
        for (const auto& b : X.blk)
            for (int r = 0; r < b.rows; ++r)
                for (int q = 0; q < b.cols; ++q) xb[b.off + (size_t)r * b.cols + q] = xh[dense_index(b, r, q)];
    sw.w.ensure(n, 1, c.st);
    MPSPT_CUDA(cudaMemcpyAsync(sw.w.p.get(), xb.data(), n * sizeof(double), cudaMemcpyHostToDevice, c.st));
    double* dout = sw.w.Ap.as<double>();
    if (op == MPSPT_LOCAL_SIGMA) {
        sw.omA.build(sw.WA, i);
        TwoSitePlan& pl = (sw.lo_kind == GEMM_F64) ? sw.sig : sw.sig_lo;
        pl.build(sw.omA, X, X, bL, bL, bR, bR, sw.LA[i], sw.RA[i + 2], sw.WA.dq[i + 2],
                 sw.w.p.as<double>(), dout, c.st);
        pl.run(c.st);
        sw.check_tc();
    } else if (op == MPSPT_LOCAL_RHS) {
        TwoT X0;
        X0.build(c.psi0.bond[i], c.psi0.bond[i + 2], {});
        sw.w.ensure(n, X0.n, c.st);
        sw.product(sw.prod0, c.psi0, i, X0, sw.w.x0.as<double>());
        sw.omV.build(sw.WV, i);
        sw.rhs.build(sw.omV, X, X0, bL, c.psi0.bond[i], bR, c.psi0.bond[i + 2], sw.LV[i], sw.RV[i + 2],
                     sw.WV.dq[i + 2], sw.w.x0.as<double>(), dout, c.st);
        sw.rhs.run(c.st);
    } else if (op == MPSPT_LOCAL_DIAG) {
        sw.omA.build(sw.WA, i);
        sw.dia.build(sw.omA, X, bL, bR, sw.LA[i], sw.RA[i + 2], sw.WA.dq[i], sw.WA.dq[i + 2], dout, c.st);
        sw.dia.run(c.st);
    } else {
        throw Error(MPSPT_ERR_INVALID, "unknown local operator");
    }
    MPSPT_CUDA(cudaMemcpyAsync(ob.data(), dout, n * sizeof(double), cudaMemcpyDeviceToHost, c.st));
    MPSPT_CUDA(cudaStreamSynchronize(c.st));
    std::fill(out, out + (size_t)DL * 16 * DR, 0.0);
    for (const auto& b : X.blk)
        for (int r = 0; r < b.rows; ++r)
            for (int q = 0; q < b.cols; ++q) out[dense_index(b, r, q)] = ob[b.off + (size_t)r * b.cols + q];
}

}  // namespace mpspt
