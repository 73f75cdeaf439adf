#include "eig.h"

#include <algorithm>

namespace mpspt {

namespace {
constexpr int kMaxSweepsF64 = 60;      // float64 Jacobi from the identity
constexpr int kMaxSweepsF32 = 12;      // float32 start (a cap is not an error: the polish follows)
constexpr int kMaxSweepsPolish = 30;   // float64 polish of V^T A V
constexpr int kPolishBatch = 6;        // sweeps launched before the host looks at the stop flags
constexpr int kClusterMinN = 48;       // float64 sweeps on CTA clusters from this size
size_t a16(size_t b) { return (b + 15) & ~(size_t)15; }
}  // namespace

void EigSolver::jacobi(const std::vector<EigTask>& et, const std::vector<const double*>& in, int vinit, bool f32,
                       int maxs, bool want_w, cudaStream_t st, int batch) {
    const int nt = (int)et.size();
    std::vector<size_t> off(nt);
    size_t tot = 0;
    for (int i = 0; i < nt; ++i) {
        off[i] = tot;
        tot += a16(jac_p_bytes(et[i].n)) + a16(jac_rot_bytes(et[i].n)) + 16;
    }
    scratch.ensure(tot + 16, st);
    flags.ensure((size_t)nt * sizeof(int) + 16, st);
    nflags = nt;
    unsigned char* base = static_cast<unsigned char*>(scratch.get());
    std::vector<JacTask> jt(nt);
    std::vector<JacRows> rows;
    int smem = 0;
    for (int i = 0; i < nt; ++i) {
        const int n = et[i].n;
        unsigned char* P = base + off[i];
        unsigned char* R = P + a16(jac_p_bytes(n));
        unsigned char* S = R + a16(jac_rot_bytes(n));
        check_range(in[i], (size_t)n * n * sizeof(double), "jacobi A");
        check_range(P, jac_p_bytes(n), "jacobi P");
        check_range(R, jac_rot_bytes(n), "jacobi rot");
        check_range(S, 16, "jacobi state");
        jt[i] = {in[i], P, R, et[i].V, want_w ? et[i].w : nullptr, reinterpret_cast<double*>(S),
                 flags.as<int>() + i, reinterpret_cast<int*>(S + 12), n, vinit, 0, 0};
        const int rpb = jac_rows_per_block(n, f32);
        for (int r0 = 0; r0 < n; r0 += rpb) {
            const int nr = std::min(rpb, n - r0);
            rows.push_back({i, r0, nr, 0});
            smem = std::max(smem, nr * (n | 1) * (f32 ? 4 : 8));
        }
    }
    // float64 sweeps of larger matrices run on clusters of 8 CTAs (one SM's
    // float64 pipe is the limit); the rest on one CTA each.  Both kernels do
    // the same arithmetic per entry.
    std::vector<JacTask> one, clu;
    int csm = 0;
    for (int i = 0; i < nt; ++i) {
        const int cs = f32 ? 0 : jac_cluster_smem(et[i].n);
        if (et[i].n >= kClusterMinN && cs > 0) {
            clu.push_back(jt[i]);
            csm = std::max(csm, cs);
        } else {
            one.push_back(jt[i]);
        }
    }
    // the apply blocks index the full task list
    upload(djt, jt, st);
    upload(drows, rows, st);
    if (!one.empty()) upload(djt1, one, st);
    if (!clu.empty()) upload(djtc, clu, st);
    // Sweeps are launched in batches; a matrix that has stopped turns its
    // later launches into no-ops, and between batches the host reads the
    // stop flags (one small copy and a sync) so that the tail of a long cap
    // is only launched when some matrix still needs it.
    if (batch <= 0) batch = maxs + 1;
    for (int s0 = 0; s0 <= maxs; s0 += batch) {
        if (s0 > 0) {
            if (!flag_host) MPSPT_CUDA(cudaMallocHost(&flag_host, 4096 * sizeof(int)));
            bool all = true;
            for (int c0 = 0; c0 < nt && all; c0 += 4096) {
                const int nc = std::min(4096, nt - c0);
                MPSPT_CUDA(cudaMemcpyAsync(flag_host, flags.as<int>() + c0, nc * sizeof(int), cudaMemcpyDeviceToHost, st));
                MPSPT_CUDA(cudaStreamSynchronize(st));
                for (int i = 0; i < nc; ++i) all = all && flag_host[i] != 0;
            }
            if (all) break;
        }
        for (int s = s0; s <= maxs && s < s0 + batch; ++s) {
            if (!one.empty()) launch_jac_sweep(djt1.as<JacTask>(), (int)one.size(), s, maxs, f32, st);
            if (!clu.empty()) launch_jac_sweep_cluster(djtc.as<JacTask>(), (int)clu.size(), s, maxs, csm, st);
            if (s < maxs) launch_jac_apply(djt.as<JacTask>(), drows.as<JacRows>(), (int)rows.size(), smem, s, f32, st);
        }
    }
    if (stats) {   // sweeps per matrix (diagnostics; synchronises)
        for (int i = 0; i < nt; ++i) {
            int k = 0;
            MPSPT_CUDA(cudaMemcpyAsync(&k, jt[i].nsw, sizeof(int), cudaMemcpyDeviceToHost, st));
            MPSPT_CUDA(cudaStreamSynchronize(st));
            long long* acc = f32 ? sweeps32 : (vinit ? sweeps_polish : sweeps64);
            acc[0] += k;
            acc[1] += 1;
            acc[2] = std::max<long long>(acc[2], k);
        }
    }
}

void EigSolver::run(const std::vector<EigTask>& et, bool fp64_only, cudaStream_t st) {
    if (et.empty()) return;
    std::vector<const double*> in;
    for (const auto& t : et) {
        require(t.n >= 1 && t.n <= 2048, "eigenproblem size must be in [1, 2048]");
        check_range(t.V, (size_t)t.n * t.n * sizeof(double), "eig V");
        check_range(t.w, (size_t)t.n * sizeof(double), "eig w");
        in.push_back(t.A);
    }
    if (fp64_only) {
        jacobi(et, in, 0, false, kMaxSweepsF64, true, st);
        return;
    }
    jacobi(et, in, 0, true, kMaxSweepsF32, false, st, kPolishBatch);
    size_t tot = 0;
    std::vector<size_t> off;
    for (const auto& t : et) { off.push_back(tot); tot += (size_t)t.n * t.n; }
    vt.ensure((tot + 1) * sizeof(double), st);
    g.ensure((tot + 1) * sizeof(double), st);
    std::vector<EigTask> ns;
    for (size_t i = 0; i < et.size(); ++i) ns.push_back({g.as<double>() + off[i], nullptr, nullptr, et[i].n, 0});
    upload(dtns, ns, st);
    // C_i = op(A_i) B_i for every task (n x n, leading dimension n)
    enum Src { TA, TV, TVT, TG };
    auto ptr = [&](Src s, size_t i) -> double* {
        switch (s) {
            case TA: return const_cast<double*>(et[i].A);
            case TV: return et[i].V;
            case TVT: return vt.as<double>() + off[i];
            default: return g.as<double>() + off[i];
        }
    };
    auto batched = [&](Src a, int trans, Src b, Src c) {
        ge.clear();
        for (size_t i = 0; i < et.size(); ++i) {
            const int n = et[i].n;
            const int m0 = ge.mark();
            ge.op(ptr(a, i), n, ptr(b, i), n, n, trans, 1.0);
            ge.block(ptr(c, i), n, n, n, 0, m0);
        }
        ge.upload(st);
        ge.run(st);
    };
    batched(TV, 1, TV, TG);        // G = V^T V
    launch_ns_prep(dtns.as<EigTask>(), (int)ns.size(), st);
    batched(TV, 0, TG, TVT);       // Vt = V (3/2 I - 1/2 G)
    batched(TVT, 1, TVT, TG);
    launch_ns_prep(dtns.as<EigTask>(), (int)ns.size(), st);
    batched(TVT, 0, TG, TV);       // V = Vt (3/2 I - 1/2 Vt^T Vt)
    batched(TA, 0, TV, TVT);       // Vt = A V
    batched(TV, 1, TVT, TG);       // G = B = V^T A V
    std::vector<const double*> bin;
    for (size_t i = 0; i < et.size(); ++i) bin.push_back(g.as<double>() + off[i]);
    jacobi(et, bin, 1, false, kMaxSweepsPolish, true, st, kPolishBatch);
}

}  // namespace mpspt
