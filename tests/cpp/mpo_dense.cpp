// Host-only check of the library's MPO builder: reads integrals, builds the
// MPO of one operator with the library's term generators, contracts it to a
// dense 4^k x 4^k matrix and writes it out.  Used by tests/test_host_mpo.py.
// usage: mpo_dense <in.bin> <out.bin> [mask]   (in: k ka which eps[k] h[k*k] eri[k^4] e0)
// mask: one character per site, '1' = the site is held empty (local state
// |0> on both sides).  Each run of such sites is applied with the library's
// run maps (RunMaps) instead of site by site, and the output is the operator
// on the other sites' 4^(k - #empty) space.
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../paper_1408_5092_gb300/csrc/mpo.h"

using namespace mpspt;

int main(int argc, char** argv) {
    if (argc != 3 && argc != 4) return 2;
    FILE* f = std::fopen(argv[1], "rb");
    if (!f) return 3;
    int hdr[3];
    if (std::fread(hdr, sizeof(int), 3, f) != 3) return 4;
    const int k = hdr[0], ka = hdr[1], which = hdr[2];
    std::vector<double> eps(k), h((size_t)k * k), eri((size_t)k * k * k * k);
    double e0 = 0;
    if (std::fread(eps.data(), 8, eps.size(), f) != eps.size()) return 5;
    if (std::fread(h.data(), 8, h.size(), f) != h.size()) return 5;
    if (std::fread(eri.data(), 8, eri.size(), f) != eri.size()) return 5;
    if (std::fread(&e0, 8, 1, f) != 1) return 5;
    std::fclose(f);
    std::vector<Term> t;
    if (which == 0) {          // Fock-type A: f_act (passed in h) + eps n_a - e0
        add_one_body(t, h, k, 0, ka, 0, ka);
        add_number(t, eps, ka, k);
        t.push_back(Term{-e0, 0, {}});
    } else if (which == 1) {   // Dyall-type A
        add_one_body(t, h, k, 0, ka, 0, ka);
        add_two_body(t, eri, k, 0, ka, 0, ka, -1);
        add_number(t, eps, ka, k);
        t.push_back(Term{-e0, 0, {}});
    } else if (which == 2) {   // RHS operator
        add_one_body(t, h, k, ka, k, 0, ka);
        add_two_body(t, eri, k, 0, k, 0, ka, ka);
    } else {                   // full H
        add_one_body(t, h, k, 0, k, 0, k);
        add_two_body(t, eri, k, 0, k, 0, k, -1);
    }
    MPO W = build_mpo(t, k, ka);
    std::vector<char> empty(k, 0);
    if (argc == 4) {
        if ((int)std::strlen(argv[3]) != k) return 6;
        for (int p = 0; p < k; ++p) empty[p] = argv[3][p] == '1';
    }
    RunMaps rm(W);
    // dense contraction: T[a] is 4^c x 4^c (c = sites that are not held empty)
    std::vector<std::vector<double>> T(1, std::vector<double>(1, 1.0));
    int dim = 1;
    for (int p = 0; p < k;) {
        if (empty[p]) {   // a run [p, q): T_new[b] = sum_a map(a -> b) T[a]
            int q = p + 1;
            while (q < k && empty[q]) ++q;
            const RunMap& R = rm.get(p, q);
            std::vector<std::vector<double>> Tn(W.dim[q], std::vector<double>((size_t)dim * dim, 0.0));
            for (int b = 0; b < W.dim[q]; ++b)
                for (int r = R.ptr[b]; r < R.ptr[b + 1]; ++r)
                    for (size_t x = 0; x < Tn[b].size(); ++x) Tn[b][x] += R.val[r] * T[R.col[r]][x];
            T.swap(Tn);
            p = q;
            continue;
        }
        std::vector<std::vector<double>> Tn(W.dim[p + 1]);
        const int nd = dim * 4;
        for (auto& v : Tn) v.assign((size_t)nd * nd, 0.0);
        for (const auto& e : W.W[p]) {
            const Mat4& m = W.ops[e.op];
            const auto& A = T[e.a];
            auto& B = Tn[e.b];
            for (int i = 0; i < dim; ++i)
                for (int j = 0; j < dim; ++j) {
                    const double a = A[(size_t)i * dim + j];
                    if (a == 0.0) continue;
                    for (int s = 0; s < 4; ++s)
                        for (int u = 0; u < 4; ++u)
                            B[(size_t)(i * 4 + s) * nd + j * 4 + u] += a * e.coef * m[s * 4 + u];
                }
        }
        T.swap(Tn);
        dim = nd;
        ++p;
    }
    FILE* g = std::fopen(argv[2], "wb");
    int d[2] = {dim, (int)W.dim.size()};
    std::fwrite(d, sizeof(int), 2, g);
    std::fwrite(W.dim.data(), sizeof(int), W.dim.size(), g);
    std::fwrite(T[0].data(), 8, T[0].size(), g);
    std::fclose(g);
    return 0;
}
