// Host-only check of the library's MPO builder: reads integrals, builds the
// MPO of one operator with the library's term generators, contracts it to a
// dense 4^k x 4^k matrix and writes it out.  Used by tests/test_host_mpo.py.
// usage: mpo_dense <in.bin> <out.bin>   (in: k ka which eps[k] h[k*k] eri[k^4] e0)
#include <cstdio>
#include <vector>

#include "../../paper_1408_5092_gb300/csrc/mpo.h"

using namespace mpspt;

int main(int argc, char** argv) {
    if (argc != 3) return 2;
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
    // dense contraction: T[a] is 4^c x 4^c
    std::vector<std::vector<double>> T(1, std::vector<double>(1, 1.0));
    int dim = 1;
    for (int p = 0; p < k; ++p) {
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
    }
    FILE* g = std::fopen(argv[2], "wb");
    int d[2] = {dim, (int)W.dim.size()};
    std::fwrite(d, sizeof(int), 2, g);
    std::fwrite(W.dim.data(), sizeof(int), W.dim.size(), g);
    std::fwrite(T[0].data(), 8, T[0].size(), g);
    std::fclose(g);
    return 0;
}
