// MPO construction (Eq. 4) as a finite-state machine over site factors.
//
// A term c * o_1 ... o_n is reordered to ascending sites (stable, sign of the
// permutation).  With the Jordan-Wigner string, an operator on site q acts as
// the parity P on every site p < q, so the term equals the product over
// sites of F_p = (its local operators on p, in order) * P^(#its operators on
// sites > p).  Bond states at a cut are: I (nothing applied), a prefix
// (factors of sites left of the cut already applied, coefficient pending),
// a suffix (coefficient applied, factors right of the cut pending; this is a
// complementary operator), or F (done).  The coefficient is applied at one
// "centre" site per term; prefixes and suffixes are shared between terms, so
// the bond dimension is O(k^2) for two-body operators and O(k_a^2 + k_v) for
// the first-order right-hand side operator.
#include "mpo.h"

#include <algorithm>
#include <cmath>

namespace mpspt {
namespace {

Mat4 m_ident() { Mat4 m{}; m[0] = m[5] = m[10] = m[15] = 1.0; return m; }
Mat4 m_parity() { Mat4 m{}; m[0] = 1; m[5] = -1; m[10] = -1; m[15] = 1; return m; }

// c+_alpha: |0>->|a>, |b>->|ab>;  c+_beta: |0>->|b>, |a>-> -|ab>.
Mat4 m_local(int spin, bool dag) {
    Mat4 c{};
    if (spin == 0) { c[1 * 4 + 0] = 1.0; c[3 * 4 + 2] = 1.0; }
    else { c[2 * 4 + 0] = 1.0; c[3 * 4 + 1] = -1.0; }
    if (dag) return c;
    Mat4 t{};
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) t[i * 4 + j] = c[j * 4 + i];
    return t;
}

Mat4 m_mul(const Mat4& a, const Mat4& b) {
    Mat4 r{};
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double s = 0;
            for (int k = 0; k < 4; ++k) s += a[i * 4 + k] * b[k * 4 + j];
            r[i * 4 + j] = s;
        }
    return r;
}

struct Table {
    std::map<std::array<long long, 16>, int> ids;
    std::vector<Mat4> mats;
    int get(const Mat4& m) {
        std::array<long long, 16> k;
        for (int i = 0; i < 16; ++i) k[i] = std::llround(m[i] * 1099511627776.0);  // 2^40
        auto it = ids.find(k);
        if (it != ids.end()) return it->second;
        int id = (int)mats.size();
        ids[k] = id;
        mats.push_back(m);
        return id;
    }
};

// kind: 0 = I, 1 = prefix, 2 = suffix, 3 = F; v = (site, factor id) pairs
struct Key {
    int kind;
    std::vector<int> v;
    bool operator<(const Key& o) const { return kind != o.kind ? kind < o.kind : v < o.v; }
    bool operator==(const Key& o) const { return kind == o.kind && v == o.v; }
};

struct StateInfo {
    QN q;
    int parity;
};

struct Trans {
    int fid = -1;       // shared transition
    bool centre = false;
    Mat4 acc{};         // centre: accumulated coefficient * factor
};

int centre_site(const std::vector<int>& s, int k_split) {
    int m = (int)s.size();
    if (m == 0) return 0;
    if (m == 1) return s[0];
    if (s.back() >= k_split) return s[m - 2];  // leave one virtual site open
    // active-only: put the coefficient at the middle op site, leaning to the
    // side that keeps the shorter half of the chain open
    bool left_half = s[0] + s[m - 1] < k_split;
    if (m == 3) return s[1];
    return left_half ? s[m / 2] : s[m / 2 - 1];
}

}  // namespace

MPO build_mpo(const std::vector<Term>& terms, int nsite, int k_split) {
    Table tab;
    const int fI = tab.get(m_ident());
    const int fP = tab.get(m_parity());
    std::vector<std::map<Key, int>> sid(nsite + 1);
    std::vector<std::vector<Key>> skey(nsite + 1);
    std::map<Key, StateInfo> info;
    std::map<Key, std::pair<int, int>> pass;       // site range of pass-throughs
    std::vector<std::map<std::pair<int, int>, Trans>> tr(nsite);
    const Key KI{0, {}}, KF{3, {}};
    info[KI] = {QN(0, 0), 0};
    info[KF] = {QN(0, 0), 0};

    auto id_at = [&](int cut, const Key& k) {
        auto& m = sid[cut];
        auto it = m.find(k);
        if (it != m.end()) return it->second;
        int id = (int)skey[cut].size();
        m[k] = id;
        skey[cut].push_back(k);
        return id;
    };
    auto set_shared = [&](int p, int a, int b, int fid) {
        auto it = tr[p].find({a, b});
        if (it == tr[p].end()) { Trans t; t.fid = fid; tr[p][{a, b}] = t; return; }
        if (it->second.centre || it->second.fid != fid)
            throw Error(MPSPT_ERR_INVALID, "MPO builder: inconsistent shared transition");
    };
    auto add_centre = [&](int p, int a, int b, const Mat4& m, double c) {
        auto it = tr[p].find({a, b});
        if (it == tr[p].end()) {
            Trans t; t.centre = true;
            for (int i = 0; i < 16; ++i) t.acc[i] = c * m[i];
            tr[p][{a, b}] = t;
            return;
        }
        if (!it->second.centre) throw Error(MPSPT_ERR_INVALID, "MPO builder: centre collision");
        for (int i = 0; i < 16; ++i) it->second.acc[i] += c * m[i];
    };

    for (const Term& t : terms) {
        if (t.c == 0.0) continue;
        require(t.n % 2 == 0, "MPO builder: odd fermion terms unsupported");
        FOp ops[4];
        for (int i = 0; i < t.n; ++i) ops[i] = t.op[i];
        // stable insertion sort by site, sign from transpositions of distinct sites
        double sign = 1.0;
        for (int i = 1; i < t.n; ++i)
            for (int j = i; j > 0 && ops[j - 1].j / 2 > ops[j].j / 2; --j) {
                std::swap(ops[j - 1], ops[j]);
                sign = -sign;
            }
        const double c = t.c * sign;
        if (t.n == 0) {
            int a = id_at(0, KI), b = id_at(1, KF);
            add_centre(0, a, b, tab.mats[fI], c);
            continue;
        }
        std::vector<int> sites;
        for (int i = 0; i < t.n; ++i)
            if (sites.empty() || sites.back() != ops[i].j / 2) sites.push_back(ops[i].j / 2);
        const int m = (int)sites.size();
        std::vector<int> fac(m);
        std::vector<QN> fq(m);
        std::vector<int> fpar(m);
        for (int k = 0; k < m; ++k) {
            Mat4 f = m_ident();
            int nright = 0, nhere = 0;
            QN q;
            for (int i = 0; i < t.n; ++i) {
                int p = ops[i].j / 2;
                if (p == sites[k]) {
                    f = m_mul(f, m_local(ops[i].j % 2, ops[i].dag));
                    int d = ops[i].dag ? 1 : -1;
                    q = q + QN(d, d * (ops[i].j % 2 == 0 ? 1 : -1));
                    ++nhere;
                } else if (p > sites[k]) {
                    ++nright;
                }
            }
            if (nright % 2) f = m_mul(f, m_parity());
            fac[k] = tab.get(f);
            fq[k] = q;
            fpar[k] = nhere % 2;
        }
        QN tot;
        for (auto& q : fq) tot = tot + q;
        require(tot == QN(0, 0), "MPO builder: term does not conserve N and Sz");
        const int cs = centre_site(sites, k_split);
        // key of the state at a cut
        auto key_at = [&](int cut) -> Key {
            if (cut <= sites[0]) return KI;
            if (cut > sites[m - 1]) return KF;
            Key k;
            if (cut <= cs) {
                k.kind = 1;
                for (int i = 0; i < m && sites[i] < cut; ++i) { k.v.push_back(sites[i]); k.v.push_back(fac[i]); }
            } else {
                k.kind = 2;
                for (int i = 0; i < m; ++i)
                    if (sites[i] >= cut) { k.v.push_back(sites[i]); k.v.push_back(fac[i]); }
            }
            return k;
        };
        for (int k = 0; k < m; ++k) {
            const int p = sites[k];
            Key ka = key_at(p), kb = key_at(p + 1);
            int a = id_at(p, ka), b = id_at(p + 1, kb);
            if (p == cs) add_centre(p, a, b, tab.mats[fac[k]], c);
            else set_shared(p, a, b, fac[k]);
            if (kb.kind == 1 || kb.kind == 2) {
                QN q;
                int par = 0;
                if (kb.kind == 1) {
                    for (int i = 0; i <= k; ++i) { q = q + fq[i]; par ^= fpar[i]; }
                } else {
                    for (int i = k + 1; i < m; ++i) { q = q - fq[i]; par ^= fpar[i]; }
                }
                info[kb] = {q, par};
                int lo = p + 1, hi = sites[k + 1] - 1;
                if (lo <= hi) {
                    auto it = pass.find(kb);
                    if (it == pass.end()) pass[kb] = {lo, hi};
                    else { it->second.first = std::min(it->second.first, lo);
                           it->second.second = std::max(it->second.second, hi); }
                }
            }
        }
    }
    for (auto& kv : pass) {
        const Key& k = kv.first;
        int fid = info[k].parity ? fP : fI;
        for (int p = kv.second.first; p <= kv.second.second; ++p)
            set_shared(p, id_at(p, k), id_at(p + 1, k), fid);
    }
    for (int p = 0; p < nsite; ++p) {
        set_shared(p, id_at(p, KI), id_at(p + 1, KI), fI);
        set_shared(p, id_at(p, KF), id_at(p + 1, KF), fI);
    }
    // prune states not on a path from I (cut 0) to F (cut nsite)
    std::vector<std::vector<char>> fw(nsite + 1), bw(nsite + 1);
    for (int c = 0; c <= nsite; ++c) { fw[c].assign(skey[c].size(), 0); bw[c].assign(skey[c].size(), 0); }
    fw[0][sid[0][KI]] = 1;
    for (int p = 0; p < nsite; ++p)
        for (auto& kv : tr[p]) if (fw[p][kv.first.first]) fw[p + 1][kv.first.second] = 1;
    bw[nsite][sid[nsite][KF]] = 1;
    for (int p = nsite - 1; p >= 0; --p)
        for (auto& kv : tr[p]) if (bw[p + 1][kv.first.second]) bw[p][kv.first.first] = 1;
    MPO out;
    out.nsite = nsite;
    out.dim.resize(nsite + 1);
    out.dq.resize(nsite + 1);
    out.W.resize(nsite);
    std::vector<std::vector<int>> renum(nsite + 1);
    for (int c = 0; c <= nsite; ++c) {
        std::vector<int> alive;
        for (int i = 0; i < (int)skey[c].size(); ++i) if (fw[c][i] && bw[c][i]) alive.push_back(i);
        std::sort(alive.begin(), alive.end(), [&](int x, int y) { return skey[c][x] < skey[c][y]; });
        renum[c].assign(skey[c].size(), -1);
        for (int i = 0; i < (int)alive.size(); ++i) {
            renum[c][alive[i]] = i;
            out.dq[c].push_back(info[skey[c][alive[i]]].q);
        }
        out.dim[c] = (int)alive.size();
    }
    for (int p = 0; p < nsite; ++p) {
        for (auto& kv : tr[p]) {
            int a = renum[p][kv.first.first], b = renum[p + 1][kv.first.second];
            if (a < 0 || b < 0) continue;
            const Trans& t = kv.second;
            if (t.centre) {
                bool zero = true;
                for (double v : t.acc) if (v != 0.0) zero = false;
                if (zero) continue;
                out.W[p].push_back({a, b, tab.get(t.acc), 1.0});
            } else {
                out.W[p].push_back({a, b, t.fid, 1.0});
            }
        }
        std::sort(out.W[p].begin(), out.W[p].end(), [](const MpoEntry& x, const MpoEntry& y) {
            return x.a != y.a ? x.a < y.a : x.b < y.b;
        });
    }
    out.ops = tab.mats;
    out.index();
    return out;
}

void MPO::index() {
    out_ptr.assign(nsite, {});
    in_ptr.assign(nsite, {});
    in_idx.assign(nsite, {});
    for (int p = 0; p < nsite; ++p) {
        const auto& E = W[p];
        out_ptr[p].assign(dim[p] + 1, 0);
        in_ptr[p].assign(dim[p + 1] + 1, 0);
        for (const auto& e : E) {
            ++out_ptr[p][e.a + 1];
            ++in_ptr[p][e.b + 1];
        }
        for (int a = 0; a < dim[p]; ++a) out_ptr[p][a + 1] += out_ptr[p][a];
        for (int b = 0; b < dim[p + 1]; ++b) in_ptr[p][b + 1] += in_ptr[p][b];
        in_idx[p].resize(E.size());
        std::vector<int> fill(in_ptr[p].begin(), in_ptr[p].end() - 1);
        for (int q = 0; q < (int)E.size(); ++q) in_idx[p][fill[E[q].b]++] = q;
    }
}

RunMaps::RunMaps(const MPO& W_) : W(W_) {
    out.resize(W.nsite);
    for (int s = 0; s < W.nsite; ++s) {
        out[s].resize(W.dim[s]);
        for (const auto& e : W.W[s]) {
            const double v = W.ops[e.op][0];   // <0|o|0>
            if (v != 0.0) out[s][e.a].push_back({e.b, e.coef * v});
        }
    }
}

const RunMap& RunMaps::get(int s0, int s1) {
    require(s0 >= 0 && s0 < s1 && s1 <= W.nsite, "run of empty sites out of range");
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = maps.find({s0, s1});
        if (it != maps.end()) return *it->second;
    }
    // propagate every source state through the run (frontiers are short:
    // an operator string either passes an empty site unchanged or dies)
    std::vector<std::vector<std::pair<int, double>>> to(W.dim[s1]);
    std::vector<std::pair<int, double>> cur, nxt;
    for (int a = 0; a < W.dim[s0]; ++a) {
        cur.assign(1, {a, 1.0});
        for (int s = s0; s < s1 && !cur.empty(); ++s) {
            nxt.clear();
            for (const auto& xw : cur)
                for (const auto& bc : out[s][xw.first]) nxt.push_back({bc.first, xw.second * bc.second});
            if (nxt.size() > 1) {   // merge paths that meet (sum in path order)
                std::stable_sort(nxt.begin(), nxt.end(),
                                 [](const std::pair<int, double>& x, const std::pair<int, double>& y) {
                                     return x.first < y.first;
                                 });
                size_t w = 0;
                for (size_t r = 0; r < nxt.size(); ++r) {
                    if (w > 0 && nxt[w - 1].first == nxt[r].first) nxt[w - 1].second += nxt[r].second;
                    else nxt[w++] = nxt[r];
                }
                nxt.resize(w);
            }
            cur.swap(nxt);
        }
        for (const auto& bw : cur)
            if (bw.second != 0.0) to[bw.first].push_back({a, bw.second});
    }
    std::unique_ptr<RunMap> m(new RunMap);
    m->ptr.assign(W.dim[s1] + 1, 0);
    for (int b = 0; b < W.dim[s1]; ++b) {
        m->ptr[b + 1] = m->ptr[b] + (int)to[b].size();
        for (const auto& aw : to[b]) {
            m->col.push_back(aw.first);
            m->val.push_back(aw.second);
        }
    }
    std::lock_guard<std::mutex> g(mu);
    auto& slot = maps[{s0, s1}];
    if (!slot) slot = std::move(m);
    return *slot;
}

void add_one_body(std::vector<Term>& out, const std::vector<double>& t, int k,
                  int p0, int p1, int q0, int q1) {
    for (int p = p0; p < p1; ++p)
        for (int q = q0; q < q1; ++q) {
            double v = t[(size_t)p * k + q];
            if (v == 0.0) continue;
            for (int s = 0; s < 2; ++s) {
                Term tm{v, 2, {}};
                tm.op[0] = {2 * p + s, true};
                tm.op[1] = {2 * q + s, false};
                out.push_back(tm);
            }
        }
}

void add_two_body(std::vector<Term>& out, const std::vector<double>& eri, int k,
                  int p0, int p1, int q0, int q1, int vmin) {
    // c+_ps c+_rt c_st c_qs == c+_rt c+_ps c_qs c_st: merge (p,q,s) <-> (r,s,t)
    auto E = [&](int p, int q, int r, int s) {
        return eri[(((size_t)p * k + q) * k + r) * k + s];
    };
    for (int p = p0; p < p1; ++p)
        for (int q = q0; q < q1; ++q)
            for (int r = p0; r < p1; ++r)
                for (int s = q0; s < q1; ++s) {
                    if (vmin >= 0 && p < vmin && r < vmin) continue;
                    double v = E(p, q, r, s);
                    if (v == 0.0) continue;
                    for (int a = 0; a < 2; ++a)
                        for (int b = 0; b < 2; ++b) {
                            if (a == b && (p == r || q == s)) continue;
                            long k1 = ((long)p * k + q) * 2 + a, k2 = ((long)r * k + s) * 2 + b;
                            if (k1 > k2) continue;
                            double c = (k1 < k2) ? v : 0.5 * v;
                            Term tm{c, 4, {}};
                            tm.op[0] = {2 * p + a, true};
                            tm.op[1] = {2 * r + b, true};
                            tm.op[2] = {2 * s + b, false};
                            tm.op[3] = {2 * q + a, false};
                            out.push_back(tm);
                        }
                }
}

void add_number(std::vector<Term>& out, const std::vector<double>& eps, int a0, int a1) {
    for (int a = a0; a < a1; ++a) {
        if (eps[a] == 0.0) continue;
        for (int s = 0; s < 2; ++s) {
            Term tm{eps[a], 2, {}};
            tm.op[0] = {2 * a + s, true};
            tm.op[1] = {2 * a + s, false};
            out.push_back(tm);
        }
    }
}

}  // namespace mpspt
