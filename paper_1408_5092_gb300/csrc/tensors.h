// Block-sparse tensors of the sweep.  Every block is a dense row-major
// matrix stored contiguously in one device buffer; block tables live on the
// host and are turned into task lists by the planner.
#pragma once
#include <vector>

#include "core.h"
#include "mpo.h"

namespace mpspt {

// MPS site tensor A[l, s, r]: blocks (sl, s) -> sr = sector of q(sl) + q(s).
struct SiteT {
    struct B { int sl, s, sr; size_t off; };
    std::vector<B> blk;
    std::vector<int> idx;   // sl*4 + s -> block or -1
    size_t n = 0;
    DBuf d;
    void build(const Bond& L, const Bond& R, cudaStream_t st) {
        blk.clear();
        idx.assign((size_t)L.nsec() * 4, -1);
        n = 0;
        for (int sl = 0; sl < L.nsec(); ++sl)
            for (int s = 0; s < 4; ++s) {
                int sr = R.find(L.sec[sl].q + site_qn(s));
                if (sr < 0) continue;
                idx[(size_t)sl * 4 + s] = (int)blk.size();
                blk.push_back({sl, s, sr, n});
                n += (size_t)L.sec[sl].dim * R.sec[sr].dim;
            }
        d.alloc(n * sizeof(double), st);
    }
    int find(int sl, int s) const { return idx[(size_t)sl * 4 + s]; }
    double* ptr(const B& b) const { return d.as<double>() + b.off; }
};

// Environment (renormalised operators) at one cut for an MPO with state QN
// changes dq: blocks (a, sb, sk) with q_bra(sb) = q_ket(sk) + dq[a].  Blocks
// are stored ket sector by ket sector (a inner), so all blocks on one ket
// sector form one tall row-major panel (rows: the bra blocks of every a,
// width: dim(sk)); poff / prows give the panels, roff a block's first row.
struct EnvT {
    struct B { int a, sb, sk; size_t off; int roff; };
    std::vector<B> blk;
    std::vector<int> idx;   // a*nsk + sk -> block or -1
    std::vector<size_t> poff;
    std::vector<int> prows;
    int nsk = 0;
    size_t n = 0;
    DBuf d;
    // live (optional): MPO states whose blocks exist; the others are known
    // to be zero and are left out (find() returns -1 for them).  reuse: keep
    // the device buffer when it is large enough (stream-ordered reuse by a
    // caller that launches on one stream) instead of a fresh allocation.
    void build(const std::vector<QN>& dq, const Bond& bra, const Bond& ket, cudaStream_t st,
               const std::vector<char>* live = nullptr, bool reuse = false) {
        blk.clear();
        nsk = ket.nsec();
        idx.assign(dq.size() * (size_t)nsk, -1);
        poff.assign(nsk, 0);
        prows.assign(nsk, 0);
        n = 0;
        for (int sk = 0; sk < nsk; ++sk) {
            poff[sk] = n;
            for (int a = 0; a < (int)dq.size(); ++a) {
                if (live && !(*live)[a]) continue;
                int sb = bra.find(ket.sec[sk].q + dq[a]);
                if (sb < 0) continue;
                idx[(size_t)a * nsk + sk] = (int)blk.size();
                blk.push_back({a, sb, sk, n, prows[sk]});
                n += (size_t)bra.sec[sb].dim * ket.sec[sk].dim;
                prows[sk] += bra.sec[sb].dim;
            }
        }
        if (reuse) d.ensure(n * sizeof(double) + 8, st);
        else d.alloc(n * sizeof(double) + 8, st);
    }
    int find(int a, int sk) const { return idx[(size_t)a * nsk + sk]; }
    double* ptr(const B& b) const { return d.as<double>() + b.off; }
    double* panel(int sk) const { return d.as<double>() + poff[sk]; }
};

// Two-site tensor x[l, s1, s2, r]: blocks (sl, s1, s2) -> sr, stored in
// right-panel order (sr, sl, s1, s2) so that all blocks sharing a right
// sector form one tall row-major panel.  `allowed_mid` (if non-empty)
// restricts N of q(sl) + q(s1), the QN at the internal cut.
struct TwoT {
    struct B { int sl, s1, s2, sr; size_t off; int rows, cols; };
    struct Panel { int sr; int b0, b1; int rows; size_t off; };
    std::vector<B> blk;
    std::vector<int> idx;   // (sl*16 + s1*4 + s2) -> block or -1
    std::vector<Panel> panels;
    size_t n = 0;
    void build(const Bond& L, const Bond& R, const std::vector<int>& allowed_mid) {
        blk.clear();
        panels.clear();
        idx.assign((size_t)L.nsec() * 16, -1);
        n = 0;
        for (int sr = 0; sr < R.nsec(); ++sr) {
            Panel p{sr, (int)blk.size(), 0, 0, n};
            for (int sl = 0; sl < L.nsec(); ++sl)
                for (int s1 = 0; s1 < 4; ++s1) {
                    QN mid = L.sec[sl].q + site_qn(s1);
                    if (!allowed_mid.empty()) {
                        bool ok = false;
                        for (int v : allowed_mid) ok |= (mid.n == v);
                        if (!ok) continue;
                    }
                    for (int s2 = 0; s2 < 4; ++s2) {
                        if (!(mid + site_qn(s2) == R.sec[sr].q)) continue;
                        idx[(size_t)sl * 16 + s1 * 4 + s2] = (int)blk.size();
                        B b{sl, s1, s2, sr, n, L.sec[sl].dim, R.sec[sr].dim};
                        blk.push_back(b);
                        n += (size_t)b.rows * b.cols;
                        p.rows += b.rows;
                    }
                }
            p.b1 = (int)blk.size();
            if (p.b1 > p.b0) panels.push_back(p);
        }
    }
    int find(int sl, int s1, int s2) const { return idx[(size_t)sl * 16 + s1 * 4 + s2]; }
};

}  // namespace mpspt
