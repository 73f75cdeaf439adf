// Matrix product operators (Eq. 4) built from second-quantised term lists.
#pragma once
#include <array>
#include <map>
#include <memory>
#include <mutex>
#include <utility>
#include <vector>

#include "core.h"

namespace mpspt {

struct FOp {      // elementary fermion operator on spin-orbital j = 2p + s
    int j;
    bool dag;
};

struct Term {     // c * op[0] op[1] ... op[n-1] (product order)
    double c;
    int n;
    FOp op[4];
};

using Mat4 = std::array<double, 16>;   // row-major <n|o|n'> on |0>,|a>,|b>,|ab>

struct MpoEntry {
    int a, b;     // state at cut p, state at cut p+1
    int op;       // index into MPO::ops
    double coef;
};

struct MPO {
    int nsite = 0;
    std::vector<int> dim;                    // states per cut, cut = 0..nsite
    std::vector<std::vector<QN>> dq;         // QN change carried by each state
    std::vector<std::vector<MpoEntry>> W;    // per site, sorted by (a, b)
    std::vector<Mat4> ops;                   // local operator table
    // Entry indices of each site by source state (W[p][out_ptr[p][a] ..
    // out_ptr[p][a+1]]) and by target state (in_idx[p][in_ptr[p][b] ..
    // in_ptr[p][b+1]], in increasing a); filled by index().
    std::vector<std::vector<int>> out_ptr, in_ptr, in_idx;
    void index();
};

// Builds the MPO of sum(terms) on nsite sites.  Sites >= k_split are the
// "virtual" region (the centre rule differs there, see mpo.cpp).
MPO build_mpo(const std::vector<Term>& terms, int nsite, int k_split);

// Transfer of MPO states across a run of sites [s0, s1) on which bra and ket
// are both empty (identity sites, local state |0>): only the <0|o|0>
// element of each site operator acts, so the run is a sparse linear map of
// the MPO states at cut s0 to those at cut s1 (a state that needs a creator
// or annihilator on the run dies; the rest pass with their coefficients).
// CSR over the target states: sources of b are col[ptr[b] .. ptr[b+1]).
struct RunMap {
    std::vector<int> ptr, col;
    std::vector<double> val;
};

// Run maps of one MPO, computed on first use and shared by threads.
class RunMaps {
  public:
    explicit RunMaps(const MPO& W);
    const RunMap& get(int s0, int s1);

  private:
    const MPO& W;
    std::vector<std::vector<std::vector<std::pair<int, double>>>> out;   // site, a -> (b, coef <0|o|0>)
    std::mutex mu;
    std::map<std::pair<int, int>, std::unique_ptr<RunMap>> maps;
};

// Term generators (orbital index = site index).
void add_one_body(std::vector<Term>& out, const std::vector<double>& t, int k,
                  int p0, int p1, int q0, int q1);
// 1/2 sum (pq|rs) c+_ps c+_rt c_st c_qs over p in [p0,p1), q in [q0,q1),
// r in [p0,p1), s in [q0,q1), optionally keeping only quadruples with
// p >= vmin or r >= vmin.
void add_two_body(std::vector<Term>& out, const std::vector<double>& eri, int k,
                  int p0, int p1, int q0, int q1, int vmin);
void add_number(std::vector<Term>& out, const std::vector<double>& eps, int a0, int a1);

}  // namespace mpspt
