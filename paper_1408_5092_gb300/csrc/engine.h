// MPS-PT engine: problem set-up, the two-site Hylleraas sweep, expectation
// values.  Host code orchestrates; every contraction runs in the kernels.
#pragma once
#include <map>
#include <memory>
#include <vector>

#include "core.h"
#include "kernels.h"
#include "learned.h"
#include "mpo.h"
#include "plans.h"
#include "tensors.h"

namespace mpspt {

struct MpsD {
    int nsite = 0;
    std::vector<Bond> bond;      // nsite + 1 cuts
    std::vector<SiteT> A;        // nsite sites
};

// Host copy of a QN-labelled MPS (dense tensors, for import / export / init).
struct MpsHost {
    int nsite = 0;
    std::vector<Bond> bond;
    std::vector<std::vector<double>> T;  // dense D_l x 4 x D_r
};

struct Problem {
    int k = 0, ka = 0, kv = 0, nel = 0, nq = 0;
    std::vector<double> h, L, eri;       // semicanonical virtual basis
    std::vector<double> gamma, f, eps;   // 1-RDM (ka x ka), Fock (k x k), diag(f)
    double e_ref = 0.0;
    bool have_int = false, have_ref = false;
    std::vector<double> h_in, L_in;      // as given
    std::vector<double> ci;
};

// Per-stream resources of one concurrent solve: stream, reduction scratch,
// CG scalars and their pinned host mirrors, tensor-core error flag.
struct Lane {
    cudaStream_t st = 0;
    bool own_stream = false;
    DBuf red, cnt, cg, scal, tcerr;
    std::unique_ptr<PinnedRing> ring;   // staging of this lane's task lists
    void* rb = nullptr;                 // page-locked readback buffer
    size_t rb_bytes = 0;
    void* readback(size_t bytes);       // grows rb (after a stream sync) as needed
    CgState* cg_host = nullptr;
    double* scal_host = nullptr;
    explicit Lane(cudaStream_t s, bool create = false);
    ~Lane();
};

struct Ctx {
    mpspt_options opt;
    cudaStream_t st = 0;
    Problem P;
    MpsD psi0;                            // reference on the full chain
    std::map<int, MPO> mpoA, mpoV;        // keyed by H0 choice
    std::unique_ptr<MPO> mpoH, mpoI;
    // reduction scratch and CG scalars
    DBuf red, cnt, cg;
    CgState* cg_host = nullptr;           // pinned mirror
    double* scal_host = nullptr;          // pinned scalars
    DBuf scal;
    DBuf tcerr;                           // tensor-core kernel error flag
    std::string last_error;
    std::unique_ptr<Lane> lane0;          // resources on the context stream
    const Mlp* net = nullptr;             // learned initial guess (opt.use_learned)
    std::unique_ptr<Mlp> own_net;         // a network trained by mpspt_train_preconditioner
    std::unique_ptr<Autotuner> tuner;     // GEMM tile shapes (opt.autotune)
    std::string tuner_path;               // opt.autotune_cache
    // harvesting of training pairs from plain solves (block features -> the
    // least-squares (gamma, delta) of the converged solution)
    bool harvesting = false;
    size_t harvest_max = 0;
    std::vector<float> harvest_x, harvest_t;

    explicit Ctx(const mpspt_options& o);
    ~Ctx();
    double e0(int h0) const;
    const MPO& A_mpo(int h0);
    const MPO& V_mpo();
    const MPO& H_mpo();
    const MPO& I_mpo();
    void sync() { MPSPT_CUDA(cudaStreamSynchronize(st)); }
};

void set_integrals(Ctx& c, int ka, int kv, int nel, const double* h, const double* L, int nq);
void set_reference(Ctx& c, const double* ci, long long n);
// Reference as an active-space MPS (host tensors, any norm): gamma and E_ref
// by MPO transfers on the device, then finish_reference.
void set_reference_mps(Ctx& c, MpsHost act);
// With P.gamma, P.e_ref set and P.h / P.L / P.eri in the input basis: the
// generalised Fock matrix, semicanonical virtuals, eps and Psi0 on the full
// chain.
void finish_reference(Ctx& c, MpsHost& act);

struct SweepResult {
    double e2 = 0.0;
    std::vector<double> e2_sweep;
    double max_disc = 0.0;
    long long cg_iters = 0, sigma_calls = 0;
    double sigma_flops = 0.0, sigma_ms = 0.0, wall_ms = 0.0;
    int max_bond = 0;
    std::vector<double> sweep_ms;
    long long launches = 0;
    long long learned_used = 0, learned_rejected = 0;
    long long sigma64_calls = 0;
    double sigma64_flops = 0.0, sigma64_ms = 0.0;
    bool converged = false;              // last sweep met e_tol
    std::vector<long long> sigma_cum;    // sigma applications (all precisions) at each sweep end
    double host_wait_ms = 0.0;           // host time blocked in stream synchronisations
    std::vector<double> disc_sweep;      // max discarded weight of each sweep
};

// One MPS-PT problem on a chain of sites: the full space (active + all
// virtual orbitals) or one virtual-pair partition (active + a [+ b]).
struct Chain {
    int nsite = 0, ka = 0;
    QN target;
    std::vector<std::vector<int>> filt;   // allowed N_left per cut (empty = any)
    const MPO* WA = nullptr;              // H0 - E0 on the chain
    const MPO* WV = nullptr;              // RHS operator on the chain
    MpsD psi0;                            // reference on the chain (views)
    std::vector<int> orbs;                // full-space orbital of each site
    bool ground = false;                  // ground-state DMRG of WA (WV, psi0 unused)
};
struct PartOps {
    MPO A, V;
};
Chain full_chain(Ctx& c, int h0);
Chain partition_chain(Ctx& c, int h0, int a, int b, PartOps& ops);

std::unique_ptr<MpsD> minimize(Ctx& c, const Chain& ch, int M, SweepResult& res, Lane* lane = nullptr);
// Independent virtual-pair partitions, run concurrently on n_lanes streams;
// e2_part[i] receives E2 of pair i, the return value their sum in pair order.
double minimize_partitioned(Ctx& c, int h0, const std::vector<std::pair<int, int>>& pairs,
                            const std::vector<int>& Ms, int n_lanes, std::vector<double>& e2_part,
                            SweepResult& res);
std::unique_ptr<MpsD> minimize(Ctx& c, int h0, int M, SweepResult& res);
// Ground-state DMRG of H_act + s2_penalty S^2 in the (n_elec, Sz = 0) sector
// at bond dimension <= M0 (two-site sweep, Davidson local solver); installs
// the result as the reference and returns it (active sites only).
std::unique_ptr<MpsD> ground_state(Ctx& c, int M0, double s2_penalty, SweepResult& res);
double expectation(Ctx& c, const MPO& W, const MpsD& bra, const MpsD& ket);
double expectation(Ctx& c, const MPO& W, const MpsD& bra, const MpsD& ket, cudaStream_t st);
double third_order(Ctx& c, int h0, const MpsD& psi1);

// E3 (Eq. 5) of Psi1 = sum of the listed partitions' Psi1: the partitions
// are solved as in minimize_partitioned, kept, written on the full chain, and
//   E3 = sum_P E3(Psi1^P) + 2 sum_{P < P'} <Psi1^P|H|Psi1^P'>
// (partitions are orthogonal and H0 keeps every virtual occupation, so the
// cross terms of H0 and of the norm vanish).
struct PartE3 {
    double e2 = 0.0, e3 = 0.0, e3_cross = 0.0;
    double setup_ms = 0.0;        // operators of the E3 phase (H, H0 - E0, 1 MPOs and run maps)
    double e3_ms = 0.0;           // the transfers
    double wait_ms = 0.0;         // E3 phase: host time blocked on the device, summed over lanes
    double flops = 0.0;           // E3 phase: float64 GEMM flops of the transfers
    double plan_bytes = 0.0;      // E3 phase: task-list bytes uploaded
    long long transfers = 0;
    std::vector<double> e2_part, e3_part;
    std::vector<double> h_pair;   // n x n, <Psi1^i|H|Psi1^j> off the diagonal, 0 on it
};
double third_order_partitioned(Ctx& c, int h0, const std::vector<std::pair<int, int>>& pairs,
                               const std::vector<int>& Ms, int n_lanes, PartE3& out, SweepResult& res);
void embed_partition(const Problem& P, const MpsD& part, int a, int b, MpsD& out, cudaStream_t st);
void local_apply(Ctx& c, int h0, const MpsD& psi1, int i, int op, const double* x, double* out);

std::unique_ptr<MpsD> mps_upload(const MpsHost& h, cudaStream_t st);
MpsHost mps_download(const MpsD& m, cudaStream_t st);

}  // namespace mpspt
