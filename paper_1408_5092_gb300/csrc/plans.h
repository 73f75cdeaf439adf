// Planner: turns each contraction of the sweep into device task lists.
#pragma once
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "kernels.h"
#include "tensors.h"

namespace mpspt {

// GEMM_TC: split-bf16 tcgen05; GEMM_TC16: split-f16 tcgen05 (same tiles)
enum GemmKind { GEMM_F64 = 0, GEMM_F32 = 1, GEMM_TC = 2, GEMM_TC16 = 3 };
inline bool is_tc(int kind) { return kind == GEMM_TC || kind == GEMM_TC16; }

struct GemmPlan;

// Tile-shape autotuner of the CUDA-core grouped GEMM.  A plan's shape class
// is (arithmetic, skinny, and log2 buckets of the median block rows, columns
// and K-length and of the block count).  The first plan of a class times
// every candidate tile on its own operands (outputs redirected to scratch,
// so no result changes), keeps the fastest, and later plans of the class
// reuse it.  The table can be read from and written to a text file.
struct Autotuner {
    using Key = std::tuple<int, int, int, int, int, int>;
    std::mutex mu;
    std::map<Key, std::pair<int, int>> best;
    long long timed = 0, reused = 0;
    // Scratch outputs and task list of the timing launches.  Plans on any
    // lane call the tuner, and a lane's stream ends with its call, so these
    // are plain (not stream-ordered) allocations that outlive every lane.
    // A buffer that has to grow is kept (freed with the tuner) rather than
    // freed while other lanes may be capturing graphs.
    struct RawBuf {
        void* p = nullptr;
        size_t n = 0;
        std::vector<void*> old;
        void ensure(size_t bytes);
        ~RawBuf();
    };
    RawBuf scratch, dtasks;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    ~Autotuner();
    // (tm, tn) for the plan (its blocks recorded, its ops uploaded)
    std::pair<int, int> choose(const GemmPlan& g, cudaStream_t st);
    void load(const std::string& path);
    void save(const std::string& path);
};

struct GemmPlan {
    int tm = GEMM_TM, tn = GEMM_TN;   // output tile (TC kernel: 128 x 64; skinny: 16 x 128)
    Autotuner* tuner = nullptr;       // CUDA-core kinds only: choose the tile per shape class
    int kind = GEMM_F64;
    bool skinny = false;
    int* err = nullptr;               // TC kernel error flag (device)
    const int* skip = nullptr;        // device flag: launch becomes a no-op when set
    void set_kind(int k, int* e, bool skinny_ = false) {
        kind = k;
        err = e;
        skinny = skinny_ && !is_tc(k);
        if (is_tc(k)) { tm = tc_tile_m(); tn = tc_tile_n(); }
        else if (skinny) { tm = 16; tn = 128; }
        else { tm = GEMM_TM; tn = GEMM_TN; }
    }
    // output blocks as planned; split into tm x tn tasks at upload
    struct Blk {
        double* C;
        long long cmap_off;
        int ldc, m, n, accumulate, op0, op1, cmap_rows;
    };
    std::vector<Blk> blocks;
    std::vector<GemmTask> tasks;
    std::vector<GemmOp> ops;
    std::vector<int> cmaps;           // host copy of all column / row maps
    std::vector<long long> task_cmap; // per task: offset into cmaps or -1
    double flops = 0.0;   // algorithmic: sum over ops of 2 m n k (each product once)
    DBuf dtasks, dops, dcmaps;
    // split-K: partial tiles and their ordered reductions
    std::vector<SplitRed> reds;
    std::vector<long long> red_cmap;
    DBuf dreds, dpart;
    void clear() {
        blocks.clear(); tasks.clear(); ops.clear(); cmaps.clear(); task_cmap.clear(); reds.clear(); red_cmap.clear();
        flops = 0.0;
    }
    // K-chunks of a block: blocks with a small output and a long K-list are
    // summed by several CTAs (the chunking depends only on the block, not on
    // the tile shape, so every tile gives the same rounding)
    static int kchunks(long long m, long long n, long long K);
    // tasks of the recorded blocks for a tile shape (no cmap pointers yet);
    // with rd, split-K chunk tasks get partial-tile offsets (in doubles, from
    // the partial buffer's start) and rd receives the reductions
    void split(int tm_, int tn_, std::vector<GemmTask>& out, std::vector<long long>* cm,
               std::vector<SplitRed>* rd = nullptr, std::vector<long long>* rcm = nullptr,
               size_t* part_elems = nullptr) const;
    int mark() const { return (int)ops.size(); }
    void op(const double* A, int lda, const double* B, int ldb, int k, int trans, double alpha) {
        if (k <= 0) return;
        ops.push_back({A, B, lda, ldb, k, trans, alpha});
    }
    long long add_cmap(const std::vector<int>& m) {
        long long o = (long long)cmaps.size();
        cmaps.insert(cmaps.end(), m.begin(), m.end());
        return o;
    }
    // close the output block C (m x n) whose K-list is ops[op0, end); with
    // cmap_off >= 0 the element addresses come from the map (see GemmTask)
    void block(double* C, int ldc, int m, int n, int accumulate, int op0, long long cmap_off = -1,
               int cmap_rows = 0);
    void upload(cudaStream_t st);
    void run(cudaStream_t st) const;
};

// Two-site operator sum_{a,c} L_a (Omega_ac) R_c with Omega_ac = sum_b W1_ab (x) W2_bc.
struct Omega {
    struct E { int a, c, out, in; double v; };   // out/in = s1*4 + s2
    std::vector<E> e;                              // sorted by (a, out, c, in)
    std::vector<int> first;                        // first entry per (a*16 + out), size Da*16+1
    int Da = 0;
    void build(const MPO& W, int i);
    int begin(int a, int out) const { return first[(size_t)a * 16 + out]; }
    int end(int a, int out) const { return first[(size_t)a * 16 + out + 1]; }
};

// sigma-type application: out(bra layout) = sum L_a Omega_ac R_c x(ket layout).
// Per bond step the environments are packed per sector (Rpack: all R_c
// blocks on one ket right sector stacked; Lpack: all L_a blocks on one bra
// left sector side by side).  Then per application:
//   g1:  T_p = x_panel(p) Rpack^T           one GEMM per ket right sector
//   mix: V_stack(sl) = sum Omega coef T      memory-bound block sums
//   g2:  out(sl, :) = Lpack(sl) V_stack(sl)  one long-K GEMM per bra left
//        sector, scattered into the two-site layout by a column map
struct TwoSitePlan {
    GemmPlan g1, g2, g2s;            // g2: wide rows, g2s: few rows (skinny tiles)
    std::vector<MixTask> mtasks;
    std::vector<MixSrc> msrc;
    DBuf dmt, dms;
    DBuf T, V, Lp, Rp, pk;
    size_t tsize = 0;
    int kind = GEMM_F64;
    const int* skip = nullptr;
    void set_kind(int k, int* e) {
        kind = k;
        g1.set_kind(k, e);
        g2.set_kind(k, e);
        g2s.set_kind(k, e, true);
    }
    void set_skip(const int* s) { skip = s; g1.skip = s; g2.skip = s; g2s.skip = s; }
    void set_tuner(Autotuner* t) { g1.tuner = t; g2.tuner = t; g2s.tuner = t; }
    void build(const Omega& om, const TwoT& bra, const TwoT& ket, const Bond& braL,
               const Bond& ketL, const Bond& braR, const Bond& ketR, const EnvT& L,
               const EnvT& R, const std::vector<QN>& dqR, const double* x, double* out,
               cudaStream_t st);
    void run(cudaStream_t st) const {
        g1.run(st);
        launch_mix(dmt.as<MixTask>(), (int)mtasks.size(), dms.as<MixSrc>(), st, skip);
        g2.run(st);
        g2s.run(st);
    }
    double flops() const { return g1.flops + g2.flops + g2s.flops; }
};

// Jacobi diagonal of sum L_a Omega_ac R_c on the bra layout.
struct DiagPlan {
    std::vector<DiagTask> tasks;
    std::vector<DiagTerm> terms;
    DBuf dt, dterm;
    void build(const Omega& om, const TwoT& x, const Bond& L, const Bond& R, const EnvT& Le,
               const EnvT& Re, const std::vector<QN>& dqL, const std::vector<QN>& dqR,
               double* out, cudaStream_t st);
    void run(cudaStream_t st) const;
};

// x[sl,s1,s2,sr] = A_i[sl,s1,sm] A_{i+1}[sm,s2,sr]
void plan_product(GemmPlan& g, const TwoT& x, double* xd, const Bond& mid, const SiteT& A,
                  const SiteT& B, const Bond& L);

// Left transfer: Lnew_b = sum (a,s,t) W_ab[s,t] Abra(s)^T L_a Aket(t); Y scratch.
// Environment update in three steps (the same scheme as sigma):
//   g1:  Y_kb = L_panel(ket sector of kb) A_ket(kb)     one GEMM per ket block
//        (right update: Y_kb = A_ket(kb) R_panel^T)
//   mix: Z_(out, s) = sum over MPO entries and t of W_ab(s, t) Y_(a, kb(t))
//   g2:  L_new(out) = sum_s A_bra(s)^T Z_(out, s)          (<= 4 products)
struct EnvPlan {
    GemmPlan g1, g2;
    void set_tuner(Autotuner* t) { g1.tuner = t; g2.tuner = t; }
    DBuf Y, Z, dmt, dms;
    std::vector<MixTask> mt;
    std::vector<MixSrc> ms;
    void build_left(const MPO& W, int site, const EnvT& L, const SiteT& Abra, const SiteT& Aket,
                    const Bond& braL, const Bond& ketL, const Bond& braR, const Bond& ketR,
                    EnvT& Lnew, cudaStream_t st);
    void build_right(const MPO& W, int site, const EnvT& R, const SiteT& Abra, const SiteT& Aket,
                     const Bond& braL, const Bond& ketL, const Bond& braR, const Bond& ketR,
                     EnvT& Rnew, cudaStream_t st);
    // L_new = L carried across a run of empty sites (one mix launch; the
    // bonds do not change across the run).
    void build_left_run(const RunMap& T, const EnvT& L, const Bond& bra, const Bond& ket, EnvT& Lnew,
                        cudaStream_t st);
    void run(cudaStream_t st) const {
        g1.run(st);
        launch_mix(dmt.as<MixTask>(), (int)mt.size(), dms.as<MixSrc>(), st);
        g2.run(st);
    }
    double flops() const { return g1.flops + g2.flops; }
    // bytes of the task lists the last build uploads (GEMM tasks and operand
    // lists, mix tasks and sources)
    size_t plan_bytes() const {
        return mt.size() * sizeof(MixTask) + ms.size() * sizeof(MixSrc) +
               (g1.tasks.size() + g2.tasks.size()) * sizeof(GemmTask) +
               (g1.ops.size() + g2.ops.size()) * sizeof(GemmOp);
    }

  private:
    void upload_mix(cudaStream_t st);
};

}  // namespace mpspt
