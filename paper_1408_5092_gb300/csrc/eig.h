// Batched symmetric eigen-decomposition of the truncation step's density
// matrices (one dense block per composite QN sector).
#pragma once
#include <vector>

#include "core.h"
#include "kernels.h"
#include "plans.h"

namespace mpspt {

struct EigSolver {
    DBuf scratch, vt, g, djt, djt1, djtc, drows, dtns;
    // per task of the last stage run: 1 converged, 2 stopped by the sweep
    // cap (device ints, valid once the stream has reached them)
    DBuf flags;
    int nflags = 0;
    int* flag_host = nullptr;   // page-locked copy of the flags between sweep batches
    ~EigSolver() { if (flag_host) cudaFreeHost(flag_host); }
    GemmPlan ge;   // batched square GEMMs of the float64 stage
    bool stats = false;   // count sweeps per matrix (sum, matrices, max)
    long long sweeps32[3] = {0, 0, 0}, sweeps_polish[3] = {0, 0, 0}, sweeps64[3] = {0, 0, 0};

    // For every task: A (n x n, symmetric, left unchanged) -> V (eigenvectors
    // as columns) and w (unsorted eigenvalues).  All pointers must lie in
    // library allocations.  fp64_only: float64 Jacobi from the identity.
    // Otherwise three stages:
    //  1. cyclic Jacobi in float32 from the identity (the float64 pipe is the
    //     scarce one on this GPU), giving V orthonormal to float32 rounding;
    //  2. two Newton-Schulz steps V <- V (3/2 I - 1/2 V^T V) in float64, each
    //     squaring the departure from orthonormality;
    //  3. B = V^T A V in float64 (nearly diagonal) and float64 Jacobi on B
    //     starting from V, to the same float64 convergence test.
    void run(const std::vector<EigTask>& et, bool fp64_only, cudaStream_t st);

  private:
    // Jacobi from the given inputs (one per task) into the tasks' V (and w)
    void jacobi(const std::vector<EigTask>& et, const std::vector<const double*>& in, int vinit, bool f32, int maxs,
                bool want_w, cudaStream_t st, int batch = 0);
};

}  // namespace mpspt
