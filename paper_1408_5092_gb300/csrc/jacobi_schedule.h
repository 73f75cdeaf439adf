// Pair schedules of the batched Jacobi eigensolver (kernels_eig.cu).  Host
// and device code: the host tests check the schedules' coverage.
#pragma once

#if defined(__CUDACC__)
#define JAC_HD __host__ __device__ __forceinline__
#else
#define JAC_HD inline
#endif

namespace mpspt {

// Round-robin ordering: in round r (0 <= r < m - 1) slot k pairs (pa, pb);
// over the m - 1 rounds every pair of 0 .. m-1 meets exactly once.
JAC_HD void rr_pair(int k, int r, int m, int& pa, int& pb) {
    pa = (k == 0) ? 0 : ((k - 1 + r) % (m - 1)) + 1;
    pb = ((m - 1 - k - 1 + r) % (m - 1)) + 1;
}

// Pair schedule of one sweep: the round-robin ordering, m - 1 rounds of
// m/2 slots (m = n rounded up to even).  A slot is a pair (p < q) or a
// single index (q = -1) that is not rotated in that round; every index is
// in exactly one slot per round, so the 2x2 block update over all slot
// pairs touches every matrix entry once, and every pair meets once per
// sweep.
struct Sched {
    int n, m, half;
    JAC_HD void init(int n_) {
        n = n_; m = n + (n & 1); half = m / 2;
    }
    JAC_HD int rounds() const { return m - 1; }
    JAC_HD int slots(int) const { return half; }
    JAC_HD void slot(int r, int k, int& p, int& q) const {
        int x, y;
        rr_pair(k, r, m, x, y);
        p = x < y ? x : y;
        q = x < y ? y : x;
        if (q >= n) q = -1;
    }
};

}  // namespace mpspt
