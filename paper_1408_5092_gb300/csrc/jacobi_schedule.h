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

// Pair schedule of one sweep.  A round is a list of slots; a slot is a pair
// (p < q) or a single index (q = -1) that is not rotated in that round, and
// every index is in exactly one slot, so the 2x2 block update over all slot
// pairs touches every matrix entry once.
//  mode 0: the round-robin ordering (m - 1 rounds of m/2 slots).
//  mode 1 (float64 polish after the float32 start): indices sorted by
//    decreasing diagonal; S = those within 1e-8 of the largest, the rest R.
//    Rounds: all S x S pairs (round robin on S), then all S x R pairs (the
//    smaller side against cyclic shifts of the larger), then R x R (round
//    robin on R).  Couplings of the large eigenvalues to the near-null
//    directions are removed before rotations inside the near-null cluster
//    move them around, which the round-robin order keeps doing sweep after
//    sweep (linear instead of quadratic convergence from a float32 start).
struct Sched {
    int mode, n, m, half;
    int kS, R, mS, mR, rA, rB, rC, a, b;
    bool smallS;
    const int* perm;
    JAC_HD void init(int mode_, int n_, const int* perm_, int kS_) {
        mode = mode_; n = n_; m = n + (n & 1); half = m / 2; perm = perm_;
        kS = kS_; R = n - kS;
        mS = kS + (kS & 1); mR = R + (R & 1);
        rA = kS >= 2 ? mS - 1 : 0;
        smallS = kS <= R;
        a = smallS ? kS : R;
        b = smallS ? R : kS;
        rB = (kS > 0 && R > 0) ? b : 0;
        rC = R >= 2 ? mR - 1 : 0;
    }
    JAC_HD int rounds() const { return mode == 0 ? m - 1 : rA + rB + rC; }
    JAC_HD int slots(int r) const {
        if (mode == 0) return half;
        if (r < rA) return mS / 2 + R;
        r -= rA;
        if (r < rB) return b;
        return mR / 2 + kS;
    }
    JAC_HD void slot(int r, int k, int& p, int& q) const {
        int x, y;
        if (mode == 0) {
            rr_pair(k, r, m, x, y);
            p = x < y ? x : y;
            q = x < y ? y : x;
            if (q >= n) q = -1;
            return;
        }
        if (r < rA) {
            if (k < mS / 2) {
                rr_pair(k, r, mS, x, y);
                const int lo = x < y ? x : y, hi = x < y ? y : x;
                p = perm[lo];
                q = hi < kS ? perm[hi] : -1;
            } else {
                p = perm[kS + (k - mS / 2)];
                q = -1;
            }
        } else if ((r -= rA) < rB) {
            const int jl = (k + r) % b;
            const int li = smallS ? kS + jl : jl;
            if (k < a) { p = perm[smallS ? k : kS + k]; q = perm[li]; }
            else { p = perm[li]; q = -1; }
        } else {
            r -= rB;
            if (k < mR / 2) {
                rr_pair(k, r, mR, x, y);
                const int lo = x < y ? x : y, hi = x < y ? y : x;
                p = perm[kS + lo];
                q = hi < R ? perm[kS + hi] : -1;
            } else {
                p = perm[k - mR / 2];
                q = -1;
            }
        }
        if (q >= 0 && q < p) { const int t = p; p = q; q = t; }
    }
};

}  // namespace mpspt
