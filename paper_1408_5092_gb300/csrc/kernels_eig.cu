// Batched cyclic Jacobi for the density-matrix eigenproblems of the
// truncation step, one launch per sweep.
//
// k_jac_sweep (one CTA of 512 threads per matrix): the symmetric matrix is
// kept as its packed upper triangle, in shared memory when it fits (float64
// up to n = 215, float32 up to n = 305), else in the task's global scratch.
// A sweep is the m-1 rounds of the round-robin ordering; in a round the m/2
// disjoint pairs get their rotations (threshold: negligible a_pq are
// skipped), then every unordered 2x2 block {k, l} of pairs is updated once
// (R_k^T A_kl R_l; the symmetric partner is implied).  The applied rotations
// of each round are recorded, compacted, in the task's rotation list.
//
// k_jac_apply (one warp per block of rows of V): V <- V R for the
// recorded rotations, in order.  A row of V is touched independently of the
// others, so each lane owns one row in shared memory and runs through the
// whole list without synchronisation; the work spreads over many SMs.
//
// The host launches sweep 0, apply 0, sweep 1, apply 1, ... up to maxs.  A
// sweep first measures off(A)^2 and stops the task (flag, eigenvalues
// written) when off^2 <= STOP * |A|_F^2, when a small off-norm stalled at
// the rounding floor, or at sweep maxs; later launches for that task return
// at once.
#include <cooperative_groups.h>

#include "jacobi_schedule.h"
#include "kernels.h"

namespace mpspt {
namespace {

constexpr int JAC_THREADS = 512;
constexpr int JAC_SMEM = 200704;     // dynamic shared memory of the sweep kernel

template <class T>
struct RotE {
    T c, s;
    int p, q;
};

// stop: off(A)^2 <= stop |A|_F^2; a pair is not rotated when |a_pq| <= skip
// sqrt|a_pp a_qq| or |a_pq| <= absf |A|_F; a solve that reached off(A)^2 <=
// stall |A|_F^2 also ends when a sweep shrinks off(A)^2 by less than 19%.
// (A rounding-level absf and a tighter float64 stall let the solves end
// sooner but moved the sweep's energies by 1e-7..1e-6 against the oracle;
// the values below keep float64 parity.)
template <class T>
struct JacTol;
template <>
struct JacTol<double> {
    static constexpr double stop = 1e-30, skip = 1e-18, absf = 0.0, stall = 1e-8, null = 1e-14;
};
template <>
struct JacTol<float> {
    static constexpr double stop = 1e-11, skip = 1e-9, absf = 0.0, stall = 1e-8, null = 0.0;
};
// Null pairs: a pair (p, q) whose 2x2 block has every entry below
// null * |A|_F is neither rotated nor counted in the off-diagonal norm.  Its
// eigenvalues are below 2 null |A|_F, so inside such a cluster the vectors
// are set by rounding anyway; every coupling of a null index to a larger
// entry is still rotated away.  For the density matrices of the truncation
// (positive semidefinite) in float64 these are the exactly rank-deficient
// directions, far below the keep threshold; skipping them saves the sweeps
// the polish spent circulating rounding noise inside the null cluster.  The
// float32 start sweeps every pair (a null level at float32 resolution,
// 1e-6, saved float32 sweeps but cost as many float64 polish sweeps).


__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// Rounds of one sweep at most (either schedule), and the rotation-list
// layout: [nrounds][rcount per round] then `half` entries per round.
__host__ __device__ inline int jac_max_rounds(int n) { return 2 * n + 4; }
__host__ __device__ inline size_t jac_rot_head(int n) { return align16((size_t)(1 + jac_max_rounds(n)) * 4); }

// shared-memory head of the sweep kernels: rowoff, Pp, Qq (n ints each, room
// for four), Cc, Ss (n T each) and n doubles of headroom; the packed
// triangle follows
template <class T>
__host__ __device__ inline size_t jac_head_bytes(int n) {
    return align16((size_t)n * 16) + align16(2 * (size_t)n * sizeof(T)) + align16((size_t)n * 8);
}

template <class T>
__global__ void __launch_bounds__(JAC_THREADS) k_jac_sweep(const JacTask* __restrict__ tasks, int sweep, int maxs) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ double red[2][JAC_THREADS / 32];
    __shared__ double thr;
    __shared__ int stop, cnt;
    const JacTask t = tasks[blockIdx.x];
    if (sweep > 0 && *(volatile const int*)t.done) return;
    const int n = t.n;
    const int m = n + (n & 1), half = m / 2;
    const size_t np = (size_t)n * (n + 1) / 2;
    int* rowoff = reinterpret_cast<int*>(sm);
    int* Pp = rowoff + n;
    int* Qq = Pp + n;
    T* Cc = reinterpret_cast<T*>(sm + align16((size_t)n * 16));
    T* Ss = Cc + n;
    const size_t head = jac_head_bytes<T>(n);
    const bool p_sm = head + np * sizeof(T) <= (size_t)JAC_SMEM;
    T* P = p_sm ? reinterpret_cast<T*>(sm + head) : reinterpret_cast<T*>(t.P);
    T* Pg = reinterpret_cast<T*>(t.P);
    int* rhead = reinterpret_cast<int*>(t.rot);          // [0]: rounds, [1 + r]: count of round r
    RotE<T>* rlist = reinterpret_cast<RotE<T>*>(reinterpret_cast<unsigned char*>(t.rot) + jac_rot_head(n));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = JAC_THREADS / 32;
    for (int i = tid; i < n; i += JAC_THREADS) rowoff[i] = i * n - i * (i + 1) / 2;
    __syncthreads();
    if (sweep == 0) {
        for (int e = tid; e < n * n; e += JAC_THREADS) {
            const int i = e / n, j = e % n;
            if (j >= i) P[rowoff[i] + j] = (T)t.A[e];
        }
    } else if (p_sm) {
        for (size_t e = tid; e < np; e += JAC_THREADS) P[e] = Pg[e];
    }
    __syncthreads();
    auto S = [&](int a, int b) -> T& { return a <= b ? P[rowoff[a] + b] : P[rowoff[b] + a]; };
    // convergence test: |A|_F first (it sets the null level), then the
    // off-diagonal norm without null pairs
    __shared__ double nullv;
    {
        double all = 0.0;
        for (int i = warp; i < n; i += nw)
            for (int j = i + lane; j < n; j += 32) {
                const double v = (double)P[rowoff[i] + j];
                all += (j == i ? 1.0 : 2.0) * v * v;
            }
        for (int o = 16; o > 0; o >>= 1) all += __shfl_xor_sync(0xffffffffu, all, o);
        if (lane == 0) red[1][warp] = all;
        __syncthreads();
        if (tid == 0) {
            double sa = 0.0;
            for (int w = 0; w < nw; ++w) sa += red[1][w];
            nullv = JacTol<T>::null * sqrt(sa);
        }
        __syncthreads();
        const double nv = nullv;
        double off = 0.0;
        all = 0.0;
        for (int i = warp; i < n; i += nw) {
            const double di = fabs((double)P[rowoff[i] + i]);
            for (int j = i + lane; j < n; j += 32) {
                const double v = (double)P[rowoff[i] + j];
                if (j == i) { all += v * v; continue; }
                if (fabs(v) < nv && di < nv && fabs((double)P[rowoff[j] + j]) < nv) all += 2.0 * v * v;
                else off += 2.0 * v * v;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            all += __shfl_xor_sync(0xffffffffu, all, o);
        }
        __syncthreads();
        if (lane == 0) { red[0][warp] = off; red[1][warp] = all; }
        __syncthreads();
        if (tid == 0) {
            double so = 0.0, sd = 0.0;
            for (int w = 0; w < nw; ++w) { so += red[0][w]; sd += red[1][w]; }
            const double sa = so + sd;
            const double prev = sweep == 0 ? 1e300 : *t.prev;
            const int conv = (so <= JacTol<T>::stop * sa) || sa == 0.0 ||
                             (so <= JacTol<T>::stall * sa && so > 0.81 * prev) || n < 2;
            const int s = conv || sweep >= maxs;
            *t.prev = so;
            *t.done = s ? (conv ? 1 : 2) : 0;   // 2: stopped by the sweep cap
            if (s) *t.nsw = sweep;
            stop = s;
            thr = JacTol<T>::absf * sqrt(sa);
        }
        __syncthreads();
    }
    if (stop) {
        if (t.w)
            for (int i = tid; i < n; i += JAC_THREADS) t.w[i] = (double)P[rowoff[i] + i];
        return;
    }
    Sched sc;
    sc.init(n);
    const int nr = sc.rounds();
    if (tid == 0) rhead[0] = nr;
    constexpr T SKIP = (T)JacTol<T>::skip;
    for (int r = 0; r < nr; ++r) {
        const int ns = sc.slots(r);
        if (tid == 0) cnt = 0;
        __syncthreads();
        for (int k = tid; k < ns; k += JAC_THREADS) {
            int p, q;
            sc.slot(r, k, p, q);
            T c = T(1), s = T(0);
            if (q >= 0) {
                const T apq = P[rowoff[p] + q];
                const T app = P[rowoff[p] + p], aqq = P[rowoff[q] + q];
                const bool null_pair = (double)fabs(apq) < nullv && (double)fabs(app) < nullv &&
                                       (double)fabs(aqq) < nullv;
                if (!null_pair && fabs(apq) > SKIP * sqrt(fabs(app * aqq)) && (double)fabs(apq) > thr &&
                    apq != T(0)) {
                    const T th = (aqq - app) / (T(2) * apq);
                    const T tt = (th >= T(0) ? T(1) : T(-1)) / (fabs(th) + sqrt(th * th + T(1)));
                    c = T(1) / sqrt(tt * tt + T(1));
                    s = tt * c;
                }
            }
            Pp[k] = p; Qq[k] = q; Cc[k] = c; Ss[k] = s;
            if (s != T(0)) {
                const int slot = atomicAdd(&cnt, 1);   // pairs of a round commute: order is free
                rlist[(size_t)r * half + slot] = RotE<T>{c, s, p, q};
            }
        }
        __syncthreads();
        if (tid == 0) rhead[1 + r] = cnt;
        for (int k = warp; k < ns; k += nw) {
            const int p = Pp[k], q = Qq[k];
            const T ck = Cc[k], sk = Ss[k];
            for (int l = k + lane; l < ns; l += 32) {
                const T cl = Cc[l], sl = Ss[l];
                if (sk == T(0) && sl == T(0)) continue;
                if (l == k) {
                    const T app = S(p, p), apq = S(p, q), aqq = S(q, q);
                    const T r_pp = ck * app - sk * apq, r_pq = ck * apq - sk * aqq;
                    const T r_qp = sk * app + ck * apq, r_qq = sk * apq + ck * aqq;
                    S(p, p) = ck * r_pp - sk * r_pq;
                    S(q, q) = sk * r_qp + ck * r_qq;
                    S(p, q) = T(0);
                    continue;
                }
                const int u = Pp[l], v = Qq[l];
                const bool hq = q >= 0, hv = v >= 0;
                const T a_pu = S(p, u);
                const T a_pv = hv ? S(p, v) : T(0);
                const T a_qu = hq ? S(q, u) : T(0);
                const T a_qv = (hq && hv) ? S(q, v) : T(0);
                const T r_pu = ck * a_pu - sk * a_qu, r_qu = sk * a_pu + ck * a_qu;
                const T r_pv = ck * a_pv - sk * a_qv, r_qv = sk * a_pv + ck * a_qv;
                S(p, u) = cl * r_pu - sl * r_pv;
                if (hv) S(p, v) = sl * r_pu + cl * r_pv;
                if (hq) S(q, u) = cl * r_qu - sl * r_qv;
                if (hq && hv) S(q, v) = sl * r_qu + cl * r_qv;
            }
        }
        __syncthreads();
    }
    if (p_sm)
        for (size_t e = tid; e < np; e += JAC_THREADS) Pg[e] = P[e];
}

// Float64 sweep of one matrix by a cluster of JC CTAs (distributed shared
// memory).  Packed entry e lives in CTA e mod JC at slot e / JC.  Every CTA
// computes all rotations of a round from the distributed entries; the 2x2
// blocks {k, l} (k <= l) are split by k mod JC, so each CTA does 1/JC of the
// float64 update work on its own SM.  Two cluster barriers per round keep
// the pair phase and the update phase apart.  The arithmetic per entry is
// the single-CTA kernel's; only rank 0 records rotations and flags.
constexpr int JC = 8;

template <class T>
__global__ void __cluster_dims__(JC, 1, 1) __launch_bounds__(JAC_THREADS)
    k_jac_sweep_cl(const JacTask* __restrict__ tasks, int sweep, int maxs) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ double red[2][JAC_THREADS / 32];
    __shared__ double part[2][JC];
    __shared__ double thr;
    __shared__ int stop, cnt;
    const int rank = (int)cl.block_rank();
    const JacTask t = tasks[blockIdx.x / JC];
    if (sweep > 0 && *(volatile const int*)t.done) return;   // same value in every CTA of the cluster
    const int n = t.n;
    const int m = n + (n & 1), half = m / 2;
    const size_t np = (size_t)n * (n + 1) / 2;
    const size_t nloc = (np + JC - 1) / JC;
    int* rowoff = reinterpret_cast<int*>(sm);
    int* Pp = rowoff + n;
    int* Qq = Pp + n;
    T* Cc = reinterpret_cast<T*>(sm + align16((size_t)n * 16));
    T* Ss = Cc + n;
    T* Ploc = reinterpret_cast<T*>(sm + jac_head_bytes<T>(n));
    T* Pg = reinterpret_cast<T*>(t.P);
    int* rhead = reinterpret_cast<int*>(t.rot);
    RotE<T>* rlist = reinterpret_cast<RotE<T>*>(reinterpret_cast<unsigned char*>(t.rot) + jac_rot_head(n));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = JAC_THREADS / 32;
    for (int i = tid; i < n; i += JAC_THREADS) rowoff[i] = i * n - i * (i + 1) / 2;
    __syncthreads();
    if (sweep == 0) {
        for (int i = warp; i < n; i += nw)
            for (int j = i + lane; j < n; j += 32) {
                const size_t e = (size_t)rowoff[i] + j;
                if ((int)(e % JC) == rank) Ploc[e / JC] = (T)t.A[(size_t)i * n + j];
            }
    } else {
        for (size_t q = tid; q < nloc; q += JAC_THREADS) {
            const size_t e = q * JC + rank;
            if (e < np) Ploc[q] = Pg[e];
        }
    }
    cl.sync();   // every CTA of the cluster is running and has its slice before any remote access
    auto S = [&](int a, int b) -> T& {
        const size_t e = a <= b ? (size_t)rowoff[a] + b : (size_t)rowoff[b] + a;
        return cl.map_shared_rank(Ploc, (int)(e % JC))[e / JC];
    };
    // convergence test over the whole matrix (partial sums gathered in rank
    // 0): |A|_F first (it sets the null level, broadcast to every CTA), then
    // the off-diagonal norm without null pairs; the diagonal is copied into
    // the head's spare space so the null test reads it locally
    __shared__ double nullv;
    double* dg = reinterpret_cast<double*>(sm + align16((size_t)n * 16) + align16(2 * (size_t)n * sizeof(T)));
    {
        double all = 0.0;
        for (int i = warp; i < n; i += nw)
            for (int j = i + lane; j < n; j += 32) {
                const size_t e = (size_t)rowoff[i] + j;
                if ((int)(e % JC) != rank) continue;
                const double v = (double)Ploc[e / JC];
                all += (j == i ? 1.0 : 2.0) * v * v;
            }
        for (int o = 16; o > 0; o >>= 1) all += __shfl_xor_sync(0xffffffffu, all, o);
        if (lane == 0) red[1][warp] = all;
        __syncthreads();
        if (tid == 0) {
            double sd = 0.0;
            for (int w = 0; w < nw; ++w) sd += red[1][w];
            cl.map_shared_rank(&part[0][0], 0)[rank] = sd;
        }
        for (int i = tid; i < n; i += JAC_THREADS) {
            const size_t e = (size_t)rowoff[i] + i;
            dg[i] = (double)cl.map_shared_rank(Ploc, (int)(e % JC))[e / JC];
        }
        cl.sync();
        if (rank == 0 && tid == 0) {
            double sa = 0.0;
            for (int r = 0; r < JC; ++r) sa += part[0][r];
            const double nvv = JacTol<T>::null * sqrt(sa);
            for (int r = 0; r < JC; ++r) *cl.map_shared_rank(&nullv, r) = nvv;
        }
        cl.sync();
        const double nv = nullv;
        double off = 0.0;
        all = 0.0;
        for (int i = warp; i < n; i += nw)
            for (int j = i + lane; j < n; j += 32) {
                const size_t e = (size_t)rowoff[i] + j;
                if ((int)(e % JC) != rank) continue;
                const double v = (double)Ploc[e / JC];
                if (j == i) { all += v * v; continue; }
                if (fabs(v) < nv && fabs(dg[i]) < nv && fabs(dg[j]) < nv) all += 2.0 * v * v;
                else off += 2.0 * v * v;
            }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            all += __shfl_xor_sync(0xffffffffu, all, o);
        }
        __syncthreads();
        if (lane == 0) { red[0][warp] = off; red[1][warp] = all; }
        __syncthreads();
        if (tid == 0) {
            double so = 0.0, sd = 0.0;
            for (int w = 0; w < nw; ++w) { so += red[0][w]; sd += red[1][w]; }
            double* p0 = cl.map_shared_rank(&part[0][0], 0);
            p0[rank] = so;
            p0[JC + rank] = sd;
        }
        cl.sync();
        if (rank == 0 && tid == 0) {
            double so = 0.0, sd = 0.0;
            for (int r = 0; r < JC; ++r) { so += part[0][r]; sd += part[1][r]; }
            const double sa = so + sd;
            const double prev = sweep == 0 ? 1e300 : *t.prev;
            const int conv = (so <= JacTol<T>::stop * sa) || sa == 0.0 ||
                             (so <= JacTol<T>::stall * sa && so > 0.81 * prev) || n < 2;
            const int s = conv || sweep >= maxs;
            *t.prev = so;
            *t.done = s ? (conv ? 1 : 2) : 0;   // 2: stopped by the sweep cap
            if (s) *t.nsw = sweep;
            const double th = JacTol<T>::absf * sqrt(sa);
            for (int r = 0; r < JC; ++r) { *cl.map_shared_rank(&stop, r) = s; *cl.map_shared_rank(&thr, r) = th; }
        }
        cl.sync();
    }
    if (stop) {
        if (t.w)
            for (int i = tid; i < n; i += JAC_THREADS) {
                const size_t e = (size_t)rowoff[i] + i;
                if ((int)(e % JC) == rank) t.w[i] = (double)Ploc[e / JC];
            }
        return;
    }
    Sched sc;
    sc.init(n);
    const int nr = sc.rounds();
    if (rank == 0 && tid == 0) rhead[0] = nr;
    constexpr T SKIP = (T)JacTol<T>::skip;
    for (int r = 0; r < nr; ++r) {
        const int ns = sc.slots(r);
        if (tid == 0) cnt = 0;
        __syncthreads();
        for (int k = tid; k < ns; k += JAC_THREADS) {
            int p, q;
            sc.slot(r, k, p, q);
            T c = T(1), s = T(0);
            if (q >= 0) {
                const T apq = S(p, q), app = S(p, p), aqq = S(q, q);
                const bool null_pair = (double)fabs(apq) < nullv && (double)fabs(app) < nullv &&
                                       (double)fabs(aqq) < nullv;
                if (!null_pair && fabs(apq) > SKIP * sqrt(fabs(app * aqq)) && (double)fabs(apq) > thr &&
                    apq != T(0)) {
                    const T th = (aqq - app) / (T(2) * apq);
                    const T tt = (th >= T(0) ? T(1) : T(-1)) / (fabs(th) + sqrt(th * th + T(1)));
                    c = T(1) / sqrt(tt * tt + T(1));
                    s = tt * c;
                }
            }
            Pp[k] = p; Qq[k] = q; Cc[k] = c; Ss[k] = s;
            if (rank == 0 && s != T(0)) {
                const int slot = atomicAdd(&cnt, 1);
                rlist[(size_t)r * half + slot] = RotE<T>{c, s, p, q};
            }
        }
        __syncthreads();
        if (rank == 0 && tid == 0) rhead[1 + r] = cnt;
        cl.sync();   // every CTA has read the pair entries before any is updated
        for (int k = rank + JC * warp; k < ns; k += JC * nw) {
            const int p = Pp[k], q = Qq[k];
            const T ck = Cc[k], sk = Ss[k];
            for (int l = k + lane; l < ns; l += 32) {
                const T cl_ = Cc[l], sl = Ss[l];
                if (sk == T(0) && sl == T(0)) continue;
                if (l == k) {
                    const T app = S(p, p), apq = S(p, q), aqq = S(q, q);
                    const T r_pp = ck * app - sk * apq, r_pq = ck * apq - sk * aqq;
                    const T r_qp = sk * app + ck * apq, r_qq = sk * apq + ck * aqq;
                    S(p, p) = ck * r_pp - sk * r_pq;
                    S(q, q) = sk * r_qp + ck * r_qq;
                    S(p, q) = T(0);
                    continue;
                }
                const int u = Pp[l], v = Qq[l];
                const bool hq = q >= 0, hv = v >= 0;
                const T a_pu = S(p, u);
                const T a_pv = hv ? S(p, v) : T(0);
                const T a_qu = hq ? S(q, u) : T(0);
                const T a_qv = (hq && hv) ? S(q, v) : T(0);
                const T r_pu = ck * a_pu - sk * a_qu, r_qu = sk * a_pu + ck * a_qu;
                const T r_pv = ck * a_pv - sk * a_qv, r_qv = sk * a_pv + ck * a_qv;
                S(p, u) = cl_ * r_pu - sl * r_pv;
                if (hv) S(p, v) = sl * r_pu + cl_ * r_pv;
                if (hq) S(q, u) = cl_ * r_qu - sl * r_qv;
                if (hq && hv) S(q, v) = sl * r_qu + cl_ * r_qv;
            }
        }
        cl.sync();   // updates visible to every CTA before the next pair phase
    }
    for (size_t q = tid; q < nloc; q += JAC_THREADS) {
        const size_t e = q * JC + rank;
        if (e < np) Pg[e] = Ploc[q];
    }
}

template <class T>
__global__ void __launch_bounds__(32) k_jac_apply(const JacTask* __restrict__ tasks, const JacRows* __restrict__ rb,
                                                 int sweep) {
    extern __shared__ __align__(16) unsigned char sm[];
    const JacRows b = rb[blockIdx.x];
    const JacTask t = tasks[b.task];
    const int done = *(volatile const int*)t.done;
    if (sweep > 0 && done) return;
    const int n = t.n, ld = n | 1, lane = threadIdx.x;
    T* R = reinterpret_cast<T*>(sm);
    for (int e = lane; e < b.rows * n; e += 32) {
        const int i = e / n, j = e % n;
        R[i * ld + j] = (sweep == 0 && !t.vinit) ? T(b.r0 + i == j ? 1 : 0) : (T)t.V[(size_t)(b.r0 + i) * n + j];
    }
    __syncwarp();
    if (!done) {   // the whole warp takes part (shuffles); lanes >= rows only relay rotations
        const int m = n + (n & 1), half = m / 2;
        const int* rhead = reinterpret_cast<const int*>(t.rot);
        const RotE<T>* rlist =
            reinterpret_cast<const RotE<T>*>(reinterpret_cast<const unsigned char*>(t.rot) + jac_rot_head(n));
        const int nr = __ldg(rhead);
        for (int r = 0; r < nr; ++r) {
            const int c = __ldg(rhead + 1 + r);
            const RotE<T>* L = rlist + (size_t)r * half;
            // the rotations of one round act on disjoint columns.  The warp
            // reads 32 of them at a time, one per lane (coalesced), and hands
            // them round by shuffles; each lane then runs them on its own row
            // eight at a time, all loads before all stores.
            for (int j0 = 0; j0 < c; j0 += 32) {
                const int cnt = min(32, c - j0);
                RotE<T> mine{};
                if (lane < cnt) mine = L[j0 + lane];
                for (int q0 = 0; q0 < cnt; q0 += 8) {
                    const int nq = min(8, cnt - q0);
                    T cs[8], sn[8], x[8], y[8];
                    int pp[8], qq[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int src = q0 + (q < nq ? q : 0);
                        cs[q] = __shfl_sync(0xffffffffu, mine.c, src);
                        sn[q] = __shfl_sync(0xffffffffu, mine.s, src);
                        pp[q] = __shfl_sync(0xffffffffu, mine.p, src);
                        qq[q] = __shfl_sync(0xffffffffu, mine.q, src);
                    }
                    if (lane < b.rows) {
                        T* row = R + lane * ld;
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            if (q < nq) { x[q] = row[pp[q]]; y[q] = row[qq[q]]; }
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            if (q < nq) {
                                row[pp[q]] = cs[q] * x[q] - sn[q] * y[q];
                                row[qq[q]] = sn[q] * x[q] + cs[q] * y[q];
                            }
                    }
                }
            }
        }
    }
    __syncwarp();
    for (int e = lane; e < b.rows * n; e += 32) {
        const int i = e / n, j = e % n;
        t.V[(size_t)(b.r0 + i) * n + j] = (double)R[i * ld + j];
    }
}

}  // namespace

size_t jac_p_bytes(int n) { return (size_t)n * (n + 1) / 2 * sizeof(double); }
size_t jac_rot_bytes(int n) {
    const int m = n + (n & 1), half = m / 2;
    return jac_rot_head(n) + (size_t)jac_max_rounds(n) * half * sizeof(RotE<double>);
}
// Rows of V per apply block (one warp, one row per lane).
int jac_rows_per_block(int n, bool f32) {
    const size_t row = (size_t)(n | 1) * (f32 ? 4 : 8);
    const size_t r = (size_t)JAC_SMEM / row;
    return (int)(r < 32 ? (r < 1 ? 1 : r) : 32);
}

static void jac_attributes() {
    ensure_smem_attr(reinterpret_cast<const void*>(k_jac_sweep<double>), JAC_SMEM);
    ensure_smem_attr(reinterpret_cast<const void*>(k_jac_sweep<float>), JAC_SMEM);
    ensure_smem_attr(reinterpret_cast<const void*>(k_jac_apply<double>), JAC_SMEM);
    ensure_smem_attr(reinterpret_cast<const void*>(k_jac_apply<float>), JAC_SMEM);
}

void launch_jac_sweep(const JacTask* tasks, int ntask, int sweep, int maxs, bool f32, cudaStream_t st) {
    if (ntask <= 0) return;
    jac_attributes();
    count_launch();
    if (f32) k_jac_sweep<float><<<ntask, JAC_THREADS, JAC_SMEM, st>>>(tasks, sweep, maxs);
    else k_jac_sweep<double><<<ntask, JAC_THREADS, JAC_SMEM, st>>>(tasks, sweep, maxs);
}

// Shared memory of the cluster sweep for an n x n matrix (0: does not fit).
int jac_cluster_smem(int n) {
    const size_t np = (size_t)n * (n + 1) / 2;
    const size_t b = jac_head_bytes<double>(n) + (np + JC - 1) / JC * sizeof(double);
    return b <= (size_t)JAC_SMEM ? (int)b : 0;
}

void launch_jac_sweep_cluster(const JacTask* tasks, int ntask, int sweep, int maxs, int smem, cudaStream_t st) {
    if (ntask <= 0) return;
    ensure_smem_attr(reinterpret_cast<const void*>(k_jac_sweep_cl<double>), JAC_SMEM);
    count_launch();
    k_jac_sweep_cl<double><<<ntask * JC, JAC_THREADS, smem, st>>>(tasks, sweep, maxs);
}

void launch_jac_apply(const JacTask* tasks, const JacRows* rows, int nblocks, int smem, int sweep, bool f32,
                      cudaStream_t st) {
    if (nblocks <= 0) return;
    jac_attributes();
    count_launch();
    if (f32) k_jac_apply<float><<<nblocks, 32, smem, st>>>(tasks, rows, sweep);
    else k_jac_apply<double><<<nblocks, 32, smem, st>>>(tasks, rows, sweep);
}

}  // namespace mpspt
