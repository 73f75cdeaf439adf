// CUDA-core kernels of the MPS-PT hot path (sm_103a): grouped block GEMM
// (float64 / float32) driven by task lists, Jacobi diagonal, batched Jacobi
// eigensolver for the density-matrix blocks, block copies, and the CG vector
// kernels with deterministic (fixed-order) reductions.
#include "kernels.h"

#include <atomic>
#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <set>
#include <utility>

namespace mpspt {
namespace {

std::atomic<long long> g_launches{0};
thread_local long long t_launches = 0;   // this host thread's launches
inline void counted() {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    ++t_launches;
}

constexpr int TK = 16;
constexpr int NT = 256;

// float64 operand -> arithmetic type.  To float32 the rounding is done with
// integer operations: the float64 pipe of this GPU is narrow and the
// conversion instruction would bound the tile staging.  Magnitudes below
// the float32 normal range become signed zero.
__device__ __forceinline__ float d2f_rn(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7FF);
    const unsigned long long m = b & 0xFFFFFFFFFFFFFULL;
    if (e == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (m ? 0x400000u : 0u));
    const int fe = e - 1023 + 127;
    if (fe <= 0) return __uint_as_float(sign);
    if (fe >= 255) return __uint_as_float(sign | 0x7F800000u);
    const unsigned mant = (unsigned)(m >> 29);
    const unsigned rem = (unsigned)(m & 0x1FFFFFFFULL);
    unsigned f = sign | ((unsigned)fe << 23) | mant;
    if (rem > 0x10000000u || (rem == 0x10000000u && (mant & 1u))) f += 1u;
    return __uint_as_float(f);
}
template <class U>
__device__ __forceinline__ U conv(double v);
template <>
__device__ __forceinline__ double conv<double>(double v) { return v; }
template <>
__device__ __forceinline__ float conv<float>(double v) { return d2f_rn(v); }

// Grouped GEMM: one CTA per output tile, looping over the tile's K-list.
// 16x16 threads; thread (tx, ty) owns rows ty + 16 i (i < TM/16) and
// cols tx + 16 j (j < TN/16).  T: storage type, U: arithmetic type.
// Persistent: the grid is at most the resident CTAs of the GPU, and CTA b
// takes tasks b, b + gridDim.x, ... (the planner orders tasks longest first).
template <int TM, int TN, class T, class Task, class Op, class U = T>
__global__ void __launch_bounds__(NT) k_gemm(const Task* __restrict__ tasks, int ntask,
                                             const Op* __restrict__ ops,
                                             const int* __restrict__ skip) {
    if (skip && *skip) return;
    constexpr int RI = TM / 16, RJ = TN / 16;
    __shared__ U As[TK][TM + 1];
    __shared__ U Bs[TK][TN + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  for (int ti = blockIdx.x; ti < ntask; ti += gridDim.x) {
    const Task t = tasks[ti];
    U acc[RI][RJ];
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
        for (int j = 0; j < RJ; ++j) acc[i][j] = U(0);
    const int mrem = min(TM, t.m - t.r0);
    const int nrem = min(TN, t.n - t.c0);
    int kbase = 0;   // position of op o's first K index in the concatenated K-list
    for (int o = t.op0; o < t.op1; ++o) {
        const Op op = ops[o];
        const int kb = max(0, t.kb - kbase), ke = min(op.k, t.ke - kbase);
        kbase += op.k;
        if (kb >= ke) continue;
        const bool ta = op.trans & 1, tb = op.trans & 2;
        const U alpha = conv<U>(op.alpha);
        for (int k0 = kb; k0 < ke; k0 += TK) {
            const int krem = min(TK, ke - k0);
            for (int e = threadIdx.x; e < TM * TK; e += NT) {
                int i, kk;
                if (ta) { i = e % TM; kk = e / TM; }
                else { kk = e % TK; i = e / TK; }
                U v = U(0);
                if (i < mrem && kk < krem) {
                    const int row = t.r0 + i, kg = k0 + kk;
                    v = conv<U>(ta ? op.A[(size_t)kg * op.lda + row] : op.A[(size_t)row * op.lda + kg]) * alpha;
                }
                As[kk][i] = v;
            }
            for (int e = threadIdx.x; e < TN * TK; e += NT) {
                int j, kk;
                if (tb) { kk = e % TK; j = e / TK; }
                else { j = e % TN; kk = e / TN; }
                U v = U(0);
                if (j < nrem && kk < krem) {
                    const int col = t.c0 + j, kg = k0 + kk;
                    v = conv<U>(tb ? op.B[(size_t)col * op.ldb + kg] : op.B[(size_t)kg * op.ldb + col]);
                }
                Bs[kk][j] = v;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < TK; ++kk) {
                U a[RI], b[RJ];
#pragma unroll
                for (int i = 0; i < RI; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < RJ; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < RI; ++i)
#pragma unroll
                    for (int j = 0; j < RJ; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < RI; ++i) {
        const int r = ty + 16 * i;
        if (r >= mrem) continue;
#pragma unroll
        for (int j = 0; j < RJ; ++j) {
            const int c = tx + 16 * j;
            if (c >= nrem) continue;
            if (t.part) { t.part[r * TN + c] = (T)acc[i][j]; continue; }
            const int gr = t.r0 + r, gc = t.c0 + c;
            T* dst;
            if (t.cmap == nullptr) dst = t.C + (size_t)gr * t.ldc + gc;
            else if (t.cmap_rows) dst = t.C + t.cmap[2 * gr] + (size_t)gc * t.cmap[2 * gr + 1];
            else dst = t.C + t.cmap[2 * gc] + (size_t)gr * t.cmap[2 * gc + 1];
            *dst = t.accumulate ? *dst + (T)acc[i][j] : (T)acc[i][j];
        }
    }
  }
}

// Split-K reduction: partial tiles summed in ascending order (deterministic).
__global__ void k_splitk_reduce(const SplitRed* __restrict__ tasks, const int* __restrict__ skip) {
    if (skip && *skip) return;
    const SplitRed t = tasks[blockIdx.x];
    const int mrem = min(t.tm, t.m - t.r0), nrem = min(t.tn, t.n - t.c0);
    const size_t tile = (size_t)t.tm * t.tn;
    for (int e = threadIdx.x; e < mrem * nrem; e += blockDim.x) {
        const int r = e / nrem, c = e % nrem;
        double v = 0.0;
        for (int q = 0; q < t.nparts; ++q) v += t.part[q * tile + (size_t)r * t.tn + c];
        const int gr = t.r0 + r, gc = t.c0 + c;
        double* dst;
        if (t.cmap == nullptr) dst = t.C + (size_t)gr * t.ldc + gc;
        else if (t.cmap_rows) dst = t.C + t.cmap[2 * gr] + (size_t)gc * t.cmap[2 * gr + 1];
        else dst = t.C + t.cmap[2 * gc] + (size_t)gr * t.cmap[2 * gc + 1];
        *dst = t.accumulate ? *dst + v : v;
    }
}

// dst = sum coef * src over the task's source list (memory-bound).
__global__ void k_mix(const MixTask* __restrict__ tasks, const MixSrc* __restrict__ srcs,
                      const int* __restrict__ skip) {
    if (skip && *skip) return;
    const MixTask t = tasks[blockIdx.x];
    const int n = t.rows * t.cols;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int i = e / t.cols, j = e % t.cols;
        double s = 0.0;
        for (int q = t.s0; q < t.s1; ++q) {
            const MixSrc m = srcs[q];
            s += m.coef * m.src[(size_t)i * m.lds + j];
        }
        t.dst[(size_t)i * t.ldd + j] = s;
    }
}

__global__ void k_diag(const DiagTask* __restrict__ tasks, const DiagTerm* __restrict__ terms) {
    const DiagTask t = tasks[blockIdx.x];
    const int n = t.rows * t.cols;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int l = e / t.cols, r = e % t.cols;
        double s = 0.0;
        for (int k = t.t0; k < t.t1; ++k) {
            const DiagTerm d = terms[k];
            s += d.coef * d.L[(size_t)l * (d.ldL + 1)] * d.R[(size_t)r * (d.ldR + 1)];
        }
        t.out[e] = s;
    }
}

__global__ void k_copy(const CopyTask* __restrict__ tasks) {
    const CopyTask t = tasks[blockIdx.x];
    const int n = t.rows * t.cols_n;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int i = e / t.cols_n, j = e % t.cols_n;
        double v;
        if (t.trans) v = t.src[(size_t)j * t.lds + (t.cols ? t.cols[i] : i)];
        else v = t.src[(size_t)i * t.lds + (t.cols ? t.cols[j] : j)];
        t.dst[(size_t)i * t.ldd + j] = v;
    }
}

// Cyclic two-sided Jacobi with the round-robin parallel ordering.  In each
// of the m-1 rounds of a sweep the m/2 disjoint pairs (p_k, q_k) get their
// rotation R_k; the whole matrix is then updated in one pass, block by
// block: the 2x2 block of pairs (k, l) becomes R_k^T A_kl R_l (blocks are
// independent, so the update is in place), and the eigenvector columns of
// pair l are rotated by R_l.  Inside the kernel the eigenvectors are held
// transposed (row j = eigenvector j), so that a column rotation touches two
// contiguous rows.  A is kept in shared memory whenever it fits, V too when
// both fit; the rest stays in global memory (L2-resident).  A pair is
// skipped when its off-diagonal element is negligible against its diagonal
// (threshold Jacobi).  With vinit the kernel starts from the caller's
// orthonormal basis V and accumulates the rotations into it (A is then
// taken to be V0^T A_orig V0 already).
constexpr int EIG_MAXN = 2048;
constexpr int EIG_SMEM_BYTES = 200704;   // dynamic shared memory per CTA

__device__ __forceinline__ void rr_pair(int k, int r, int m, int& pa, int& pb) {
    pa = (k == 0) ? 0 : ((k - 1 + r) % (m - 1)) + 1;
    pb = ((m - 1 - k - 1 + r) % (m - 1)) + 1;
}

// In-place transpose of an n x n matrix in global memory (one CTA).
template <class T>
__device__ void transpose_inplace(T* M, int n) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        if (i < j) {
            const T x = M[(size_t)i * n + j];
            M[(size_t)i * n + j] = M[(size_t)j * n + i];
            M[(size_t)j * n + i] = x;
        }
    }
}

template <class T, class Task>
__global__ void __launch_bounds__(512) k_eig(const Task* __restrict__ tasks) {
    extern __shared__ __align__(16) unsigned char esm_raw[];
    T* esm = reinterpret_cast<T*>(esm_raw);
    const Task t = tasks[blockIdx.x];
    const int n = t.n;
    constexpr T STOP = sizeof(T) == 8 ? T(1e-30) : T(1e-11);     // off^2 <= STOP * all^2
    constexpr T SKIP = sizeof(T) == 8 ? T(1e-18) : T(1e-9);      // negligible a_pq
    constexpr int MAXSWEEP = sizeof(T) == 8 ? 40 : 12;
    const size_t nn = (size_t)n * n;
    const bool a_sm = nn * sizeof(T) <= (size_t)EIG_SMEM_BYTES;
    const bool v_sm = 2 * nn * sizeof(T) <= (size_t)EIG_SMEM_BYTES;
    T* A = a_sm ? esm : t.A;
    T* W = v_sm ? esm + nn : t.V;      // W[j*n + i] = V[i*n + j]
    __shared__ int Pp[EIG_MAXN / 2], Qq[EIG_MAXN / 2];
    __shared__ T Cc[EIG_MAXN / 2], Ss[EIG_MAXN / 2];
    __shared__ double red[2][32];
    __shared__ int stop;
    for (int e = threadIdx.x; e < (int)nn; e += blockDim.x) {
        if (a_sm) A[e] = t.A[e];
        if (!t.vinit) W[e] = (e / n == e % n) ? T(1) : T(0);
        else if (v_sm) W[(size_t)(e % n) * n + e / n] = t.V[e];
    }
    if (t.vinit && !v_sm) {
        __syncthreads();
        transpose_inplace(W, n);
    }
    __syncthreads();
    if (n > 1) {
        const int m = n + (n & 1);
        const int half = m / 2;
        double prev_off = 1e300;   // thread 0 only
        for (int sweep = 0; sweep < MAXSWEEP; ++sweep) {
            double off = 0.0, all = 0.0;
            for (int e = threadIdx.x; e < (int)nn; e += blockDim.x) {
                const double v = (double)A[e];
                all += v * v;
                if (e / n != e % n) off += v * v;
            }
            for (int o = 16; o > 0; o >>= 1) {
                off += __shfl_xor_sync(0xffffffffu, off, o);
                all += __shfl_xor_sync(0xffffffffu, all, o);
            }
            if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = off; red[1][threadIdx.x >> 5] = all; }
            __syncthreads();
            if (threadIdx.x == 0) {
                double so = 0.0, sa = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { so += red[0][w]; sa += red[1][w]; }
                // converged, or stalled at the rounding floor (a sweep that no
                // longer shrinks a small off-diagonal norm)
                stop = (so <= (double)STOP * sa) || sa == 0.0 || (so <= 1e-8 * sa && so > 0.81 * prev_off);
                prev_off = so;
            }
            __syncthreads();
            if (stop) break;
            for (int r = 0; r < m - 1; ++r) {
                for (int k = threadIdx.x; k < half; k += blockDim.x) {
                    int pa, pb;
                    rr_pair(k, r, m, pa, pb);
                    int p = min(pa, pb), q = max(pa, pb);
                    T c = T(1), s = T(0);
                    if (q < n) {
                        const T apq = A[(size_t)p * n + q];
                        const T app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                        if (fabs(apq) > SKIP * sqrt(fabs(app * aqq)) && apq != T(0)) {
                            const T th = (aqq - app) / (T(2) * apq);
                            const T tt = (th >= T(0) ? T(1) : T(-1)) / (fabs(th) + sqrt(th * th + T(1)));
                            c = T(1) / sqrt(tt * tt + T(1));
                            s = tt * c;
                        }
                    } else {
                        q = -1;  // dummy player: no rotation, single index p
                    }
                    Pp[k] = p; Qq[k] = q; Cc[k] = c; Ss[k] = s;
                }
                __syncthreads();
                // A <- J^T A J block by block
                for (int e = threadIdx.x; e < half * half; e += blockDim.x) {
                    const int k = e / half, l = e % half;
                    const int p = Pp[k], q = Qq[k], u = Pp[l], v = Qq[l];
                    const T ck = Cc[k], sk = Ss[k], cl = Cc[l], sl = Ss[l];
                    if (sk == T(0) && sl == T(0)) continue;
                    // rows p (and q), columns u (and v); rotation: new_p = c*old_p - s*old_q,
                    // new_q = s*old_p + c*old_q, applied on both sides
                    const bool hq = q >= 0, hv = v >= 0;
                    T a_pu = A[(size_t)p * n + u];
                    T a_pv = hv ? A[(size_t)p * n + v] : T(0);
                    T a_qu = hq ? A[(size_t)q * n + u] : T(0);
                    T a_qv = (hq && hv) ? A[(size_t)q * n + v] : T(0);
                    const T r_pu = ck * a_pu - sk * a_qu, r_qu = sk * a_pu + ck * a_qu;
                    const T r_pv = ck * a_pv - sk * a_qv, r_qv = sk * a_pv + ck * a_qv;
                    A[(size_t)p * n + u] = cl * r_pu - sl * r_pv;
                    if (hv) A[(size_t)p * n + v] = sl * r_pu + cl * r_pv;
                    if (hq) A[(size_t)q * n + u] = cl * r_qu - sl * r_qv;
                    if (hq && hv) A[(size_t)q * n + v] = sl * r_qu + cl * r_qv;
                }
                // eigenvector rows u, v of W (columns of V) <- rotation R_l
                for (int e = threadIdx.x; e < n * half; e += blockDim.x) {
                    const int l = e / n, i = e % n;
                    const int u = Pp[l], v = Qq[l];
                    const T cl = Cc[l], sl = Ss[l];
                    if (sl == T(0) || v < 0) continue;
                    const T wu = W[(size_t)u * n + i], wv = W[(size_t)v * n + i];
                    W[(size_t)u * n + i] = cl * wu - sl * wv;
                    W[(size_t)v * n + i] = sl * wu + cl * wv;
                }
                __syncthreads();
            }
        }
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) t.w[i] = A[(size_t)i * n + i];
    if (v_sm) {
        for (int e = threadIdx.x; e < (int)nn; e += blockDim.x) t.V[e] = W[(size_t)(e % n) * n + e / n];
    } else {
        transpose_inplace(W, n);
    }
    if (a_sm)
        for (int e = threadIdx.x; e < (int)nn; e += blockDim.x) t.A[e] = A[e];
}

// ----------------------------------------------------------------- vectors
constexpr int RB = 256;        // threads per reduction block
constexpr int RG_MAX = 1024;   // max reduction blocks

inline int red_grid(size_t n) {
    size_t g = (n + (size_t)RB * 4 - 1) / ((size_t)RB * 4);
    if (g < 1) g = 1;
    if (g > RG_MAX) g = RG_MAX;
    return (int)g;
}

template <int NV>
__device__ void block_sum(double (&v)[NV], double (*sh)[RB / 32]) {
#pragma unroll
    for (int q = 0; q < NV; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) sh[q][threadIdx.x >> 5] = v[q];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double s = 0.0;
            for (int w = 0; w < RB / 32; ++w) s += sh[q][w];
            v[q] = s;
        }
}

// Last-block-done pattern: every block stores its partial sums, the last one
// to finish adds them in block order (deterministic) and runs `fin`.
template <int NV>
__device__ bool last_block(double (&v)[NV], double* scratch, unsigned* counter, double (&tot)[NV]) {
    __shared__ bool is_last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) scratch[q * RG_MAX + blockIdx.x] = v[q];
        __threadfence();
        unsigned prev = atomicAdd(counter, 1u);
        is_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    if (threadIdx.x == 0) {
        __threadfence();
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double s = 0.0;
            for (unsigned b = 0; b < gridDim.x; ++b) s += ((volatile double*)scratch)[q * RG_MAX + b];
            tot[q] = s;
        }
        *counter = 0;
    }
    return threadIdx.x == 0;
}

__global__ void k_dot(const double* __restrict__ x, const double* __restrict__ y, size_t n,
                      double* out, double* scratch, unsigned* counter) {
    __shared__ double sh[1][RB / 32];
    double v[1] = {0.0};
    for (size_t i = blockIdx.x * (size_t)RB + threadIdx.x; i < n; i += (size_t)gridDim.x * RB)
        v[0] += x[i] * y[i];
    block_sum<1>(v, sh);
    double tot[1];
    if (last_block<1>(v, scratch, counter, tot)) *out = tot[0];
}

__global__ void k_cg_init(double* r, double* z, double* p, const double* __restrict__ b,
                          const double* __restrict__ Ax, const double* __restrict__ minv, size_t n,
                          CgState* S, double tol, double* scratch, unsigned* counter) {
    __shared__ double sh[3][RB / 32];
    double v[3] = {0.0, 0.0, 0.0};
    for (size_t i = blockIdx.x * (size_t)RB + threadIdx.x; i < n; i += (size_t)gridDim.x * RB) {
        const double ri = b[i] - Ax[i];
        const double zi = minv[i] * ri;
        r[i] = ri;
        z[i] = zi;
        p[i] = zi;
        v[0] += ri * zi;
        v[1] += ri * ri;
        v[2] += b[i] * b[i];
    }
    block_sum<3>(v, sh);
    double tot[3];
    if (last_block<3>(v, scratch, counter, tot)) {
        S->rz = tot[0];
        S->rr = tot[1];
        S->bb = tot[2];
        S->tol2 = tol * tol;
        S->iters = 0;
        S->not_spd = 0;
        S->done = (tot[1] <= tol * tol * tot[2]) || tot[2] == 0.0;
    }
}

__global__ void k_cg_pap(const double* __restrict__ p, const double* __restrict__ Ap, size_t n,
                         CgState* S, double* scratch, unsigned* counter) {
    if (S->done) return;
    __shared__ double sh[1][RB / 32];
    double v[1] = {0.0};
    for (size_t i = blockIdx.x * (size_t)RB + threadIdx.x; i < n; i += (size_t)gridDim.x * RB)
        v[0] += p[i] * Ap[i];
    block_sum<1>(v, sh);
    double tot[1];
    if (last_block<1>(v, scratch, counter, tot)) {
        S->pAp = tot[0];
        if (!(tot[0] > 0.0)) { S->not_spd = 1; S->done = 1; }
        else S->alpha = S->rz / tot[0];
    }
}

__global__ void k_cg_update(double* x, double* r, double* z, const double* __restrict__ p,
                            const double* __restrict__ Ap, const double* __restrict__ minv,
                            size_t n, CgState* S, double* scratch, unsigned* counter) {
    if (S->done) return;
    __shared__ double sh[2][RB / 32];
    const double a = S->alpha;
    double v[2] = {0.0, 0.0};
    for (size_t i = blockIdx.x * (size_t)RB + threadIdx.x; i < n; i += (size_t)gridDim.x * RB) {
        x[i] += a * p[i];
        const double ri = r[i] - a * Ap[i];
        const double zi = minv[i] * ri;
        r[i] = ri;
        z[i] = zi;
        v[0] += ri * zi;
        v[1] += ri * ri;
    }
    block_sum<2>(v, sh);
    double tot[2];
    if (last_block<2>(v, scratch, counter, tot)) {
        S->rz_new = tot[0];
        S->rr = tot[1];
        S->beta = tot[0] / S->rz;
        S->rz = tot[0];
        S->iters += 1;
        if (tot[1] <= S->tol2 * S->bb) S->done = 2;
    }
}

__global__ void k_cg_dir(double* p, const double* __restrict__ z, size_t n, const CgState* S) {
    if (S->done) return;
    const double be = S->beta;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p[i] = z[i] + be * p[i];
}

// G <- 1.5 I - 0.5 G for each task's n x n block (Newton-Schulz step)
__global__ void k_ns_prep(const EigTask* __restrict__ tasks) {
    const EigTask t = tasks[blockIdx.x];
    const int n = t.n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x)
        t.A[e] = (e / n == e % n ? 1.5 : 0.0) - 0.5 * t.A[e];
}

__global__ void k_axpy(double* y, const double* __restrict__ x, double a, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}
__global__ void k_scale(double* y, const double* __restrict__ x, double a, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = a * x[i];
}
__global__ void k_zero(double* y, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = 0.0;
}
__global__ void k_minv(double* y, const double* __restrict__ d, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = d[i] > 0.0 ? 1.0 / d[i] : 0.0;
}
// Davidson correction t = r / (theta - d), the denominator kept at least
// 1e-8 max(1, |theta|) away from zero (its sign kept)
__global__ void k_dav_corr(double* t, const double* __restrict__ r, const double* __restrict__ d, double theta,
                           size_t n) {
    const double eps = 1e-8 * fmax(1.0, fabs(theta));
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double den = theta - d[i];
        if (fabs(den) < eps) den = den < 0.0 ? -eps : eps;
        t[i] = r[i] / den;
    }
}
__global__ void k_d2f(float* y, const double* __restrict__ x, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}
__global__ void k_f2d(double* y, const float* __restrict__ x, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = (double)x[i];
}

inline int ew_grid(size_t n) {
    size_t g = (n + 255) / 256;
    if (g < 1) g = 1;
    if (g > 152 * 8) g = 152 * 8;
    return (int)g;
}

}  // namespace

long long launch_count() { return g_launches.load(); }
void count_launch() { counted(); }
long long launch_count_thread() { return t_launches; }
void uncount_launches(long long n) {
    g_launches.fetch_sub(n);
    t_launches -= n;
}

void ensure_smem_attr(const void* func, int bytes) {
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;
    thread_local std::set<std::pair<const void*, int>> seen;   // lock-free fast path per thread
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    if (seen.count({func, dev})) return;
    std::lock_guard<std::mutex> lk(mu);
    if (!done.count({func, dev})) {
        if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) return;
        done.insert({func, dev});
    }
    seen.insert({func, dev});
}

namespace {
// Resident CTAs of a kernel on the current device (occupancy x SMs), cached
// per (kernel, device).
int resident_ctas(const void* func, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> cache;
    thread_local std::map<std::pair<const void*, int>, int> mine;   // lock-free fast path per thread
    int dev = 0;
    cudaGetDevice(&dev);
    auto f = mine.find({func, dev});
    if (f != mine.end()) return f->second;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find({func, dev});
    if (it != cache.end()) return mine[{func, dev}] = it->second;
    int nb = 1, sms = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, func, threads, smem) != cudaSuccess || nb < 1) nb = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    cudaGetLastError();
    return mine[{func, dev}] = cache[{func, dev}] = nb * sms;
}

template <int TM, int TN, class U>
void launch_tile(const GemmTask* tasks, int ntask, const GemmOp* ops, cudaStream_t st, const int* skip) {
    auto* f = k_gemm<TM, TN, double, GemmTask, GemmOp, U>;
    const int grid = std::min(ntask, resident_ctas(reinterpret_cast<const void*>(f), NT, 0));
    counted();
    f<<<grid, NT, 0, st>>>(tasks, ntask, ops, skip);
}
}  // namespace

bool gemm_tile_supported(int tm, int tn) {
    return (tm == 64 && tn == 64) || (tm == 32 && tn == 64) || (tm == 64 && tn == 32) || (tm == 16 && tn == 128) ||
           (tm == 32 && tn == 32);
}

void launch_splitk_reduce(const SplitRed* tasks, int ntask, cudaStream_t st, const int* skip) {
    if (ntask > 0) { counted(); k_splitk_reduce<<<ntask, 256, 0, st>>>(tasks, skip); }
}

void launch_gemm_tile(int tm, int tn, bool f32, const GemmTask* tasks, int ntask, const GemmOp* ops, cudaStream_t st,
                      const int* skip) {
    if (ntask <= 0) return;
#define MPSPT_TILE(A, B)                                                          \
    if (tm == A && tn == B) {                                                     \
        if (f32) launch_tile<A, B, float>(tasks, ntask, ops, st, skip);           \
        else launch_tile<A, B, double>(tasks, ntask, ops, st, skip);              \
        return;                                                                   \
    }
    MPSPT_TILE(64, 64)
    MPSPT_TILE(32, 64)
    MPSPT_TILE(64, 32)
    MPSPT_TILE(16, 128)
    MPSPT_TILE(32, 32)
#undef MPSPT_TILE
    launch_tile<64, 64, double>(tasks, 0, ops, st, skip);   // unreachable for planned tiles
}

void launch_gemm_f64in_f32(const GemmTask* tasks, int ntask, const GemmOp* ops, cudaStream_t st,
                           const int* skip) {
    launch_gemm_tile(64, 64, true, tasks, ntask, ops, st, skip);
}
void launch_gemm_f64_skinny(const GemmTask* tasks, int ntask, const GemmOp* ops, cudaStream_t st,
                            const int* skip) {
    launch_gemm_tile(16, 128, false, tasks, ntask, ops, st, skip);
}
void launch_gemm_f64in_f32_skinny(const GemmTask* tasks, int ntask, const GemmOp* ops, cudaStream_t st,
                                  const int* skip) {
    launch_gemm_tile(16, 128, true, tasks, ntask, ops, st, skip);
}
void launch_mix(const MixTask* tasks, int ntask, const MixSrc* srcs, cudaStream_t st, const int* skip) {
    if (ntask > 0) { counted(); k_mix<<<ntask, 128, 0, st>>>(tasks, srcs, skip); }
}

void launch_gemm_f64(const GemmTask* tasks, int ntask, const GemmOp* ops, cudaStream_t st,
                     const int* skip) {
    launch_gemm_tile(64, 64, false, tasks, ntask, ops, st, skip);
}
void launch_diag(const DiagTask* tasks, int ntask, const DiagTerm* terms, cudaStream_t st) {
    if (ntask > 0) { counted(); k_diag<<<ntask, 256, 0, st>>>(tasks, terms); }
}
void launch_eig(const EigTask* tasks, int ntask, cudaStream_t st) {
    if (ntask <= 0) return;
    const int smem = EIG_SMEM_BYTES;
    ensure_smem_attr(reinterpret_cast<const void*>(k_eig<double, EigTask>), smem);
    counted();
    k_eig<double, EigTask><<<ntask, 512, smem, st>>>(tasks);
}

void launch_copy(const CopyTask* tasks, int ntask, cudaStream_t st) {
    if (ntask > 0) { counted(); k_copy<<<ntask, 256, 0, st>>>(tasks); }
}
void launch_ns_prep(const EigTask* tasks, int ntask, cudaStream_t st) {
    if (ntask > 0) { counted(); k_ns_prep<<<ntask, 256, 0, st>>>(tasks); }
}

void vec_zero(double* x, size_t n, cudaStream_t st) {
    if (n) { counted(); k_zero<<<ew_grid(n), 256, 0, st>>>(x, n); }
}
void vec_scale_mask(double* y, const double* x, double a, size_t n, cudaStream_t st) {
    if (n) { counted(); k_scale<<<ew_grid(n), 256, 0, st>>>(y, x, a, n); }
}
void vec_axpy(double* y, const double* x, double a, size_t n, cudaStream_t st) {
    if (n) { counted(); k_axpy<<<ew_grid(n), 256, 0, st>>>(y, x, a, n); }
}
void vec_dot(const double* x, const double* y, size_t n, double* out, double* scratch,
             unsigned* counter, cudaStream_t st) {
    counted(); k_dot<<<red_grid(n), RB, 0, st>>>(x, y, n, out, scratch, counter);
}
void f64_to_f32(float* y, const double* x, size_t n, cudaStream_t st) {
    if (n) { counted(); k_d2f<<<ew_grid(n), 256, 0, st>>>(y, x, n); }
}
void f32_to_f64(double* y, const float* x, size_t n, cudaStream_t st) {
    if (n) { counted(); k_f2d<<<ew_grid(n), 256, 0, st>>>(y, x, n); }
}
void davidson_correction(double* t, const double* r, const double* diag, double theta, size_t n, cudaStream_t st) {
    if (n) { counted(); k_dav_corr<<<ew_grid(n), 256, 0, st>>>(t, r, diag, theta, n); }
}
void make_minv(double* minv, const double* diag, size_t n, cudaStream_t st) {
    if (n) { counted(); k_minv<<<ew_grid(n), 256, 0, st>>>(minv, diag, n); }
}
void cg_init(double* r, double* z, double* p, const double* b, const double* Ax,
             const double* minv, size_t n, CgState* S, double tol, double* scratch,
             unsigned* counter, cudaStream_t st) {
    counted(); k_cg_init<<<red_grid(n), RB, 0, st>>>(r, z, p, b, Ax, minv, n, S, tol, scratch, counter);
}
void cg_step(double* x, double* r, double* z, double* p, const double* Ap, const double* minv,
             size_t n, CgState* S, double* scratch, unsigned* counter, cudaStream_t st) {
    counted(); k_cg_pap<<<red_grid(n), RB, 0, st>>>(p, Ap, n, S, scratch, counter);
    counted(); k_cg_update<<<red_grid(n), RB, 0, st>>>(x, r, z, p, Ap, minv, n, S, scratch, counter);
    counted(); k_cg_dir<<<ew_grid(n), 256, 0, st>>>(p, z, n, S);
}

}  // namespace mpspt
