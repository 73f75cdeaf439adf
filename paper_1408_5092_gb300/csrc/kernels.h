// Device kernels of the MPS-PT hot path and their task descriptors.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace mpspt {

// One K-contribution of a grouped block GEMM: C_tile += alpha * op(A) op(B).
// trans bit 0: A is stored k x m (use A^T); bit 1: B is stored n x k (use B^T).
struct GemmOp {
    const double* A;
    const double* B;
    int lda, ldb, k, trans;
    double alpha;
};

// One output tile (rows [r0, r0+TM) x cols [c0, c0+TN) of an m x n block C).
// With cmap set, element (i, j) of the block is stored at
//   C + cmap[2j] + i * cmap[2j+1]          (cmap_rows == 0, per-column map)
//   C + cmap[2i] + j * cmap[2i+1]          (cmap_rows == 1, per-row map)
// which scatters a panel GEMM straight into a block-sparse layout.
struct GemmTask {
    double* C;
    const int* cmap;
    int ldc, m, n;
    int r0, c0;
    int op0, op1;      // range of GemmOp
    int accumulate;    // 1: C += sum, 0: C = sum
    int cmap_rows;
    // split-K: the task sums the positions
    // [kb, ke) of the concatenated K-list of its ops and, with part set,
    // writes its tm x tn partial tile there (dense, row-major) instead of C;
    // a reduction task then adds the partials in order
    double* part;
    int kb, ke;
};
// Sum of the nparts partial tiles at part + q * tm * tn (q ascending) into
// the tile (r0, c0) of C, with the GemmTask addressing (cmap, accumulate).
struct SplitRed {
    const double* part;
    double* C;
    const int* cmap;
    int nparts, tm, tn;
    int ldc, m, n, r0, c0;
    int accumulate, cmap_rows;
};

constexpr int GEMM_TM = 64;
constexpr int GEMM_TN = 64;

// dst block (rows x cols, leading dim ldd) = sum_k coef_k * src_k (leading dim lds_k)
struct MixSrc {
    const double* src;
    int lds;
    int pad;
    double coef;
};
struct MixTask {
    double* dst;
    int rows, cols, ldd;
    int s0, s1;
    int pad;
};

// Jacobi diagonal of A_loc: out[l, r] += sum coef * L[l*(ldL+1)] * R[r*(ldR+1)]
struct DiagTerm {
    const double* L;
    const double* R;
    int ldL, ldR;
    double coef;
};
struct DiagTask {
    double* out;
    int rows, cols;
    int t0, t1;
};

// Symmetric eigenproblem of one dense n x n row-major block (in place).
struct EigTask {
    double* A;      // n*n, destroyed (diagonal holds eigenvalues on exit)
    double* V;      // n*n eigenvectors (columns); with vinit: initial basis, rotated in place
    double* w;      // n eigenvalues (unsorted)
    int n;
    int vinit;
};
// One matrix of the sweep-per-launch Jacobi (kernels_eig.cu).
struct JacTask {
    const double* A;   // n x n symmetric input, row-major (read by sweep 0 only)
    void* P;           // scratch: packed upper triangle, jac_p_bytes(n)
    void* rot;         // scratch: rotation lists of the current sweep, jac_rot_bytes(n)
    double* V;         // n x n eigenvectors (columns), row-major; with vinit: the start basis
    double* w;         // n eigenvalues (unsorted), or null
    double* prev;      // scratch: off-norm of the previous sweep
    int* done;         // 0 while sweeping; 1 converged; 2 stopped by the sweep cap
    int* nsw;          // scratch: sweeps performed (written when the matrix stops)
    int n, vinit;
    int pad0, pad1;
};
struct JacRows {       // rows [r0, r0 + rows) of task's V for one apply block
    int task, r0, rows, pad;
};

// Block copy with optional column selection and transpose:
//   trans 0: dst[i*ldd + j] = src[i*lds + col(j)]
//   trans 1: dst[i*ldd + j] = src[j*lds + col(i)]      col(x) = cols ? cols[x] : x
struct CopyTask {
    const double* src;
    double* dst;
    const int* cols;
    int rows, cols_n;   // shape of dst
    int lds, ldd;
    int trans;
    int pad;
};

// CG scalar block living in device memory.
struct CgState {
    double rz, rz_new, pAp, alpha, beta, rr, bb, tol2;
    int done, iters, not_spd, pad;
};

// Number of kernels launched by this library in this process.
long long launch_count();
void count_launch();
long long launch_count_thread();      // launches made by the calling host thread
void uncount_launches(long long n);   // launches that went into a captured graph (this thread's)
// Raises a kernel's dynamic shared-memory limit to `bytes` on the current
// device.  The attribute belongs to the device's context, so it is set once
// per (kernel, device); thread-safe.  A failure is not remembered: the
// launch that follows then fails and its error check reports it.
void ensure_smem_attr(const void* func, int bytes);

// Split-bfloat16 tcgen05 variant of the grouped GEMM (tiles 128 x 64; same
// task format); f16: split-float16 terms instead.  *err is set to 1 if a
// bounded mbarrier wait gave up.
int tc_tile_m();
int tc_tile_n();
void launch_gemm_tc(const GemmTask* tasks, int ntask, const GemmOp* ops, int* err, cudaStream_t st,
                    const int* skip = nullptr, bool f16 = false);
// Float32-arithmetic variant of the float64 grouped GEMM (float64 in/out).
void launch_gemm_f64in_f32(const GemmTask* tasks, int ntask, const GemmOp* ops, cudaStream_t st,
                           const int* skip = nullptr);

void launch_gemm_f64(const GemmTask* tasks, int ntask, const GemmOp* ops, cudaStream_t st,
                     const int* skip = nullptr);
// Grouped GEMM with output tile tm x tn (64x64, 32x64, 64x32, 16x128, 32x32),
// float64 or float32 arithmetic (f32) on float64 data.  Persistent: at most
// the resident CTAs are launched and each walks a stride of the task list.
bool gemm_tile_supported(int tm, int tn);
void launch_splitk_reduce(const SplitRed* tasks, int ntask, cudaStream_t st, const int* skip = nullptr);
void launch_gemm_tile(int tm, int tn, bool f32, const GemmTask* tasks, int ntask, const GemmOp* ops, cudaStream_t st,
                      const int* skip = nullptr);
// Skinny-tile (16 x 128) float64 variant for panels with few rows.
void launch_gemm_f64_skinny(const GemmTask* tasks, int ntask, const GemmOp* ops, cudaStream_t st,
                            const int* skip = nullptr);
void launch_gemm_f64in_f32_skinny(const GemmTask* tasks, int ntask, const GemmOp* ops, cudaStream_t st,
                                  const int* skip = nullptr);
void launch_mix(const MixTask* tasks, int ntask, const MixSrc* srcs, cudaStream_t st,
                const int* skip = nullptr);
void launch_diag(const DiagTask* tasks, int ntask, const DiagTerm* terms, cudaStream_t st);
void launch_eig(const EigTask* tasks, int ntask, cudaStream_t st);
size_t jac_p_bytes(int n);
size_t jac_rot_bytes(int n);
int jac_rows_per_block(int n, bool f32);
void launch_jac_sweep(const JacTask* tasks, int ntask, int sweep, int maxs, bool f32, cudaStream_t st);
// float64 sweep by clusters of 8 CTAs per matrix (distributed shared memory)
int jac_cluster_smem(int n);
void launch_jac_sweep_cluster(const JacTask* tasks, int ntask, int sweep, int maxs, int smem, cudaStream_t st);
void launch_jac_apply(const JacTask* tasks, const JacRows* rows, int nblocks, int smem, int sweep, bool f32,
                      cudaStream_t st);
void launch_ns_prep(const EigTask* tasks, int ntask, cudaStream_t st);
void launch_copy(const CopyTask* tasks, int ntask, cudaStream_t st);

// Vector kernels (n doubles).  Reductions are deterministic (fixed order).
void vec_zero(double* x, size_t n, cudaStream_t st);
void vec_scale_mask(double* y, const double* x, double a, size_t n, cudaStream_t st);  // y = a*x
void vec_axpy(double* y, const double* x, double a, size_t n, cudaStream_t st);       // y += a*x
// out[slot] = x.y  (partial sums in scratch, which needs >= 1024 doubles)
void vec_dot(const double* x, const double* y, size_t n, double* out, double* scratch,
             unsigned* counter, cudaStream_t st);
void f64_to_f32(float* y, const double* x, size_t n, cudaStream_t st);
void f32_to_f64(double* y, const float* x, size_t n, cudaStream_t st);

// Preconditioned CG building blocks on device scalars.
// r = b - Ax ; z = Minv r ; p = z ; rz = r.z ; rr = r.r ; bb = b.b
void cg_init(double* r, double* z, double* p, const double* b, const double* Ax,
             const double* minv, size_t n, CgState* S, double tol, double* scratch,
             unsigned* counter, cudaStream_t st);
// pAp = p.Ap ; alpha = rz / pAp ; x += alpha p ; r -= alpha Ap ; z = Minv r ;
// rz_new = r.z ; rr = r.r ; done if rr <= tol2 bb ; p = z + (rz_new/rz) p
void cg_step(double* x, double* r, double* z, double* p, const double* Ap, const double* minv,
             size_t n, CgState* S, double* scratch, unsigned* counter, cudaStream_t st);
void make_minv(double* minv, const double* diag, size_t n, cudaStream_t st);
// t = r / (theta - diag), denominators kept away from zero (Davidson correction)
void davidson_correction(double* t, const double* r, const double* diag, double theta, size_t n, cudaStream_t st);

// ---- learned preconditioner (kernels_mlp.cu)
struct BlockRef {      // one QN block of a two-site vector
    size_t off;
    int len;
    int pad;
};
constexpr int MLP_NF = 16;   // features per block
void mlp_gemm(int M, int N, int K, const float* A, int lda, bool ta, const float* B, int ldb, bool tb,
              float* C, int ldc, const float* bias, const float* mask, int epi, cudaStream_t st);
void mlp_gemm_bf16w(int M, int N, int K, const float* A, int lda, bool ta, const void* B, int ldb, bool tb,
                    float* C, int ldc, const float* bias, const float* mask, int epi, cudaStream_t st);
void mlp_colsum(int M, int N, const float* A, float* out, cudaStream_t st);
void mlp_mse(int B, int N, const float* Y, const float* T, float* dY, float* rowloss, cudaStream_t st);
void mlp_adam(int n, float* w, const float* g, float* m, float* v, void* wb, float lr, int step, cudaStream_t st);
void mlp_to_bf16(int n, const float* w, void* wb, cudaStream_t st);
void block_features(const BlockRef* blocks, int nb, const double* diag, const double* g, const double* xw,
                    const float* meta, float* feats, cudaStream_t st);
void block_combine(const BlockRef* blocks, int nb, const float* coef, const double* xw, const double* minv,
                   const double* bvec, double* x0, cudaStream_t st);
void block_fit(const BlockRef* blocks, int nb, const double* xw, const double* minv, const double* bvec,
               const double* x, double* out, cudaStream_t st);

}  // namespace mpspt
