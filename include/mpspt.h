/*
 * mpspt.h — C ABI of the GB300 MPS-PT library.
 *
 * MPS-PT (Sharma & Chan, "A flexible multi-reference perturbation theory by
 * minimizing the Hylleraas functional with matrix product states") obtains
 * the second-order energy E2 as the minimum of the Hylleraas functional
 *     H[Psi1] = <Psi1|H0 - E0|Psi1> + 2 <Psi1|Q V|Psi0>            (Eq. 1)
 * over matrix product states Psi1 (Eq. 3) of bond dimension M, by a two-site
 * DMRG-like sweep whose local step solves the linear equation of Fig. 1C by
 * conjugate gradient; E3 follows from Psi1 by Wigner's 2n+1 rule (Eq. 5).
 *
 * Conventions shared by every call:
 *  - spatial orbitals p = 0..k-1, k = k_act + k_virt; active orbitals first,
 *    then virtual orbitals; no core orbitals;
 *  - one MPS site per spatial orbital, local basis |0>,|a>,|b>,|ab> (codes
 *    0..3), many-body states are creators in ascending spin-orbital order
 *    (p0a, p0b, p1a, ...) applied to the vacuum;
 *  - quantum numbers (N, 2Sz); a bond index carries the QN of the part of the
 *    chain to its left;
 *  - Psi1 lies in the space X of determinants with one or two electrons in
 *    virtual orbitals, so Q acts as the identity on it and -QV Psi0 = -P_X H Psi0.
 *
 * Error behaviour: no call throws or aborts across the ABI.  On error the
 * output arguments are left untouched and the status says why;
 * mpspt_status_string() gives a message.  All device work is ordered on the
 * stream given in mpspt_options (0 = the legacy default stream); every call
 * returns only after its host-visible results are final.
 * Device memory: allocated stream-ordered from the device's default memory
 * pool; the library raises that pool's release threshold so freed memory
 * stays cached in this process between calls (cudaMemPoolTrimTo returns it).
 * Ownership: input arrays are copied, the caller keeps them.  Handles
 * (mpspt_ctx, mpspt_mps) are owned by the caller and released with
 * mpspt_destroy / mpspt_mps_free.
 */
#ifndef MPSPT_H
#define MPSPT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpspt_ctx mpspt_ctx;
typedef struct mpspt_mps mpspt_mps;

typedef enum {
    MPSPT_OK = 0,
    MPSPT_ERR_INVALID = -1,        /* bad argument or NaN/Inf in an input     */
    MPSPT_ERR_OOM = -2,            /* device memory exhausted / arena cap hit */
    MPSPT_ERR_NOT_SPD = -3,        /* CG met p^T A p <= 0 (H0 - E0 not > 0)   */
    MPSPT_ERR_NOT_CONVERGED = -4,  /* an iteration cap was reached: local CG  */
                                   /* (cg_max_iter), float64 refinement (12   */
                                   /* rounds) or truncation eigensolver       */
    MPSPT_ERR_TIMEOUT = -5,        /* a bounded device wait gave up           */
    MPSPT_ERR_CUDA = -6,           /* a CUDA runtime call failed              */
    MPSPT_ERR_STATE = -7           /* call out of order (e.g. no integrals)   */
} mpspt_status;

/* Zeroth-order Hamiltonian.  DYALL: H_act + sum_a eps_a n_a (NEVPT-type,
 * E0 = <Psi0|H_act|Psi0>, E1 = 0).  FOCK: sum_tu f_tu E_tu + sum_a eps_a n_a
 * (CASPT2-type one-body Fock operator between many-body projectors; E0 =
 * sum f_tu gamma_tu).  eps_a are the eigenvalues of the generalised Fock
 * matrix in the virtual block (semicanonical virtuals). */
typedef enum { MPSPT_H0_FOCK = 0, MPSPT_H0_DYALL = 1 } mpspt_h0;

/* Arithmetic of the local solver.  FP64: every contraction in float64.
 * FP32: contractions in float32, CG vectors float64, final energy float64.
 * MIXED_BF16: sigma contractions as three-term split-bfloat16 products on
 * the tensor cores with float32 accumulation inside a float64-refined CG;
 * the residual and the Hylleraas value are evaluated in float64.
 * MIXED_FP16: the same with float16 hi/lo terms (11-bit significands, so
 * the three products carry ~22 bits against ~16 for bfloat16; the exponent
 * range is narrow, so each inner solve runs on the residual scaled to unit
 * norm, and entries below 2^-24 of that scale are lost). */
typedef enum { MPSPT_FP64 = 0, MPSPT_FP32 = 1, MPSPT_MIXED_BF16 = 2, MPSPT_MIXED_FP16 = 3 } mpspt_prec;

typedef struct {
    int device;                 /* CUDA device ordinal                          */
    void* stream;               /* cudaStream_t, 0 = default stream             */
    mpspt_prec prec;
    int max_sweeps;             /* full (left->right->left) sweeps, <= 64       */
    double e_tol;               /* |E2(sweep n) - E2(sweep n-1)| stop criterion */
    double cg_tol;              /* relative residual |r| <= cg_tol |g|          */
    int cg_max_iter;            /* per local solve                              */
    unsigned long long seed;    /* initial Psi1 (counter-based, see below)      */
    int use_learned;            /* learned block preconditioner (0 = Jacobi);   */
                                /* full-space calls only: partitioned calls     */
                                /* keep the Jacobi start on every lane          */
    int verbose;                /* 1: one line per sweep on stderr              */
    int eig_fp64_only;          /* density-matrix eigensolver: 0 (default) =    */
                                /* float32 Jacobi start, float64 Newton-Schulz  */
                                /* re-orthonormalisation and float64 Jacobi     */
                                /* polish; 1 = float64 Jacobi from identity     */
                                /* (see mpspt_eigh_batched_ex)                  */
    double keep_rel;            /* truncation keeps density-matrix eigenvectors */
                                /* with eigenvalue > keep_rel tr(rho), at most  */
                                /* M of them; 0 = 1e-10                          */
    int autotune;               /* 1: the first grouped GEMM of each block-shape */
                                /* class times the candidate tile shapes and    */
                                /* keeps the fastest (see autotune_cache)       */
    const char* autotune_cache; /* file of tuned tile shapes: read by            */
                                /* mpspt_create, written by mpspt_destroy; NULL */
                                /* = tune in memory only                         */
    int cuda_graphs;            /* 1: each local CG solve captures a chunk of 8  */
                                /* iterations (sigma + vector updates) in a CUDA */
                                /* graph and replays it until converged; the    */
                                /* sigma time then includes the chunk's vector  */
                                /* kernels.  Needs a created stream (the legacy */
                                /* default stream cannot be captured: there the */
                                /* option has no effect); partitions always run */
                                /* on created streams                            */
} mpspt_options;

typedef struct {
    int n_sweeps;
    double e2_per_sweep[64];
    double max_discarded_weight; /* over the last sweep                          */
    long long cg_iters;          /* total CG iterations (all local solves)       */
    long long sigma_calls;       /* applications of A_loc (any precision)        */
    double sigma_flops;          /* algorithmic flops of those applications      */
    double sigma_ms;             /* device time inside them (CUDA events)        */
    double wall_ms;              /* wall time of the minimisation                */
    int max_bond_dim;
    double sweep_ms[64];         /* device time at the end of each sweep         */
    long long kernel_launches;   /* device kernels launched by the minimisation  */
    long long sigma64_calls;     /* float64 applications used for residual       */
    double sigma64_flops;        /*   refinement and the Hylleraas value when    */
    double sigma64_ms;           /*   prec != FP64 (sigma_* then count the       */
                                 /*   inner low-precision applications)          */
    long long learned_used;      /* local solves started from the learned guess  */
    long long learned_rejected;  /* ... where the warm start had lower residual  */
    int converged;               /* 1: the last sweep changed E2 by < e_tol;     */
                                 /* 0: max_sweeps ended the run first            */
    double max_discarded_per_sweep[64]; /* discarded weight, max over the bonds  */
                                 /* of each sweep                                */
    long long sigma_calls_cum[64]; /* applications of A_loc (all precisions)     */
                                 /* done by the end of each sweep                */
    double host_wait_ms;         /* host time blocked waiting for the device     */
                                 /* (partitioned: summed over the partitions)    */
    double e3_ms;                /* mpspt_third_order_partitioned: wall time of  */
    long long e3_transfers;      /*   the E3 transfers, their number, the host   */
    double e3_wait_ms;           /*   time the lanes spent waiting for the device */
    double e3_flops;             /*   (summed over lanes), the float64 GEMM flops */
    double e3_plan_bytes;        /*   and task-list bytes of the transfers, and  */
    double e3_setup_ms;          /*   the wall time of building the operators    */
                                 /*   (the full H MPO once per context); 0 from  */
                                 /*   every other call                           */
} mpspt_report;

/* Fills *opt with defaults: device 0, default stream, FP64, 30 sweeps,
 * e_tol 1e-10, cg_tol 1e-10, 1000 CG iterations, seed 1408, keep_rel 1e-10,
 * no autotuning. */
void mpspt_default_options(mpspt_options* opt);

/* Creates a context bound to opt->device.  *ctx owned by the caller. */
mpspt_status mpspt_create(mpspt_ctx** ctx, const mpspt_options* opt);
void mpspt_destroy(mpspt_ctx* ctx);   /* frees everything the context owns */

/* Integrals (host float64, copied).  h: k*k row-major symmetric one-electron
 * integrals; L: n_chol*k*k with (pq|rs) = sum_Q L[Q,p,q] L[Q,r,s] (the form
 * of Eq. 1's H = H0 + V before partitioning).  n_elec active electrons
 * (even; the reference is a singlet with Sz = 0). */
mpspt_status mpspt_set_integrals(mpspt_ctx* ctx, int k_act, int k_virt, int n_elec,
                                 const double* h, const double* L, int n_chol);

/* Reference Psi0 (Eq. 1: "the zeroth order wavefunction", a CASSCF or DMRG
 * state of the active space) as a QN-blocked MPS on the n_sites_act = k_act
 * active sites, the form a DMRG calculation produces.  Site c holds
 * blk_count[c] blocks; the blocks of all sites are listed in site order,
 * and block b has
 *   blk_meta[7b .. 7b+6] = (N_l, 2Sz_l, s, N_r, 2Sz_r, dim_l, dim_r)
 * with s the local state (0..3) and (N_r, 2Sz_r) = (N_l, 2Sz_l) + QN(s),
 * and blk_data[b] -> dim_l x dim_r doubles, row-major (host, copied).  A
 * bond sector must have the same dimension in every block that names it;
 * sectors are ordered ascending in (N, 2Sz) inside a bond.  The first bond
 * is (0, 0) and the last (n_elec, 0), both of dimension 1.  Any norm (the
 * state is normalised).  Duplicate (site, N_l, 2Sz_l, s) blocks, a QN
 * change that does not match s, or non-finite entries give
 * MPSPT_ERR_INVALID.  The library computes gamma_tu and E_ref = <H_act> by
 * MPO transfers on the device, the generalised Fock matrix, and rotates the
 * virtual orbitals to the semicanonical basis.  Requires
 * mpspt_set_integrals. */
mpspt_status mpspt_set_reference(mpspt_ctx* ctx, int n_sites_act, const int* blk_count,
                                 const int* blk_meta, const double* const* blk_data);

/* Convenience form for small active spaces: Psi0 as a dense host vector over
 * the 4^k_act active occupation strings (index = sum_p code_p
 * 4^(k_act-1-p)), copied; gamma and E_ref are computed from the vector and
 * it is converted to an exact MPS (density-matrix splits keeping every state
 * above 1e-14 of the largest).  n_ci must equal 4^k_act (k_act <= 14). */
mpspt_status mpspt_set_reference_ci(mpspt_ctx* ctx, const double* ci, long long n_ci);

/* Ground-state DMRG for the reference (the paper: the Hylleraas sweep "is
 * essentially the same as the standard DMRG sweep"): the two-site sweep
 * minimising <Psi|H_act + s2_penalty S^2|Psi> / <Psi|Psi> over active-space
 * MPS of bond dimension <= M0 in the (n_elec, Sz = 0) sector, with a
 * Davidson local eigensolver (Jacobi correction, residual <= cg_tol
 * max(1, |E|), at most cg_max_iter iterations, else
 * MPSPT_ERR_NOT_CONVERGED) and the same truncation and stopping rules
 * (keep_rel, e_tol, max_sweeps) as the first-order sweep.  s2_penalty >= 0:
 * every state of spin S is raised by s2_penalty S(S+1), so a penalty above
 * half the gap between the lowest state and the lowest singlet makes the
 * sweep find the singlet (0 = the lowest Sz = 0 state, of any spin).  The
 * start is the seeded initial state of the first-order sweep.  The result
 * is installed as the reference exactly as mpspt_set_reference would
 * install it.  e_ref (nullable): E_ref = <Psi0|H_act|Psi0> of the installed
 * state (no penalty); psi0 (nullable): the active-space MPS (free with
 * mpspt_mps_free); rep (nullable): e2_per_sweep holds the penalised energy
 * (last local Ritz value) per sweep.  Requires mpspt_set_integrals. */
mpspt_status mpspt_ground_state(mpspt_ctx* ctx, int M0, double s2_penalty, double* e_ref, mpspt_mps** psi0,
                                mpspt_report* rep);

/* E0 = <Psi0|H0|Psi0>, E1 = <Psi0|V|Psi0> = E_ref - E0 and E_ref =
 * <Psi0|H|Psi0> for the chosen H0 (Eqs. 1, 5).  Any output may be NULL. */
mpspt_status mpspt_energies(mpspt_ctx* ctx, mpspt_h0 h0, double* e0, double* e1,
                            double* e_ref);

/* The hot path: minimises Eq. 1 over MPS of bond dimension <= M with the
 * two-site sweep (paper: "the standard DMRG sweep algorithm ... instead of an
 * eigenvalue problem, a linear equation is solved at each step").  Writes E2
 * = the Hylleraas value of the last local step (float64; an upper bound to
 * the uncontracted E2 when H0 - E0 > 0 on X).  If psi1 is not NULL, *psi1
 * receives the final first-order MPS (free with mpspt_mps_free).  rep may be
 * NULL.  Initial Psi1: see the sector rule and SplitMix64 values documented
 * in the library source (seed from the options). */
mpspt_status mpspt_minimize_hylleraas(mpspt_ctx* ctx, mpspt_h0 h0, int M, double* e2,
                                      mpspt_mps** psi1, mpspt_report* rep);

/* E2 against the truncation error (the paper's convergence study of E2 with
 * M and its extrapolation in the discarded weight, Figs. 3-4 and the text on
 * the renormalisation step): minimises Eq. 1 at each bond dimension M[j]
 * (j < n_M, with the context's options; every run starts from the seeded
 * initial Psi1) and fits E2(M) = e2_extrap + slope * w(M) by least squares,
 * w(M) = the largest discarded weight of the last sweep (reading: the
 * truncation error of a converged run).  e2_M and w_M (n_M each, nullable)
 * receive the points.  n_M >= 2 with at least two distinct w, else
 * MPSPT_ERR_INVALID. */
mpspt_status mpspt_extrapolate_e2(mpspt_ctx* ctx, mpspt_h0 h0, int n_M, const int* M, double* e2_M, double* w_M,
                                  double* e2_extrap, double* slope);

/* Partitioned E2 (the paper's parallelism over virtual-orbital pairs, not
 * implemented there): H0 conserves the occupation of every semicanonical
 * virtual orbital, so the first-order problem splits exactly into
 * partitions P = (a, b), a <= b (0-based virtual indices): one electron in a
 * and one in b (a < b), or one or two electrons in a (a = b).  Each is an
 * MPS-PT problem on the chain (active orbitals, a[, b]) minimised with its
 * own bond dimension M_part[i]; E2 = sum_P E2_P in the given pair order
 * (float64).  Partitions run concurrently on n_streams CUDA streams (0 =
 * default 8).  pair_ab: 2*n_part ints; e2_part (nullable) receives E2_P. */
mpspt_status mpspt_minimize_partitioned(mpspt_ctx* ctx, mpspt_h0 h0, int n_part,
                                        const int* pair_ab, const int* M_part, int n_streams,
                                        double* e2_total, double* e2_part, mpspt_report* rep);

/* Eq. 5: E3 = <Psi1|V|Psi1> - E1 <Psi1|Psi1> with V = H - H0 (full
 * Hamiltonian MPO restricted to X), by one transfer sweep. */
mpspt_status mpspt_third_order(mpspt_ctx* ctx, mpspt_h0 h0, const mpspt_mps* psi1,
                               double* e3);

/* E3 (Eq. 5) over partitions: Psi1 = sum_P Psi1^P of the listed partitions,
 * each solved as by mpspt_minimize_partitioned (same pair_ab, M_part,
 * n_streams and the same E2 values).  The partitions occupy disjoint
 * virtual-occupation patterns and H0 keeps every pattern, so for P != P'
 * <Psi1^P|Psi1^P'> = <Psi1^P|H0|Psi1^P'> = 0, while V moves up to two
 * electrons between orbitals and couples them:
 *   E3 = sum_P E3(Psi1^P) + 2 sum_{P < P'} <Psi1^P|H|Psi1^P'>.
 * Every Psi1^P is written on the full chain (empty virtual orbitals pass the
 * bond through) and each term is one float64 MPO transfer (three for the
 * E3(Psi1^P) terms); n_part (n_part + 5) / 2 transfers in all, run
 * concurrently on the n_streams lanes.  With all k_v (k_v + 1) / 2
 * partitions at their exact bond dimensions this is the full-space E3.
 * Sums are taken in a fixed order (partitions in list order, then pairs
 * i < j row by row), so the result does not depend on n_streams.
 * Outputs: e2_total, e3_total, e3_cross (the pair sum) are required;
 * e2_part, e3_part (n_part doubles) and h_pair (n_part * n_part doubles,
 * row-major, <Psi1^i|H|Psi1^j> off the diagonal and 0 on it) may be NULL.
 * rep: the partition solves' totals plus e3_ms and e3_transfers.  The
 * partition MPSs are freed before return. */
mpspt_status mpspt_third_order_partitioned(mpspt_ctx* ctx, mpspt_h0 h0, int n_part,
                                           const int* pair_ab, const int* M_part, int n_streams,
                                           double* e2_total, double* e3_total, double* e3_cross,
                                           double* e2_part, double* e3_part, double* h_pair,
                                           mpspt_report* rep);

void mpspt_mps_free(mpspt_mps* mps);

/* MPS exchange in a dense, QN-labelled form.  bond_dims[c], c = 0..nsite:
 * bond dimensions (bond_dims[0] = bond_dims[nsite] = 1).  bond_qn: for every
 * bond index of every cut in order, the pair (N, 2Sz); indices of one QN
 * must be contiguous and sectors ascending in (N, 2Sz).  tensors[c]:
 * bond_dims[c]*4*bond_dims[c+1] doubles, row-major (l, s, r); entries that
 * violate QN conservation must be zero.  Import copies; export writes into
 * caller buffers sized from mpspt_mps_shape(). */
mpspt_status mpspt_mps_import(mpspt_ctx* ctx, int nsite, const int* bond_dims,
                              const int* bond_qn, const double* const* tensors,
                              mpspt_mps** out);
mpspt_status mpspt_mps_shape(const mpspt_mps* mps, int* nsite, int* bond_dims);
mpspt_status mpspt_mps_export(const mpspt_mps* mps, int* bond_qn, double* const* tensors);

/* Local operators at bond (i, i+1) of a given Psi1 (the Fig. 1C terms): with
 * environments of Psi1 built from both ends, and x a dense host two-site
 * tensor (bond_dims[i]*16*bond_dims[i+2], row-major (l, s1, s2, r)):
 *   MPSPT_LOCAL_SIGMA: out = A_loc x   (A_loc = projection of H0 - E0)
 *   MPSPT_LOCAL_RHS:   out = g_loc     (projection of V Psi0; x ignored)
 *   MPSPT_LOCAL_DIAG:  out = diag(A_loc) (Jacobi preconditioner)
 * Entries outside the QN-allowed blocks are written as zero.  Uses the
 * context's precision for SIGMA. */
typedef enum { MPSPT_LOCAL_SIGMA = 0, MPSPT_LOCAL_RHS = 1, MPSPT_LOCAL_DIAG = 2 } mpspt_local_op;
mpspt_status mpspt_local_apply(mpspt_ctx* ctx, mpspt_h0 h0, const mpspt_mps* psi1, int i,
                               mpspt_local_op op, const double* x, double* out);

/* ---- Learned block preconditioner ------------------------------------
 * A 3-layer perceptron (width `width`, bfloat16 weights with float32 master
 * copies, float32 accumulation, ReLU) maps 16 features of each QN block of
 * a local problem (statistics of the H0 - E0 diagonal, of g and of the warm
 * start, the block's quantum numbers and sizes) to two coefficients
 * (gamma_B, delta_B) of the block's initial guess
 *     x0_B = gamma_B * x_warm,B + delta_B * (D^-1 b)_B     (b = -g).
 * Jacobi-preconditioned CG remains the solver; in the sweep the learned
 * guess replaces the warm start only when its float64 residual is smaller,
 * and CG runs to the same tolerance, so E2 is unchanged.  Training pairs
 * come from plain solves (mpspt_harvest): the least-squares (gamma, delta)
 * of the converged solution per block.  Parameter layout: W_l row-major
 * (out x in), b_l (out); l = 1: in = 16, l = 3: out = 2.  All arrays are
 * host float32; the network lives on `device`. */
typedef struct mpspt_mlp mpspt_mlp;
mpspt_status mpspt_mlp_create(int device, int width, unsigned long long seed, mpspt_mlp** out);
void mpspt_mlp_free(mpspt_mlp* net);
mpspt_status mpspt_mlp_set_params(mpspt_mlp* net, const float* W1, const float* b1, const float* W2,
                                  const float* b2, const float* W3, const float* b3);
mpspt_status mpspt_mlp_get_params(const mpspt_mlp* net, float* W1, float* b1, float* W2, float* b2,
                                  float* W3, float* b3);
/* y (batch x 2) = network(x (batch x 16)). */
mpspt_status mpspt_mlp_forward(mpspt_mlp* net, int batch, const float* x, float* y);
/* Mean-squared-error loss 1/(2 batch) sum |y - t|^2 and its gradients with
 * respect to the master parameters (the bfloat16 rounding passed straight
 * through).  Any gradient pointer may be NULL. */
mpspt_status mpspt_mlp_gradient(mpspt_mlp* net, int batch, const float* x, const float* t, float* loss,
                                float* gW1, float* gb1, float* gW2, float* gb2, float* gW3, float* gb3);
/* Adam (beta 0.9 / 0.999) over n samples in order, minibatches of `batch`,
 * `epochs` passes; *loss = mean loss of the last epoch. */
mpspt_status mpspt_mlp_train(mpspt_mlp* net, int n, const float* x, const float* t, int epochs, int batch,
                             float lr, float* loss);
/* Runs the plain sweep (as mpspt_minimize_hylleraas) and records up to
 * max_samples training pairs: x (max x 16) features, t (max x 2) targets. */
mpspt_status mpspt_harvest(mpspt_ctx* ctx, mpspt_h0 h0, int M, int max_samples, float* x, float* t,
                           int* n_samples);
/* Attach a network to the context; used when options.use_learned is set.
 * The context does not own it (NULL detaches). */
mpspt_status mpspt_set_preconditioner(mpspt_ctx* ctx, const mpspt_mlp* net);

/* End-to-end training of the learned preconditioner on the context's own
 * problem: up to max_samples training pairs from a plain sweep at (h0, M)
 * (as mpspt_harvest), a new network of width 256 trained on the GPU for
 * `epochs` passes (Adam, minibatches of 256, learning rate 1e-3, seed from
 * the options), attached to the context (as mpspt_set_preconditioner; the
 * context owns this network and frees it with mpspt_destroy).
 * harvest_path (nullable): if the file exists, its pairs are used instead
 * of harvesting; otherwise the harvested pairs are written to it (int32 n,
 * then float32 x[n * 16], then float32 t[n * 2], native byte order).
 * loss (nullable): mean training loss of the last epoch.  The network is
 * used when options.use_learned is set. */
mpspt_status mpspt_train_preconditioner(mpspt_ctx* ctx, mpspt_h0 h0, int M, int max_samples, int epochs,
                                        const char* harvest_path, float* loss);

/* The float64 eigensolver of the truncation step (density-matrix sectors
 * rho_q = X_q X_q^T, paper text on the renormalisation step) on
 * caller data: batched cyclic Jacobi with round-robin parallel rotations.
 * Device pointers; the batch's matrices are stored back to back: matrix i
 * has size n[i] (host array, 1 <= n[i] <= 2048) and starts at offset
 * sum_{j<i} n[j]^2 of A (row-major, symmetric, not modified) and of V
 * (eigenvectors as columns), and at sum_{j<i} n[j] of w (eigenvalues, in
 * the column order of V, unsorted).  Work is ordered on `stream`
 * (cudaStream_t, 0 = default); the call allocates a work copy of A with
 * cudaMallocAsync on that stream and returns without synchronising. */
mpspt_status mpspt_eigh_batched(int device, void* stream, int batch, const int* n, const double* A,
                                double* V, double* w);

/* Same contract as mpspt_eigh_batched, with the solver the truncation step
 * uses: Jacobi with one launch per sweep (the matrix as a packed triangle in
 * shared memory, the recorded rotations applied to the rows of V by many
 * CTAs in parallel).  f32_start = 0: float64 sweeps from the identity.
 * f32_start = 1: float32 sweeps from the identity, two float64
 * Newton-Schulz steps that restore orthonormality (V <- V (3/2 I -
 * 1/2 V^T V)), then float64 sweeps on V^T A V starting from V, to the same
 * float64 convergence test.  A is left unchanged.  Allocates device scratch
 * (about 4 n^2 doubles per matrix) and returns after the stream has
 * finished the work. */
mpspt_status mpspt_eigh_batched_ex(int device, void* stream, int batch, const int* n, const double* A,
                                   double* V, double* w, int f32_start);

/* Allocation-free variant of mpspt_eigh_batched (the paper has no
 * counterpart; this is a service for callers that cannot allocate device
 * memory during the call -- hosts that reserve all device memory up front
 * for their own allocator, so that a library allocation would fail or go
 * around their accounting, and latency-bound callers that cannot afford the
 * synchronisation a fresh allocation may cost).  Same arguments, results and
 * stream ordering as mpspt_eigh_batched, but the task table and the work
 * copy of A live in one fixed device array of 2^21 doubles (16 MiB) that
 * every GPU loading the library holds until the process exits; the call
 * allocates and frees nothing.  Limits: batch <= 1024 and
 * sum_i n[i]^2 <= 2^21 - 4096 (else MPSPT_ERR_INVALID, nothing launched).
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any
 * stream capture.  The caller's current device is restored before return.
 * All calls share the array and each writes every part of it that it reads
 * (task table and matrix copy) before reading it, so nothing in it has to
 * start at zero.  Calls whose GPU work overlaps (other streams, other host
 * threads) race on it and must be serialised by the caller. */
mpspt_status mpspt_eigh_batched_noalloc(int device, void* stream, int batch, const int* n,
                                        const double* A, double* V, double* w);

const char* mpspt_status_string(mpspt_status s);

#ifdef __cplusplus
}
#endif
#endif /* MPSPT_H */
