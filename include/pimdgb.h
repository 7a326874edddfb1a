/*
 * pimdgb: batched Born-Oppenheimer energies and forces of every replica of a
 * replica-parallel ab initio simulation step, on one GB300 (sm_103a).
 *
 * The paper (arXiv:1601.02713, Sec. 2) states the problem this library
 * solves: a PIMD (or string-method) step produces n nuclear configurations
 * (replicas: beads or images); the Born-Oppenheimer energy and forces of each
 * replica are computed, gathered, and the driver moves the replicas. Each
 * energy/force here is a closed-shell restricted Hartree-Fock (RHF) direct SCF
 * in a contracted Gaussian basis: Schwarz-screened electron-repulsion integrals
 * contracted into Coulomb and exchange matrices, Pulay DIIS, diagonalisation,
 * then the analytic gradient from derivative integrals. Integral cutoff 1e-12
 * as in Sec. 3.1. All replicas of a call are evaluated together, ragged sizes
 * included, so a call is the whole force step of the paper's Fig. 1(a).
 *
 * Conventions
 *   units: coordinates in bohr, energies in hartree, gradients dE/dR in
 *          hartree/bohr (the force is minus the gradient);
 *   charge 0, closed shell (the electron count sum(Z) must be even);
 *   at most 768 basis functions per replica;
 *   all array arguments of the host entry points are caller-owned HOST memory,
 *   read before the call returns; outputs are written before it returns
 *   (the call synchronises its stream);
 *   the *_dev entry points take DEVICE pointers (caller-owned, on the device of
 *   the context) and a cudaStream_t passed as void*; they return after the
 *   results are in the caller's device buffers (the stream is synchronised).
 *   Errors are negative return codes (pimd_strerror gives a message); on error
 *   outputs are unspecified except for PIMD_ENOTCONV (see below).
 *   A context is not thread-safe: one host thread at a time per context.
 */
#ifndef PIMDGB_H
#define PIMDGB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIMD_OK 0
#define PIMD_EINVAL -1     /* bad argument: sizes, NaN coordinates, element missing from basis, odd electrons */
#define PIMD_ENOMEM -2     /* device allocation failed */
#define PIMD_ECUDA -3      /* CUDA runtime error */
#define PIMD_ENOTCONV -4   /* some replica's SCF did not converge in max_iter; outputs written, info flags it */
#define PIMD_ETIMEOUT -5   /* a bounded device wait expired */
#define PIMD_EBASIS -6     /* overlap matrix numerically singular (min eigenvalue < 1e-8) */

typedef struct pimd_ctx pimd_ctx;
typedef struct pimd_basis pimd_basis;

/* SCF options. struct_size must be sizeof(pimd_scf_opts); fields added later
 * go at the end. pimd_scf_opts_default fills the defaults shown. */
typedef struct {
    size_t struct_size;
    double conv_energy;   /* |E_k - E_{k-1}| threshold, 1e-10 hartree */
    double conv_error;    /* max |X^T (FDS - SDF) X| threshold, 1e-8 */
    int max_iter;         /* 64 */
    int diis_size;        /* 8 (Pulay subspace, 2..16) */
    double schwarz_tau;   /* 1e-12: quartets with Q_ab Q_cd below it are skipped (Sec. 3.1) */
    double fp32_tau;      /* 0: all quartets in FP64; > schwarz_tau: quartets whose bound
                             Q_ab Q_cd max|D block| is below it (D: the density increment of an
                             incremental build) are evaluated in FP32 and accumulated in FP64 */
    int guess;            /* 0 core Hamiltonian, 1 previous MOs of the same replica index (Sec. 2:
                             MOs of each replica reused as the next step's guess), falls back to 0;
                             2 learned density (the model attached by pimd_ctx_set_guess_model);
                             3 previous MOs where cached, else the learned density;
                             4 superposition of spherically averaged atomic densities (SAD:
                               fractional-occupation SCF of each isolated neutral atom, 1s 2s 2p
                               configurations, Z <= 10, computed once per basis and element);
                             5 previous MOs where cached, else SAD */
    int deterministic;    /* 0; 1: bitwise-identical results from run to run: the Fock increments,
                             the nuclear repulsion and the gradient accumulate as 64-bit fixed-point
                             integers (resolution 2^-48 for the Fock matrix, 2^-40 hartree(/bohr)
                             for the rest) with integer atomics, whose sum does not depend on the
                             order of the additions; 0 accumulates with FP64 atomics (last bits vary) */
    int want_gradient;    /* 1 */
    int use_graphs;       /* 1: from the second SCF iteration on, each iteration's kernel sequence
                             (density increment + Fock build; Fock assembly, energy and DIIS error;
                             DIIS extrapolation + diagonalisation + density) is replayed as three
                             CUDA graphs captured from the first; 0: plain launches */
    int full_every;       /* 8: after this many SCF iterations without one, the Fock build is a full
                             build (G'(D)) instead of the incremental G' += G'(D - D_prev); 1: every
                             build full. Convergence is only accepted on a full build. */
    double prim_screen;   /* 1/81: within a screened shell quartet, primitive quartets whose bound
                             qp_ij qp_kl max|D block| (qp: Schwarz factor of one primitive pair) is
                             below schwarz_tau * prim_screen are skipped in the Fock build (at most
                             81 per quartet, so their sum stays below schwarz_tau); in the gradient,
                             whose quartets are screened at schwarz_tau / 100 on Q_ab Q_cd |Gamma|
                             (Q carries no derivative scale, hence the margin), a primitive quartet
                             is skipped below schwarz_tau * prim_screen with the derivative bound
                             (qg_ij qp_kl + qp_ij qg_kl) |Gamma|, qg = qp 2 sqrt(2 max exponent),
                             which carries that scale itself; 0 keeps all */
    int reuse_mode;       /* start of a replica from its previous call (guess 1, 3, 5): 0 the density
                             2 C_occ C_occ^T of the cached MOs; 1 that density after two McWeeny
                             purification steps in the new overlap metric; 2 the aufbau density of
                             the cached Fock matrix diagonalised in the new orthogonal basis */
    /* Force-parallel split (the paper's force groups, Sec. 2: the integral
     * work of every replica shared by m processes): split_size = m > 1
     * processes call the same forces entry point with the same replicas and
     * options except split_rank (0..m-1); each evaluates every m-th quartet
     * tile of each class pair and after every Fock build, and after the
     * two-electron gradient, calls reduce_fn(buf, n, reduce_user) on the host
     * (the stream synchronised), which must replace the n doubles of the
     * DEVICE buffer buf by their sum over the m processes (an all-reduce,
     * e.g. NCCL) and return 0; all processes then take the same SCF path.
     * CUDA graphs still apply to the other kernel sequences of an iteration. */
    int split_size;       /* 1 */
    int split_rank;       /* 0 */
    int (*reduce_fn)(double* buf, long long n, void* user);
    void* reduce_user;
} pimd_scf_opts;

/* Per-replica result record. */
typedef struct {
    int iterations;       /* SCF iterations (Fock builds) */
    int converged;        /* 1 if both thresholds were met */
    double final_dE;      /* last |E_k - E_{k-1}| */
    double final_error;   /* last max |X^T (FDS - SDF) X| */
    long long nquartets;  /* screened shell quartets per Fock build */
    long long nq_fp64;    /* shell quartets of the replica executed in FP64, all Fock builds of the call */
    long long nq_fp32;    /* ... and in FP32 (mixed mode: bound below fp32_tau) */
} pimd_info;

void pimd_scf_opts_default(pimd_scf_opts* opts);

/* Create a context on CUDA device `device` (owns streams, workspaces, the
 * Boys table and the per-replica MO cache). Returns 0 or an error. */
int pimd_ctx_create(pimd_ctx** out, int device);
void pimd_ctx_destroy(pimd_ctx* ctx);

/* Basis set, per element (immutable after creation).
 *   nelem            number of elements described;
 *   Z_of_elem[e]     nuclear charge of element e (1..118, distinct);
 *   nshell_of_elem[e] number of contracted shells of element e;
 *   shell_l[s], shell_nprim[s]  angular momentum (0..2) and primitive count
 *                    (1..3) of shell s, shells of element 0 first, then 1, ...;
 *   exps, coefs      primitive exponents and raw contraction coefficients of
 *                    every shell in order (coefficients multiply normalised
 *                    primitives; the library normalises each contraction);
 *   spherical        1: d shells are the 5 real solid harmonics (m = -2..2:
 *                    sqrt3 xy, sqrt3 yz, zz-(xx+yy)/2, sqrt3 xz, sqrt3/2 (xx-yy));
 *                    0 is rejected (PIMD_EINVAL) in this version.
 * Within a shell, p functions are ordered x, y, z. */
int pimd_basis_create(pimd_basis** out, int nelem, const int* Z_of_elem, const int* nshell_of_elem,
                      const int* shell_l, const int* shell_nprim, const double* exps, const double* coefs,
                      int spherical);
void pimd_basis_destroy(pimd_basis* basis);

/* Number of basis functions of a molecule with the given charges. */
int pimd_basis_nbf(const pimd_basis* basis, int natom, const int* Z);

/* PIMD beads (Sec. 2, Fig. 1(a)): nrep replicas of the same molecule.
 *   Z[natom], coords[nrep][natom][3] (bohr)  -> energies[nrep] (hartree),
 *   gradients[nrep][natom][3] (hartree/bohr; may be NULL if opts->want_gradient == 0),
 *   info[nrep] (may be NULL). opts may be NULL (defaults). */
int pimd_bo_forces(pimd_ctx* ctx, int nrep, int natom, const int* Z, const double* coords,
                   const pimd_basis* basis, const pimd_scf_opts* opts, double* energies, double* gradients,
                   pimd_info* info);

/* String-method images (Sec. 3.2): nimg replicas of different sizes.
 *   natom_of_img[nimg]; Z_concat and coords_concat ([sum natom][3], bohr)
 *   hold the images one after another; gradients_concat is laid out the same. */
int string_images_forces(pimd_ctx* ctx, int nimg, const int* natom_of_img, const int* Z_concat,
                         const double* coords_concat, const pimd_basis* basis, const pimd_scf_opts* opts,
                         double* energies, double* gradients_concat, pimd_info* info);

/* Device-pointer variants: Z and natom_of_img stay HOST arrays (they fix the
 * work layout); coords, energies and gradients are DEVICE pointers; stream is
 * a cudaStream_t (NULL: the context's stream). */
int pimd_bo_forces_dev(pimd_ctx* ctx, int nrep, int natom, const int* Z, const double* coords_dev,
                       const pimd_basis* basis, const pimd_scf_opts* opts, double* energies_dev,
                       double* gradients_dev, pimd_info* info, void* stream);
int string_images_forces_dev(pimd_ctx* ctx, int nimg, const int* natom_of_img, const int* Z_concat,
                             const double* coords_concat_dev, const pimd_basis* basis, const pimd_scf_opts* opts,
                             double* energies_dev, double* gradients_concat_dev, pimd_info* info, void* stream);

/* Screening stage alone (Schwarz factors and quartet lists, Sec. 3.1 cutoff):
 * counts[r] = shell quartets of replica r whose bound Q_ab Q_cd is at least
 * schwarz_tau, for nrep replicas laid out as in string_images_forces (host
 * arrays). The work of a replica's Fock build grows with this count; a caller
 * that splits one step's replicas over several GPUs balances the parts by it
 * (the paper's load balance over images, Sec. 3.2). */
int pimd_screened_quartets(pimd_ctx* ctx, int nrep, const int* natom_of, const int* Z_concat,
                           const double* coords_concat, const pimd_basis* basis, double schwarz_tau,
                           long long* counts);

/* Drop the cached MOs (guesses 1, 3 and 5 then start from their fallback:
 * the core Hamiltonian, the learned density, SAD). */
void pimd_ctx_clear_guess(pimd_ctx* ctx);

/* Launch statistics of the last forces call: kernels launched, Fock builds,
 * and the device time (ms, CUDA events on the context stream) of the ERI
 * Fock-build kernels, of the two-electron gradient kernels and of the whole call. */
typedef struct {
    long long kernel_launches;
    int fock_builds;
    double ms_fock;
    double ms_grad2e;
    double ms_total;
    long long nquartets_total;   /* Schwarz-screened quartets over all replicas (full build) */
    double eri_flops_per_build;  /* executed floating-point operations of the primitive loop per Fock build,
                                    averaged over the call's builds (generated recursion + per-primitive
                                    set-up and Boys, counted from the generated code), all replicas */
    double eris_per_build;       /* executed unique contracted basis-function ERIs per Fock build (average) */
    double eri_flops32_per_build;  /* the same operations count for the FP32 quartets (mixed mode) */
    long long quartets_fp64;     /* executed shell quartets of all Fock builds of the call, FP64 */
    long long quartets_fp32;     /* ... and FP32 (fp32_tau > 0) */
    double eris32_per_build;     /* the part of eris_per_build evaluated in FP32 */
    double grad_flops;           /* executed floating-point operations of the two-electron gradient's
                                    primitive loop in FP64 (generated recursion to order L + 1 with its
                                    four accumulated sets, set-up and Boys), all replicas */
    double grad_flops32;         /* the same for its FP32 quartets (mixed mode) */
    long long grad_quartets;     /* executed shell quartets of the two-electron gradient */
} pimd_stats;
int pimd_last_stats(const pimd_ctx* ctx, pimd_stats* out);

/* SCF convergence record of replica `rep` in the last forces call: per SCF
 * iteration k < min(returned count, maxit), energy[k] (hartree, the energy of
 * that iteration's Fock build), error[k] (max |X^T (FDS - SDF) X|) and
 * full_build[k] (1 full Fock build, 0 incremental). Any output may be NULL.
 * Returns the number of iterations of the replica, or a negative error. */
int pimd_last_trace(const pimd_ctx* ctx, int rep, int maxit, double* energy, double* error, int* full_build);

/* Fock builds of the last forces call, per SCF iteration k < min(returned
 * count, maxit) (one build covers every replica still iterating): ms[k] the
 * device time of the build (CUDA events on the context stream) and
 * quartets[k] the shell quartets it executed (FP64 and FP32). Either output
 * may be NULL. Returns the number of iterations, or a negative error. */
int pimd_last_fock_times(const pimd_ctx* ctx, int maxit, double* ms, long long* quartets);

/* Testing hooks (same kernels as the forces path):
 * pimd_fock_dev: for nrep replicas of one molecule and a given density
 *   D[nrep][N][N] (device), write G = J - K/2 (device, [nrep][N][N]) with
 *   J_mn = sum D_ls (mn|ls), K_mn = sum D_ls (ml|ns) (Schwarz cutoff
 *   schwarz_tau; quartets below fp32_tau in FP32 when fp32_tau > schwarz_tau).
 * pimd_one_electron: S, T, V matrices of one molecule (host arrays [N][N]).
 * pimd_boys_dev: F_dev[i] = F_m(T_dev[i]) = int_0^1 t^(2m) exp(-T t^2) dt for
 *   n device values, order 0 <= m <= 12 (the tabulated evaluation of the ERI
 *   kernels); a negative or non-finite T gives NaN. */
int pimd_fock_dev(pimd_ctx* ctx, int nrep, int natom, const int* Z, const double* coords, const pimd_basis* basis,
                  double schwarz_tau, double fp32_tau, const double* D_dev, double* G_dev);
int pimd_one_electron(pimd_ctx* ctx, int natom, const int* Z, const double* coords, const pimd_basis* basis,
                      double* S, double* T, double* V);
int pimd_boys_dev(pimd_ctx* ctx, int n, int m, const double* T_dev, double* F_dev);
/* pimd_boys_f32_dev: the same function in the FP32 evaluation of the
 *   mixed-precision quartets (float T_dev[n] -> float F_dev[n], 0 <= m <= 12);
 *   variant 0 is the compile-time-order form of the straight-line ERI
 *   kernels, 1 the runtime-order form of the cooperative kernels. */
int pimd_boys_f32_dev(pimd_ctx* ctx, int n, int m, const float* T_dev, float* F_dev, int variant);
/* pimd_sad_atomic_density: the atomic density of element Z used by the SAD
 * guess (guess = 4, 5), host array D[n][n], n = functions of Z in the basis. */
int pimd_sad_atomic_density(pimd_ctx* ctx, const pimd_basis* basis, int Z, double* D, int n);

/* Batched symmetric eigensolver of the SCF diagonalisation step (the
 * Roothaan-Hall eigenproblem solved in every SCF cycle, Sec. 3.1): nmat
 * symmetric n x n matrices A_dev[nmat][n][n] (device, row-major) ->
 * eigenvalues evals_dev[nmat][n] in ascending order and eigenvectors as the
 * columns of V_dev[nmat][n][n] (device, row-major; V[i][k] is component i of
 * vector k). One-sided Jacobi on A + sigma I (sigma from the Gershgorin
 * bound), n <= 768. Uses a workspace of the context (allocated on demand).
 * stream: the caller's cudaStream_t or NULL; the call returns after the results
 * are written. PIMD_ENOTCONV (results written) if some matrix is still
 * rotating after 60 sweeps. */
int pimd_eigh_dev(pimd_ctx* ctx, int nmat, int n, const double* A_dev, double* V_dev, double* evals_dev,
                  void* stream);

/* The same eigensolver for callers that must not allocate device memory
 * (the paper has no counterpart: this is a library convenience). Callers whose
 * device memory is owned by another allocator, or whose loop must not take the
 * implicit device synchronisation of cudaMalloc/cudaFree, cannot use the
 * context-based call above; this one calls no allocator at all. Its workspace
 * is a fixed device array of 2,097,152 doubles (16 MiB) plus room for 1024
 * matrix descriptors, held by every GPU that loads the library until the
 * process exits. Limits: n <= 768, nmat <= 1024 and nmat * n * n <= 2,097,152, else
 * PIMD_EINVAL. Arguments as for pimd_eigh_dev; no context is needed (the
 * current CUDA device is used). Unlike pimd_eigh_dev, the call only enqueues
 * its kernels on `stream` and returns without waiting for them: the results
 * are in V_dev and evals_dev once the stream reaches that point, and a matrix
 * that exceeds the solver's sweep limit is not reported (pimd_eigh_dev returns
 * PIMD_ENOTCONV for it). The first call on a device resolves the array
 * addresses on that device; make that first call before any stream capture.
 * All calls share the one workspace, which keeps the last call's contents
 * (the solver overwrites every element it reads): calls that overlap on the
 * GPU (from several host threads or streams) race and give wrong results. */
int pimd_eigh_noalloc(int nmat, int n, const double* A_dev, double* V_dev, double* evals_dev, void* stream);

/* ------------------------------------------------------------------------
 * Learned initial density (no counterpart in the paper, which reuses the
 * previous step's MOs, Sec. 2): a multilayer perceptron predicts every
 * atom-pair block of the density matrix, A == B included, from invariant
 * features of the pair's environment, in a local frame of the pair (e_z along
 * A -> B, or for A == B towards A's nearest neighbour; e_x from the atom
 * nearest the midpoint, or A's second-nearest neighbour). Blocks of pairs
 * more than 4 Angstrom apart are zero. The predicted blocks are rotated to
 * the lab frame, same-atom blocks symmetrised, and the matrix scaled to
 * tr(D S) = number of electrons; the SCF's first Fock build and
 * diagonalisation then make it idempotent. It changes the number of SCF
 * iterations, never the converged result. Elements H, C and O only, at most
 * 14 basis functions and 8 shells per atom.
 * Network: 96 features -> 3 hidden layers of 256 (SiLU) -> one linear head
 * per pair type (the same atom H, C or O; the element pairs OO, OC, OH, CC,
 * CH, HH), head width = the block size. BF16 GEMMs on the 5th-generation
 * tensor cores (tcgen05) with FP32 accumulation, FP32 master weights, Adam. Everything runs on the device of
 * the current CUDA device at creation.
 */
typedef struct pimd_guess pimd_guess;

/* Create a model for the basis (its per-element shells fix the head sizes);
 * weights initialised from `seed` (Glorot uniform). */
int pimd_guess_create(pimd_guess** out, const pimd_basis* basis, unsigned long long seed);
void pimd_guess_destroy(pimd_guess* g);
/* Number of parameters (weights and biases, in the layout of pimd_guess_mlp_grad). */
long long pimd_guess_nparam(const pimd_guess* g);
/* Converge the SCF of nrep replicas of one molecule (arguments as for
 * pimd_bo_forces; the gradient is not computed) and add every replica's
 * converged density blocks, in the local frames, with the pairs' features to
 * the model's training set (held on the device). info[nrep] may be NULL. */
int pimd_guess_add_data(pimd_guess* g, pimd_ctx* ctx, int nrep, int natom, const int* Z, const double* coords,
                        const pimd_basis* basis, const pimd_scf_opts* opts, pimd_info* info);
/* Replicas in the training set. */
long long pimd_guess_ndata(const pimd_guess* g);
void pimd_guess_clear_data(pimd_guess* g);
/* `epochs` passes of Adam (learning rate lr) over the training set, one step
 * per pimd_guess_add_data call's replicas; loss_history[epochs] (may be NULL)
 * gets each epoch's mean squared error over the set, weighted per entry. */
int pimd_guess_train(pimd_guess* g, int epochs, double lr, double* loss_history);
/* Mean squared error of the current weights over the training set. */
int pimd_guess_loss(pimd_guess* g, double* loss);
/* Weights to / from a file (the model's basis must match). */
int pimd_guess_save(const pimd_guess* g, const char* path);
int pimd_guess_load(pimd_guess* g, const char* path);
/* Attach (or with NULL detach) the model used by guess = 2 and 3; the
 * context does not own it. */
int pimd_ctx_set_guess_model(pimd_ctx* ctx, pimd_guess* g);

/* Testing hooks of the learned guess (same kernels as above).
 * pimd_guess_pair_data: the pair rows of one molecule: npair_out, pair_AB
 *   [npair][2] (A, B atom indices), block_off[npair] (offset of the pair's
 *   block, row-major nbf_A x nbf_B, in local_out / local_in), feats
 *   [npair][96] (float), frames [npair][9] (rows e_x, e_y, e_z); if D (host,
 *   N x N) is given, local_out gets M_A^T D_AB M_B for every pair; if
 *   local_in is given, D_out (N x N) gets the lab blocks M_A L M_B^T of the
 *   pairs within the cutoff (same-atom blocks symmetrised first), zero
 *   elsewhere, unscaled. Arrays sized for npair_max pairs (n(n+1)/2) and
 *   nout_max block entries.
 * pimd_guess_mlp_grad: loss (mean over all n x width entries) and gradients
 *   of the network on given features X[n][96] and targets Y[n][width] of one
 *   pair type (0..2 the same atom H, C, O; 3..8 the pairs OO, OC, OH, CC, CH,
 *   HH, heavier element first; width = nbf_A x nbf_B); params_out / grads_out (pimd_guess_nparam floats each, may be
 *   NULL) get the FP32 weights and the gradient. Layout per layer k (3 hidden,
 *   then 9 heads): W_k row-major [fan_in][fan_out], then b_k[fan_out]. */
int pimd_guess_pair_data(pimd_guess* g, int natom, const int* Z, const double* coords, const double* D,
                         const float* local_in, int npair_max, long long nout_max, int* npair_out, int* pair_AB,
                         long long* block_off, float* feats, double* frames, float* local_out, double* D_out);
int pimd_guess_mlp_grad(pimd_guess* g, int n, int type, const float* X, const float* Y, double* loss,
                        float* params_out, float* grads_out);
/* pimd_bf16_gemm_dev: the network's GEMM alone, C[M][N] (float, device) =
 *   op(A) op(B) with bf16 device matrices A, B (row-major, leading dimensions
 *   lda, ldb; ta / tb = 1 reads the transpose), FP32 accumulation, on the
 *   5th-generation tensor cores (tcgen05, accumulator in tensor memory).
 *   PIMD_ETIMEOUT if a bounded wait expired. */
int pimd_bf16_gemm_dev(int M, int N, int K, const void* A, int lda, int ta, const void* B, int ldb, int tb, float* C,
                       int ldc, void* stream);

/* Autotuner (the paper has none: its work distribution is a static MPI
 * split): per quartet class pair, times the Fock build of the given replicas
 * (SAD density, the options' thresholds) with every generated kernel variant
 * (straight-line kernel with ket tiles of 32, 64 or 128 quartets per block;
 * cooperative tape kernel) and then the gradient with each of its
 * variants, and keeps the fastest in the context; later calls on the context
 * use them. widths[64] (may be NULL): widths[cp] = the Fock choice (32, 64,
 * 128, or 0 for the cooperative kernel), widths[32 + cp] = the gradient choice
 * (0 cooperative, 1 straight-line), cp < 21 for s/p/d. ms_best (may be NULL):
 * the summed Fock-build time of the chosen variants. Elements up to Z = 10
 * (it uses the SAD density). */
int pimd_autotune(pimd_ctx* ctx, int nrep, int natom, const int* Z, const double* coords, const pimd_basis* basis,
                  const pimd_scf_opts* opts, int* widths, double* ms_best);

/* Roofline denominators measured on the device: FP64 FMA, FP32 FMA and FP64
 * tensor-core MMA throughput in TFLOP/s (bounded microbenchmarks, ~1 s). Any
 * output pointer may be NULL. No counterpart in the paper (measurement aid). */
int pimd_peak_bench(int device, double* fp64_tflops, double* fp32_tflops, double* dmma_tflops);

const char* pimd_strerror(int code);
/* Detail of the last error a call on ctx returned (which CUDA call failed and
 * its message, or which argument was rejected); "" if none. The string belongs
 * to the context and stays valid until its next call. */
const char* pimd_last_error(const pimd_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
