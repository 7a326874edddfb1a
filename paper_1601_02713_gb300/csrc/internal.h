// Internal interface between the host-side SCF driver and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "pimd_dev.cuh"

struct pimd_basis;
struct pimd_guess;

namespace pimd {

// molecule-level arrays of one call (all replicas concatenated)
struct AtomsDev {
    const double* xyz;      // [natom_total][3]
    const double* Z;        // [natom_total]
    const int* rep_atom0;   // [nrep + 1] first atom of each replica
};

struct BasisPrimDev {
    const double* exps;     // normalised basis primitives
    const double* coefs;
    const int* sprim;       // per shell: first primitive in exps/coefs
    const int* snprim;      // per shell: number of primitives
};

// pair data of `npair` pairs listed in P (sa/sb already set)
void launch_pair_data(const Pairs& P, int* npp, double* pp, const Shells& S, const BasisPrimDev& B,
                      cudaStream_t st);

// S, T, V (spherical) of every pair into the replica matrices
void launch_one_electron(const Pairs& P, const Shells& S, const BasisPrimDev& B, const AtomsDev& At,
                         const Reps& R, double* Sm, double* Tm, double* Vm, const double* boys, cudaStream_t st);

// one-electron gradient: 2 sum D dh/dA - 2 sum W dS/dA (bra derivatives over ordered pairs)
// plus the Hellmann-Feynman term, accumulated into grad[natom_total][3]
void launch_grad_1e(const Pairs& P, const Shells& S, const BasisPrimDev& B, const AtomsDev& At, const Reps& R,
                    const double* D, const double* W, double* grad, const double* boys, double fxs,
                    cudaStream_t st);

// nuclear repulsion energy per replica (added into enn[rep]) and its gradient
// (fxs > 0: enn and grad are fixed-point accumulators, see det_add)
void launch_vnn(const AtomsDev& At, int natom_total, const int* atom_rep, double* enn, double* grad,
                cudaStream_t st, double fxs = 0.0);
// in-place conversion of n values between FP64 and the fixed-point integers
// of det_add (scale fxs)
void launch_double_to_fixed(double* a, long long n, double fxs, cudaStream_t st);
void launch_fixed_to_double(double* a, long long n, double fxs, cudaStream_t st);

// ERI kernels, per class pair index (0..20 over (X, Y), X >= Y in the order
// ss, ps, pp, ds, dp, dd)
int n_class_pairs();
void class_pair_ls(int cp, int* la, int* lb, int* lc, int* ld);
// floating-point operations per primitive quartet of class pair cp: the
// generated recursion plus per-primitive set-up, Boys and prefactor
long long class_vrr_flops(int cp);
long long class_grad_flops(int cp);   // per primitive quartet of the gradient
// Fock build of one class pair: quartets with bound >= max(tau, fp32_tau) in
// FP64 (D, boys), those in [tau, fp32_tau) in FP32 (Df, boysf); counters
// cnt[0..1] FP64 quartets / primitive quartets, cnt[2..3] the same in FP32;
// bs = threads per block = the tiles' ket width for the straight-line
// kernel, bs = 0 for the cooperative kernel (a class with one variant
// ignores the choice)
// tau_prim: primitive quartets with qp_i qp_j max|D block| below it are skipped (0: none)
// fxs > 0: G accumulated as fixed-point integers scaled by fxs (deterministic mode, det_add)
void launch_jk(int cp, const Pairs& P, const Shells& S, const Reps& R, const Tile* tiles, int ntiles,
               const double* D, const float* Df, double* G, const double* boys, const float* boysf, double tau,
               double fp32_tau, const double* Dsh, unsigned long long* cnt, int bs, double tau_prim, double fxs,
               cudaStream_t st);
// kernel variants generated for a class pair: the cooperative tape
// kernel and the straight-line kernel, for the Fock build and the gradient
bool class_pair_coop(int cp);
bool class_pair_straight(int cp);
bool grad_pair_coop(int cp);
bool grad_pair_straight(int cp);
void launch_schwarz(int pair_class, const Pairs& P, const Shells& S, const int* list, int n, const double* boys,
                    double* Q, cudaStream_t st);
// primitive-pair Schwarz factors qp of the listed pairs of one class; reorders
// each pair's primitive data in pp by descending qp
void launch_prim_schwarz(int pair_class, const Pairs& P, const Shells& S, const int* list, int n,
                         const double* boys, double* pp, float* qp, float* qg, cudaStream_t st);
// two-electron gradient of class pair cp: quartets with bound Q_ab Q_cd |Gamma|
// >= max(tau, fp32_tau) in FP64, those in [tau, fp32_tau) in FP32; variant 0
// the cooperative kernel, 1 the straight-line kernel with bs threads per
// block (a class with one variant ignores the choice)
// (tau_prim: primitive quartets with (qg_i qp_j + qp_i qg_j) |Gamma| below it are skipped; 0 none)
// cnt[0..1]: executed FP64 quartets and primitive quartets, cnt[2..3] FP32
void launch_grad2e(int cp, const Pairs& P, const Shells& S, const Reps& R, const Tile* tiles, int ntiles,
                   const double* D, double* grad, const double* boys, const float* boysf, double tau,
                   double fp32_tau, const double* Dsh, unsigned long long* cnt, int variant, int bs,
                   double tau_prim, double fxs, cudaStream_t st);
void grad2e_tapes_upload();   // once per device
void boys_table_upload(double** dev_tab, float** dev_tabf);
// FP32 copies for the mixed-precision quartets
void launch_to_float(const double* src, float* dst, long long n, cudaStream_t st);

// ------------------------------------------------------------------ linalg
struct GemmDesc {
    int M, N, K;
    const double* A;
    int lda, ta;
    const double* B;
    int ldb, tb;
    double* C;
    int ldc;
    double alpha, beta;
    int rep;          // replica (checked against the active mask; -1: always)
};
void launch_gemm(const GemmDesc* d_desc, int ndesc, int maxM, int maxN, const int* active, cudaStream_t st);

struct RepMat {       // per replica matrix view
    int N, nocc;
    long long off;    // element offset of the N x N matrices
};
// one-sided Jacobi eigensolver of symmetric A (per replica, ascending order):
// evals[rep][N] (offset rep * ldE), V columns = eigenvectors (row-major N x N at off);
// notconv[rep] (may be NULL) is set to 1 for a matrix still rotating after the sweep limit
void launch_jacobi(const RepMat* d_rm, int nrep, const double* A, double* V, double* evals, int ldE,
                   double* work, const int* active, int shift_to_spd, cudaStream_t st, int* notconv = nullptr);

void launch_fock_assemble(const RepMat* rm, int nrep, const double* h, const double* G, double* F,
                          const int* active, cudaStream_t st);
void launch_energy(const RepMat* rm, int nrep, const double* D, const double* h, const double* F,
                   const double* enn, double* E, const int* active, cudaStream_t st);
void launch_antisym(const RepMat* rm, int nrep, const double* M, double* E, const int* active, cudaStream_t st);
void launch_maxabs(const RepMat* rm, int nrep, const double* A, double* out, const int* active, cudaStream_t st);
void launch_orth_from_eig(const RepMat* rm, int nrep, const double* U, const double* s, int ldE, double* X,
                          cudaStream_t st);
void launch_scale_cols(const RepMat* rm, int nrep, const double* C, const double* evals, int ldE, double* out,
                       const int* mask, cudaStream_t st);
// DIIS
// (stride: elements between one replica's history matrices, maxN^2)
void launch_diis_store(const RepMat* rm, int nrep, const double* F, const double* E, double* Fh, double* Eh,
                       const int* slot, int hist, long long stride, const int* active, cudaStream_t st);
void launch_diis_dots(const RepMat* rm, int nrep, const double* Eh, const int* slot, const int* count, int hist,
                      long long stride, double* B, const int* active, cudaStream_t st);
void launch_diis_solve(int nrep, const double* B, const int* slot, const int* count, int hist, double* coef,
                       const int* active, cudaStream_t st);
void launch_diis_combine(const RepMat* rm, int nrep, const double* Fh, const double* coef, int hist,
                         long long stride, const double* F, double* Fbar, const int* diis_on, const int* active,
                         cudaStream_t st);
void launch_copy_mats(const RepMat* rm, int nrep, const double* src, double* dst, const int* mask,
                      cudaStream_t st);
void launch_identity(const RepMat* rm, int nrep, double* A, const int* mask, cudaStream_t st);
void launch_boys_eval(int n, int m, const double* T, double* F, const double* boys, cudaStream_t st);
void launch_boys_eval_f32(int n, int m, const float* T, float* F, const float* boysf, int variant, cudaStream_t st);
void gather_xyz(const double* atom_xyz, const int* shell_atom, int nshell, double* shell_xyz, cudaStream_t st);
void add_mats(const RepMat* rm, int nrep, const double* A, const double* B, double* C, cudaStream_t st);
// shell-pair bounds Dsh[r][a][b] = max |M_mn| over the block (replicas in mask)
void launch_shell_bounds(const Shells& S, const Reps& R, int nrep, int maxsh, const double* M, double* Dsh,
                         const int* mask, cudaStream_t st);
// incremental Fock build: dD = D - Dprev (mode 1) or D (mode 2), G zeroed for
// mode 2, Dprev <- D; mode 0 replicas untouched
void launch_delta_density(const RepMat* rm, int nrep, const double* D, double* Dprev, double* dD, double* G,
                          const int* mode, cudaStream_t st);

// D[rep] block (f0..f0+n)^2 <- src[off..off+n*n] for each descriptor {rep, f0, n, off}
void launch_place_blocks(const RepMat* rm, const int* desc4, int nblk, const double* src, double* D,
                         cudaStream_t st);

// ------------------------------------------------------------------ learned guess
// shells (angular momenta into l_out, at most maxsh) of element Z: count, or -1
int basis_elem_shells(const pimd_basis* b, int Z, int* l_out, int maxsh);
// basis functions per atom of element Z in the model's basis, or -1
int guess_elem_nbf(const pimd_guess* g, int Z);
int guess_device(const pimd_guess* g);
// converged densities d_D [rm] of nrep replicas -> a training row set of the model
int guess_collect_device(pimd_guess* g, int nrep, const int* natom_of, const int* Zc,
                         const std::vector<int>& atom_f0, const double* d_xyz, const int* d_Z, const int* d_atom0,
                         const RepMat* d_rm, double* d_D, cudaStream_t st);
// predicted densities of the replicas in mask (host and device copies) into d_D
int guess_predict_device(pimd_guess* g, int nrep, const int* natom_of, const int* Zc,
                         const std::vector<int>& atom_f0, const std::vector<int>& mask, const double* d_xyz,
                         const int* d_Z, const int* d_atom0, const RepMat* d_rm, const int* d_mask, const double* d_S,
                         double* d_tmp, long long mtot, double* d_D, cudaStream_t st);

}  // namespace pimd
