// Device-side data layout shared by the kernels of the batched RHF library.
//
// Every replica (PIMD bead or string image) of one call is laid out
// side by side: shells, shell pairs and matrices of all replicas live in
// single arrays, indexed by global shell / pair ids and by per-replica matrix
// offsets, so that one launch covers the whole batch (the paper's n replicas
// of a step, Sec. 2), ragged sizes included.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define PIMD_MAXPRIM 3                       // primitives per contracted shell
#define PIMD_MAXPP (PIMD_MAXPRIM * PIMD_MAXPRIM)
#define PIMD_LMAX 2                          // s, p, d shells

namespace pimd {

__host__ __device__ constexpr int ncart(int l) { return (l + 1) * (l + 2) / 2; }
__host__ __device__ constexpr int nsph(int l) { return l < 2 ? ncart(l) : 2 * l + 1; }
// position of (lx, ly, lz) in the order lx = l..0, ly = l-lx..0
__host__ __device__ constexpr int cart_index(int lx, int ly, int lz)
{
    return (lx + ly + lz - lx) * (lx + ly + lz - lx + 1) / 2 + lz;
}

// primitive-pair fields, stored SoA: pp[((f * PIMD_MAXPP) + k) * npair + g];
// the first PP_NERI are what the Fock-build primitive loop reads
enum PPField {
    PP_P = 0,             // p = a + b
    PP_PX, PP_PY, PP_PZ,  // Gaussian product centre P
    PP_K,                 // sqrt(2) pi^{5/4} c_a c_b exp(-ab/p |AB|^2) / p
    PP_PAX, PP_PAY, PP_PAZ,  // P - A
    PP_O2P,               // 1 / (2p)
    PP_O2PP,              // 1 / (2p^2)
    PP_EA, PP_EB,         // exponents a, b (gradient weights)
    PP_NF
};
constexpr int PP_NERI = PP_EA;

struct Shells {           // all replicas concatenated
    const double* xyz;    // [nshell][3] centre (bohr)
    const int* l;
    const int* bf;        // first basis function within the replica
    const int* atom;      // global atom index
    const int* rep;       // replica index
};

struct Pairs {
    int n;                // number of shell pairs (all replicas)
    const int* sa;        // shell with the larger l
    const int* sb;
    const int* npp;       // primitive pairs kept
    const double* pp;     // SoA primitive-pair data
    const double* Q;      // Schwarz factor sqrt(max |(ab|ab)|)
    const float* ppf;     // FP32 copy of pp (mixed-precision quartets)
    const float* qp;      // qp[k * n + g]: Schwarz factor sqrt(max |(ij|ij)|) of primitive pair k alone
                          // (contraction coefficients included); the primitive pairs of every shell
                          // pair are stored in descending order of it
    const float* qg;      // qg[k * n + g] = qp_k 2 sqrt(2 max(a_k, b_k)): the scale of the derivative
                          // integrals of primitive pair k (d/dA of a Gaussian of exponent a ~ sqrt(2a))
};

struct Reps {
    const int* nbf;             // functions per replica
    const long long* moff;      // offset of the replica's N x N matrices
    const int* active;          // 1 while the replica's SCF runs
    const int* sh0;             // first (global) shell of each replica
    const int* nsh;             // shells per replica
    const long long* dsoff;     // offset of the replica's nsh x nsh shell-pair density bounds
    unsigned long long* qrep;   // [nrep][2] executed Fock-build quartets per replica: FP64, FP32
};

// max |M_mn| over the functions of shells (a, b) of replica r (global shell ids)
__device__ __forceinline__ double shell_bound(const Reps& R, const double* __restrict__ Dsh, int r, int a, int b)
{
    const int a0 = R.sh0[r], n = R.nsh[r];
    return __ldg(Dsh + R.dsoff[r] + (size_t)(a - a0) * n + (b - a0));
}

// Accumulation into a shared FP64 result: *p += v with an FP64 atomic, or,
// for bitwise-reproducible runs (fxs > 0), as a 64-bit fixed-point integer
// (v scaled by fxs and rounded) with an integer atomic, which is associative,
// so the sum does not depend on the order of the additions. The buffer then
// holds integers until it is converted back (fixed_to_double).
__device__ __forceinline__ void det_add(double* p, double v, double fxs)
{
    if (fxs > 0.0)
        atomicAdd((unsigned long long*)p, (unsigned long long)__double2ll_rn(v * fxs));
    else
        atomicAdd(p, v);
}
// fixed-point scales of the deterministic mode: Fock increments (|G'| < 2^15),
// gradients and nuclear-repulsion energies (|.| < 2^23)
constexpr double kFixG = 281474976710656.0;     // 2^48
constexpr double kFixGrad = 1099511627776.0;    // 2^40

// one block of quartets: bra pair ab with ket pairs [c0, c1)
struct Tile {
    int ab, c0, c1, rep;
};

}  // namespace pimd
