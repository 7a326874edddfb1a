// Learned initial density: a multilayer perceptron predicts each atom-pair
// block of a replica's density matrix from the pair's local environment; the
// SCF starts from the assembled matrix (its first Fock build and
// diagonalisation turn it into an idempotent density) and converges to the
// same solution as from any other guess, so the guess only changes the number
// of iterations.
//
// * Pairs (A, B), A == B included, of every replica; a pair farther apart than
//   4 Angstrom gets a zero block and no weight in training.
// * Local frame per pair: e_z along A -> B (for A == B towards A's nearest
//   neighbour), e_x from the atom nearest to the midpoint (for A == B the second
//   nearest neighbour of A) made orthogonal to e_z, e_y = e_z x e_x; distance
//   ties go to the lower atom index.
// * Invariant features (80, padded to 96): element one-hots of A and B, a
//   same-atom flag, R_AB, 16 Gaussians of R_AB, and the 8 atoms nearest to the
//   midpoint (element one-hot, coordinates in the local frame, 1/r).
// * Blocks are predicted in the local frame and rotated back with the
//   representation of the frame on each atom's shells (s: 1, p: the 3x3
//   rotation, d: the 5x5 matrix of the real solid harmonics).
// * Network: 96 -> 256 -> 256 -> 256 (SiLU) -> one linear head per pair type,
//   head width = block size. GEMMs in BF16 on the 5th-generation tensor cores
//   (tcgen05, FP32 accumulator in tensor memory); FP32 master weights and Adam;
//   training on the device.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <vector>

#include "../../include/pimdgb.h"
#include "internal.h"
#include "umma_gemm.cuh"

namespace pimd {

constexpr int G_NNEIGH = 8, G_NRBF = 16, G_NF = 96, G_H = 256;
constexpr double G_RCUT = 4.0 / 0.529177210903;
constexpr int G_NTYPE = 9;   // same H, same C, same O, then OO, OC, OH, CC, CH, HH
constexpr int G_NLAYER = 3;
constexpr int G_MAXBF = 14;  // basis functions per atom
constexpr int G_MAXSH = 8;

__host__ __device__ inline int elem_index(int Z) { return Z == 1 ? 0 : (Z == 6 ? 1 : (Z == 8 ? 2 : -1)); }

// type of a pair with elem(A) >= elem(B)
__host__ __device__ inline int pair_type(int eA, int eB, bool same)
{
    if (same) return eA;
    if (eA == 2) return eB == 2 ? 3 : (eB == 1 ? 4 : 5);
    if (eA == 1) return eB == 1 ? 6 : 7;
    return 8;
}

struct GuessPair {
    int rep, A, B, type;  // A, B global atom indices, elem(A) >= elem(B)
    int fa, fb;           // first function of A and B within the replica
    long long out_off;    // offset of the pair's block in the output buffer
};

struct ElemShells {
    int nsh[3];
    int l[3][G_MAXSH];
    int nbf[3];
};

// ---------------------------------------------------------------- features
__device__ inline void vsub(const double* a, const double* b, double* o)
{
    o[0] = a[0] - b[0];
    o[1] = a[1] - b[1];
    o[2] = a[2] - b[2];
}
__device__ inline double vdot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
__device__ inline double vdist(const double* a, const double* b)
{
    double d[3];
    vsub(a, b, d);
    return sqrt(vdot(d, d));
}

// frame rows (e_x, e_y, e_z), features (bf16 and optionally float) and the
// cutoff flag of one pair per thread
__global__ void featurize_kernel(const GuessPair* pairs, int npair, const double* xyz, const int* Zat,
                                 const int* rep_atom0, __nv_bfloat16* X, float* Xf, double* frames, int* within)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= npair) return;
    const GuessPair gp = pairs[q];
    const int a0 = rep_atom0[gp.rep], a1 = rep_atom0[gp.rep + 1];
    const double* RA = xyz + 3 * gp.A;
    const double* RB = xyz + 3 * gp.B;
    const bool same = gp.A == gp.B;
    double M[3], ez[3], v[3];
    int ref = -1;
    for (int x = 0; x < 3; x++) M[x] = 0.5 * (RA[x] + RB[x]);
    if (!same) {
        vsub(RB, RA, ez);
        double best = 1e300;
        for (int i = a0; i < a1; i++) {
            if (i == gp.A || i == gp.B) continue;
            const double r = vdist(xyz + 3 * i, M);
            if (r < best) {
                best = r;
                ref = i;
            }
        }
    } else {
        int n1 = -1, n2 = -1;
        double b1 = 1e300, b2 = 1e300;
        for (int i = a0; i < a1; i++) {
            if (i == gp.A) continue;
            const double r = vdist(xyz + 3 * i, RA);
            if (r < b1) {
                b2 = b1;
                n2 = n1;
                b1 = r;
                n1 = i;
            } else if (r < b2) {
                b2 = r;
                n2 = i;
            }
        }
        if (n1 >= 0) vsub(xyz + 3 * n1, RA, ez);
        else {
            ez[0] = 0.0;
            ez[1] = 0.0;
            ez[2] = 1.0;
        }
        ref = n2;
    }
    const double nz = sqrt(vdot(ez, ez));
    for (int x = 0; x < 3; x++) ez[x] /= nz;
    if (ref >= 0) vsub(xyz + 3 * ref, M, v);
    else {
        v[0] = 1.0;
        v[1] = 0.0;
        v[2] = 0.0;
    }
    double pr = vdot(v, ez);
    for (int x = 0; x < 3; x++) v[x] -= pr * ez[x];
    if (sqrt(vdot(v, v)) < 1e-8) {
        // reference on the pair axis: any direction normal to e_z
        v[0] = fabs(ez[0]) < 0.9 ? 1.0 : 0.0;
        v[1] = fabs(ez[0]) < 0.9 ? 0.0 : 1.0;
        v[2] = 0.0;
        pr = vdot(v, ez);
        for (int x = 0; x < 3; x++) v[x] -= pr * ez[x];
    }
    const double nx = sqrt(vdot(v, v));
    const double ex[3] = {v[0] / nx, v[1] / nx, v[2] / nx};
    const double ey[3] = {ez[1] * ex[2] - ez[2] * ex[1], ez[2] * ex[0] - ez[0] * ex[2], ez[0] * ex[1] - ez[1] * ex[0]};
    double* U = frames + 9 * (size_t)q;
    for (int x = 0; x < 3; x++) {
        U[x] = ex[x];
        U[3 + x] = ey[x];
        U[6 + x] = ez[x];
    }
    float f[G_NF];
    for (int i = 0; i < G_NF; i++) f[i] = 0.f;
    f[elem_index(Zat[gp.A])] = 1.f;
    f[3 + elem_index(Zat[gp.B])] = 1.f;
    f[6] = same ? 1.f : 0.f;
    const double R = vdist(RB, RA);
    f[7] = (float)R;
    const double w = G_RCUT / (G_NRBF - 1);
    for (int k = 0; k < G_NRBF; k++) {
        const double t = (R - k * w) / w;
        f[8 + k] = (float)exp(-t * t);
    }
    // the G_NNEIGH atoms nearest to the midpoint (A and B excluded), by (r, index)
    double last_r = -1.0;
    int last_i = -1;
    for (int k = 0; k < G_NNEIGH; k++) {
        int bi = -1;
        double br = 1e300;
        for (int i = a0; i < a1; i++) {
            if (i == gp.A || i == gp.B) continue;
            const double r = vdist(xyz + 3 * i, M);
            const bool after = r > last_r || (r == last_r && i > last_i);
            if (after && r < br) {
                br = r;
                bi = i;
            }
        }
        if (bi < 0) break;
        last_r = br;
        last_i = bi;
        double d[3];
        vsub(xyz + 3 * bi, M, d);
        float* gk = f + 24 + 7 * k;
        gk[elem_index(Zat[bi])] = 1.f;
        gk[3] = (float)vdot(ex, d);
        gk[4] = (float)vdot(ey, d);
        gk[5] = (float)vdot(ez, d);
        gk[6] = (float)(1.0 / fmax(br, 1e-6));
    }
    for (int i = 0; i < G_NF; i++) {
        X[(size_t)q * G_NF + i] = __float2bfloat16(f[i]);
        if (Xf) Xf[(size_t)q * G_NF + i] = f[i];
    }
    within[q] = R <= G_RCUT ? 1 : 0;
}

// ---------------------------------------------------------------- rotations
// phi_lab = M phi_local for one shell of angular momentum l (U: frame rows).
// A lab function evaluated at r = U^T r' is a combination of local functions:
// p: M = U^T; d: M[n][m] = <Q_m, U Q_n U^T> / 1.5, Q_n the traceless quadratic
// form of harmonic n (<Q_m, Q_n> = 1.5 delta_mn).
__device__ void shell_rot(int l, const double* U, double* M)
{
    if (l == 0) {
        M[0] = 1.0;
        return;
    }
    if (l == 1) {
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) M[i * 3 + j] = U[j * 3 + i];
        return;
    }
    const double h = 0.8660254037844386;  // sqrt3 / 2
    // sqrt3 xy, sqrt3 yz, zz-(xx+yy)/2, sqrt3 xz, sqrt3/2 (xx-yy)
    const double Q[5][9] = {{0, h, 0, h, 0, 0, 0, 0, 0},
                            {0, 0, 0, 0, 0, h, 0, h, 0},
                            {-0.5, 0, 0, 0, -0.5, 0, 0, 0, 1.0},
                            {0, 0, h, 0, 0, 0, h, 0, 0},
                            {h, 0, 0, 0, -h, 0, 0, 0, 0}};
    for (int n = 0; n < 5; n++) {
        double T[9];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double s = 0.0;
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++) s += U[i * 3 + a] * Q[n][a * 3 + b] * U[j * 3 + b];
                T[i * 3 + j] = s;
            }
        for (int m = 0; m < 5; m++) {
            double s = 0.0;
            for (int k = 0; k < 9; k++) s += Q[m][k] * T[k];
            M[n * 5 + m] = s / 1.5;
        }
    }
}

// element (i, j) of the representation of shell angular momentum l
// (s: 1; p: Rp; d: Rd)
__device__ __forceinline__ double rep_el(int l, const double* Rp, const double* Rd, int i, int j)
{
    return l == 0 ? 1.0 : (l == 1 ? Rp[i * 3 + j] : Rd[i * 5 + j]);
}

// The atoms' representations are block diagonal over their shells, so a
// block is rotated shell pair by shell pair:
// to_local = 1: blocks <- M_A^T D_AB M_B (float);
// to_local = 0: D_AB <- M_A L M_B^T (and D_BA its transpose) for the pairs
// within the cutoff, L the predicted block with same-atom blocks symmetrised.
__global__ void block_rotate_kernel(const GuessPair* pairs, int npair, const double* frames, ElemShells es,
                                    const int* Zat, const RepMat* rms, double* Dmat, float* blocks,
                                    const int* within, int to_local)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= npair) return;
    const GuessPair gp = pairs[q];
    if (!to_local && !within[q]) return;
    const int eA = elem_index(Zat[gp.A]), eB = elem_index(Zat[gp.B]);
    if (eA < 0 || eB < 0) return;
    const int nb = es.nbf[eB];
    const double* U = frames + 9 * (size_t)q;
    double Rp[9], Rd[25];
    shell_rot(1, U, Rp);
    shell_rot(2, U, Rd);
    const int N = rms[gp.rep].N;
    double* D = Dmat + rms[gp.rep].off;
    float* blk = blocks + gp.out_off;
    const bool same = gp.A == gp.B;
    int oa = 0;
    for (int sa = 0; sa < es.nsh[eA]; sa++) {
        const int la = es.l[eA][sa], ka = nsph(la);
        int ob = 0;
        for (int sb = 0; sb < es.nsh[eB]; sb++) {
            const int lb = es.l[eB][sb], kb = nsph(lb);
            for (int i = 0; i < ka; i++)
                for (int j = 0; j < kb; j++) {
                    double s = 0.0;
                    for (int k = 0; k < ka; k++)
                        for (int l = 0; l < kb; l++) {
                            if (to_local) {
                                const double d = D[(size_t)(gp.fa + oa + k) * N + gp.fb + ob + l];
                                s += rep_el(la, Rp, Rd, k, i) * d * rep_el(lb, Rp, Rd, l, j);
                            } else {
                                const int r = oa + k, c = ob + l;
                                const double L = same ? 0.5 * ((double)blk[r * nb + c] + (double)blk[c * nb + r])
                                                      : (double)blk[r * nb + c];
                                s += rep_el(la, Rp, Rd, i, k) * L * rep_el(lb, Rp, Rd, j, l);
                            }
                        }
                    if (to_local) {
                        blk[(oa + i) * nb + ob + j] = (float)s;
                    } else {
                        D[(size_t)(gp.fa + oa + i) * N + gp.fb + ob + j] = s;
                        if (!same) D[(size_t)(gp.fb + ob + j) * N + gp.fa + oa + i] = s;
                    }
                }
            ob += kb;
        }
        oa += ka;
    }
}

// D <- D * 2 nocc / tr(D S) for the replicas in mask (one block per replica)
__global__ void electron_scale_kernel(const RepMat* rms, int nrep, double* D, const double* S, const int* mask)
{
    const int r = blockIdx.x;
    if (r >= nrep || (mask && !mask[r])) return;
    const RepMat rm = rms[r];
    __shared__ double red[32];
    __shared__ double fac;
    double s = 0.0;
    for (long long e = threadIdx.x; e < (long long)rm.N * rm.N; e += blockDim.x) s += D[rm.off + e] * S[rm.off + e];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += red[k];
        fac = t > 0.0 ? 2.0 * rm.nocc / t : 1.0;
    }
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)rm.N * rm.N; e += blockDim.x) D[rm.off + e] *= fac;
}

// ---------------------------------------------------------------- BF16 GEMM
// C[M x N] (fp32) = op(A) op(B) on the 5th-generation tensor cores (see
// umma_gemm.cuh); every call of the network has beta = 0. A bounded wait that
// expires sets the per-device flag g_umma_err, checked after each pass.
__device__ int g_umma_err;

static int* umma_err_ptr()
{
    static int* ptr[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return nullptr;
    if (!ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_umma_err) != cudaSuccess) return nullptr;
        ptr[dev] = (int*)p;
    }
    return ptr[dev];
}

static void gemm_bf16(int M, int N, int K, const __nv_bfloat16* A, int lda, int ta, const __nv_bfloat16* B, int ldb,
                      int tb, float* C, int ldc, float beta, cudaStream_t st)
{
    (void)beta;
    if (M <= 0 || N <= 0 || K <= 0) return;
    dim3 grid((N + UMMA_N - 1) / UMMA_N, (M + UMMA_M - 1) / UMMA_M);
    bf16_gemm_tc_kernel<<<grid, 128, 0, st>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, umma_err_ptr());
}

// 0, or PIMD_ETIMEOUT (and the flag cleared) if a GEMM's bounded wait expired
static int umma_status(cudaStream_t st)
{
    int* p = umma_err_ptr();
    if (!p) return PIMD_ECUDA;
    int h = 0;
    if (cudaMemcpyAsync(&h, p, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PIMD_ECUDA;
    if (h) {
        cudaMemsetAsync(p, 0, sizeof(int), st);
        return PIMD_ETIMEOUT;
    }
    return PIMD_OK;
}

static inline dim3 ew(long long n)
{
    return dim3((unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 4096)));
}

// Z += bias (per column); H = SiLU(Z) (act) or Z, in bf16, if H is given
__global__ void bias_act_kernel(float* Z, const float* b, __nv_bfloat16* H, long long n, int cols, int act)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float z = Z[i] + b[i % cols];
        Z[i] = z;
        if (H) H[i] = __float2bfloat16(act ? z / (1.f + expf(-z)) : z);
    }
}

// dZ = dH * SiLU'(Z), SiLU'(z) = s (1 + z (1 - s)), s the logistic function
__global__ void silu_back_kernel(const float* dH, const float* Z, __nv_bfloat16* dZb, float* dZf, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float z = Z[i];
        const float s = 1.f / (1.f + expf(-z));
        const float d = dH[i] * s * (1.f + z * (1.f - s));
        dZf[i] = d;
        dZb[i] = __float2bfloat16(d);
    }
}

// out[c] = sum over rows of A[r][c]; 32 columns per block, 8 row partitions
__global__ void colsum_kernel(const float* A, int rows, int cols, float* out)
{
    const int c = blockIdx.x * 32 + (threadIdx.x & 31);
    const int part = threadIdx.x >> 5, nparts = blockDim.x >> 5;
    __shared__ double red[8][32];
    double s = 0.0;
    if (c < cols)
        for (int r = part; r < rows; r += nparts) s += A[(size_t)r * cols + c];
    red[part][threadIdx.x & 31] = s;
    __syncthreads();
    if (part == 0 && c < cols) {
        double t = 0.0;
        for (int p = 0; p < nparts; p++) t += red[p][threadIdx.x];
        out[c] = (float)t;
    }
}

// MSE with per-row weights: dOut = 2 w (Out - Y) inv_n (bf16 and fp32),
// loss += sum w (Out - Y)^2 inv_n
__global__ void mse_kernel(const float* Out, const float* Y, const float* w, int rows, int cols, double inv_n,
                           __nv_bfloat16* dOb, float* dOf, double* loss)
{
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)rows * cols;
         i += (long long)gridDim.x * blockDim.x) {
        const float ww = w[i / cols];
        const float d = Out[i] - Y[i];
        s += (double)ww * d * d;
        const float gi = (float)(2.0 * inv_n) * ww * d;
        dOf[i] = gi;
        dOb[i] = __float2bfloat16(gi);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(loss, s * inv_n);
}

// Adam (Kingma and Ba): moments m, v with bias corrections c1 = 1 - b1^t, c2 = 1 - b2^t
__global__ void adam_kernel(float* W, const float* g, float* m, float* v, __nv_bfloat16* Wb, long long n, float lr,
                            float b1, float b2, float eps, float c1, float c2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float w = W[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        W[i] = w;
        Wb[i] = __float2bfloat16(w);
    }
}

__global__ void to_bf16_kernel(const float* a, __nv_bfloat16* b, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16(a[i]);
}

// ---------------------------------------------------------------- buffers
struct DevOwned {
    std::vector<void*> owned;
    DevOwned() = default;
    DevOwned(const DevOwned&) = delete;
    DevOwned& operator=(const DevOwned&) = delete;
    ~DevOwned() { release(); }
    void release()
    {
        for (void* p : owned) cudaFree(p);
        owned.clear();
    }
    template <typename T>
    int alloc(T** p, size_t n)
    {
        if (cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return PIMD_ENOMEM;
        }
        owned.push_back(*p);
        return PIMD_OK;
    }
};

#define GK(call)             \
    do {                     \
        int rc_ = (call);    \
        if (rc_) return rc_; \
    } while (0)

// pair rows of a set of replicas, sorted by pair type
struct GuessRows : DevOwned {
    int npair = 0;
    long long nrep = 0;
    std::vector<GuessPair> pairs;
    std::vector<int> type_start;  // [G_NTYPE + 1]
    long long nout = 0;
    double inv_n = 0.0;           // 1 / weighted entries (training rows)
    GuessPair* d_pairs = nullptr;
    __nv_bfloat16* X = nullptr;
    double* frames = nullptr;
    int* within = nullptr;
    float* Y = nullptr;           // targets (training rows)
    float* w = nullptr;           // row weights (training rows)
};

// activations and gradients, shared by all row sets
struct GuessScratch : DevOwned {
    long long cap_rows = 0, cap_out = 0;
    float* Z[G_NLAYER] = {};
    __nv_bfloat16* H[G_NLAYER] = {};
    float* Out = nullptr;
    __nv_bfloat16* dOb = nullptr;
    float* dOf = nullptr;
    float* dH = nullptr;
    __nv_bfloat16* dZb = nullptr;
    float* dZf = nullptr;
    double* d_loss = nullptr;
    int ensure(long long rows, long long nout)
    {
        if (rows <= cap_rows && nout <= cap_out && d_loss) return PIMD_OK;
        release();
        cap_rows = std::max(rows, cap_rows);
        cap_out = std::max(nout, cap_out);
        const size_t nh = (size_t)cap_rows * G_H;
        for (int k = 0; k < G_NLAYER; k++) {
            GK(alloc(&Z[k], nh));
            GK(alloc(&H[k], nh));
        }
        GK(alloc(&Out, cap_out));
        GK(alloc(&dOb, cap_out));
        GK(alloc(&dOf, cap_out));
        GK(alloc(&dH, nh));
        GK(alloc(&dZb, nh));
        GK(alloc(&dZf, nh));
        GK(alloc(&d_loss, 1));
        return PIMD_OK;
    }
};

}  // namespace pimd

using namespace pimd;

struct pimd_guess {
    ElemShells es{};
    int out_dim[G_NTYPE] = {};
    long long woff[G_NLAYER + G_NTYPE] = {}, boff[G_NLAYER + G_NTYPE] = {};
    long long nparam = 0;
    float *W = nullptr, *G = nullptr, *Mo = nullptr, *Vo = nullptr;
    __nv_bfloat16* Wb = nullptr;
    int step = 0;
    int device = 0;
    std::vector<std::unique_ptr<GuessRows>> data;
    long long ndata = 0;
    GuessScratch scr;
};

static int layer_in(int k) { return k == 0 ? G_NF : G_H; }
static int layer_out(const pimd_guess* g, int k) { return k < G_NLAYER ? G_H : g->out_dim[k - G_NLAYER]; }

namespace pimd {

int guess_elem_nbf(const pimd_guess* g, int Z)
{
    const int e = elem_index(Z);
    return (g && e >= 0 && g->es.nsh[e] > 0) ? g->es.nbf[e] : -1;
}

int guess_device(const pimd_guess* g) { return g->device; }

// rows of the replicas with mask[r] != 0 (all if mask is empty): pair list,
// features, frames and cutoff flags
static int rows_setup(const pimd_guess* g, GuessRows& wk, int nrep, const int* natom_of, const int* Zc,
                      const std::vector<int>& atom_f0, const std::vector<int>& mask, const double* d_xyz,
                      const int* d_Z, const int* d_atom0, cudaStream_t st)
{
    std::vector<std::vector<GuessPair>> by(G_NTYPE);
    int a0 = 0;
    wk.nrep = 0;
    for (int r = 0; r < nrep; r++) {
        if (mask.empty() || mask[r]) {
            wk.nrep++;
            for (int i = 0; i < natom_of[r]; i++)
                for (int j = i; j < natom_of[r]; j++) {
                    int A = a0 + i, B = a0 + j;
                    int eA = elem_index(Zc[A]), eB = elem_index(Zc[B]);
                    if (eA < 0 || eB < 0 || g->es.nsh[eA] == 0 || g->es.nsh[eB] == 0) return PIMD_EINVAL;
                    if (eB > eA) {
                        std::swap(A, B);
                        std::swap(eA, eB);
                    }
                    const int t = pair_type(eA, eB, A == B);
                    by[t].push_back(GuessPair{r, A, B, t, atom_f0[A], atom_f0[B], 0});
                }
        }
        a0 += natom_of[r];
    }
    wk.type_start.assign(G_NTYPE + 1, 0);
    wk.pairs.clear();
    long long off = 0;
    for (int t = 0; t < G_NTYPE; t++) {
        wk.type_start[t] = (int)wk.pairs.size();
        for (auto& p : by[t]) {
            p.out_off = off;
            off += g->out_dim[t];
            wk.pairs.push_back(p);
        }
    }
    wk.type_start[G_NTYPE] = (int)wk.pairs.size();
    wk.npair = (int)wk.pairs.size();
    wk.nout = off;
    const int n = wk.npair;
    GK(wk.alloc(&wk.d_pairs, n));
    GK(wk.alloc(&wk.X, (size_t)n * G_NF));
    GK(wk.alloc(&wk.frames, (size_t)n * 9));
    GK(wk.alloc(&wk.within, n));
    if (n == 0) return PIMD_OK;
    if (cudaMemcpyAsync(wk.d_pairs, wk.pairs.data(), sizeof(GuessPair) * n, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return PIMD_ECUDA;
    featurize_kernel<<<(n + 127) / 128, 128, 0, st>>>(wk.d_pairs, n, d_xyz, d_Z, d_atom0, wk.X, nullptr, wk.frames,
                                                      wk.within);
    return cudaGetLastError() == cudaSuccess ? PIMD_OK : PIMD_ECUDA;
}

}  // namespace pimd

// forward pass: hidden layers over all rows, then each type's head into s.Out
static void guess_forward(const pimd_guess* g, const GuessRows& wk, GuessScratch& s, cudaStream_t st)
{
    const int n = wk.npair;
    const __nv_bfloat16* in = wk.X;
    for (int k = 0; k < G_NLAYER; k++) {
        const int fi = layer_in(k);
        gemm_bf16(n, G_H, fi, in, fi, 0, g->Wb + g->woff[k], G_H, 0, s.Z[k], G_H, 0.f, st);
        bias_act_kernel<<<ew((long long)n * G_H), 256, 0, st>>>(s.Z[k], g->W + g->boff[k], s.H[k], (long long)n * G_H,
                                                               G_H, 1);
        in = s.H[k];
    }
    for (int t = 0; t < G_NTYPE; t++) {
        const int r0 = wk.type_start[t], nr = wk.type_start[t + 1] - r0;
        if (nr == 0) continue;
        const int od = g->out_dim[t];
        float* out = s.Out + wk.pairs[r0].out_off;
        gemm_bf16(nr, od, G_H, s.H[G_NLAYER - 1] + (size_t)r0 * G_H, G_H, 0, g->Wb + g->woff[G_NLAYER + t], od, 0, out,
                  od, 0.f, st);
        bias_act_kernel<<<ew((long long)nr * od), 256, 0, st>>>(out, g->W + g->boff[G_NLAYER + t], nullptr,
                                                               (long long)nr * od, od, 0);
    }
}

// loss (into s.d_loss) and its gradient with respect to every parameter (g->G)
static int guess_backward(pimd_guess* g, const GuessRows& wk, GuessScratch& s, cudaStream_t st)
{
    const int n = wk.npair;
    cudaMemsetAsync(s.d_loss, 0, sizeof(double), st);
    cudaMemsetAsync(g->G, 0, sizeof(float) * g->nparam, st);
    cudaMemsetAsync(s.dH, 0, sizeof(float) * (size_t)n * G_H, st);
    for (int t = 0; t < G_NTYPE; t++) {
        const int r0 = wk.type_start[t], nr = wk.type_start[t + 1] - r0;
        if (nr == 0) continue;
        const int od = g->out_dim[t];
        const long long o = wk.pairs[r0].out_off;
        mse_kernel<<<ew((long long)nr * od), 256, 0, st>>>(s.Out + o, wk.Y + o, wk.w + r0, nr, od, wk.inv_n, s.dOb + o,
                                                          s.dOf + o, s.d_loss);
        // head: dW = H^T dOut, db = column sums of dOut, dH = dOut W^T
        gemm_bf16(G_H, od, nr, s.H[G_NLAYER - 1] + (size_t)r0 * G_H, G_H, 1, s.dOb + o, od, 0,
                  g->G + g->woff[G_NLAYER + t], od, 0.f, st);
        colsum_kernel<<<(od + 31) / 32, 256, 0, st>>>(s.dOf + o, nr, od, g->G + g->boff[G_NLAYER + t]);
        gemm_bf16(nr, G_H, od, s.dOb + o, od, 0, g->Wb + g->woff[G_NLAYER + t], od, 1, s.dH + (size_t)r0 * G_H, G_H,
                  0.f, st);
    }
    for (int k = G_NLAYER - 1; k >= 0; k--) {
        silu_back_kernel<<<ew((long long)n * G_H), 256, 0, st>>>(s.dH, s.Z[k], s.dZb, s.dZf, (long long)n * G_H);
        const int fi = layer_in(k);
        const __nv_bfloat16* in = k == 0 ? wk.X : s.H[k - 1];
        gemm_bf16(fi, G_H, n, in, fi, 1, s.dZb, G_H, 0, g->G + g->woff[k], G_H, 0.f, st);
        colsum_kernel<<<G_H / 32, 256, 0, st>>>(s.dZf, n, G_H, g->G + g->boff[k]);
        if (k > 0) gemm_bf16(n, fi, G_H, s.dZb, G_H, 0, g->Wb + g->woff[k], G_H, 1, s.dH, G_H, 0.f, st);
    }
    return cudaGetLastError() == cudaSuccess ? PIMD_OK : PIMD_ECUDA;
}

static void guess_adam(pimd_guess* g, float lr, cudaStream_t st)
{
    g->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    adam_kernel<<<ew(g->nparam), 256, 0, st>>>(g->W, g->G, g->Mo, g->Vo, g->Wb, g->nparam, lr, b1, b2, 1e-8f,
                                               1.f - powf(b1, (float)g->step), 1.f - powf(b2, (float)g->step));
}

extern "C" void pimd_guess_destroy(pimd_guess* g)
{
    if (!g) return;
    cudaFree(g->W);
    cudaFree(g->G);
    cudaFree(g->Mo);
    cudaFree(g->Vo);
    cudaFree(g->Wb);
    delete g;
}

extern "C" int pimd_guess_create(pimd_guess** out, const pimd_basis* basis, unsigned long long seed)
{
    if (!out || !basis) return PIMD_EINVAL;
    *out = nullptr;
    std::unique_ptr<pimd_guess> g(new pimd_guess());
    if (cudaGetDevice(&g->device) != cudaSuccess) return PIMD_ECUDA;
    const int Zs[3] = {1, 6, 8};
    for (int e = 0; e < 3; e++) {
        int ls[64];
        const int ns = basis_elem_shells(basis, Zs[e], ls, 64);
        g->es.nsh[e] = 0;
        g->es.nbf[e] = 0;
        if (ns <= 0) continue;
        if (ns > G_MAXSH) return PIMD_EINVAL;
        g->es.nsh[e] = ns;
        for (int s = 0; s < ns; s++) {
            g->es.l[e][s] = ls[s];
            g->es.nbf[e] += nsph(ls[s]);
        }
        if (g->es.nbf[e] > G_MAXBF) return PIMD_EINVAL;
    }
    if (g->es.nsh[0] + g->es.nsh[1] + g->es.nsh[2] == 0) return PIMD_EINVAL;
    for (int t = 0; t < G_NTYPE; t++) {
        static const int pa[G_NTYPE][2] = {{0, 0}, {1, 1}, {2, 2}, {2, 2}, {2, 1}, {2, 0}, {1, 1}, {1, 0}, {0, 0}};
        g->out_dim[t] = std::max(1, g->es.nbf[pa[t][0]] * g->es.nbf[pa[t][1]]);
    }
    long long o = 0;
    for (int k = 0; k < G_NLAYER + G_NTYPE; k++) {
        g->woff[k] = o;
        o += (long long)layer_in(k) * layer_out(g.get(), k);
        g->boff[k] = o;
        o += layer_out(g.get(), k);
    }
    g->nparam = o;
    // W ~ U(-a, a), a = sqrt(6 / (fan_in + fan_out)) (Glorot), heads scaled by
    // 0.1; biases 0; uniform numbers from a 64-bit linear congruential stream
    std::vector<float> h(o, 0.f);
    uint64_t s = seed * 6364136223846793005ull + 1442695040888963407ull;
    auto rnd = [&]() {
        s = s * 6364136223846793005ull + 1442695040888963407ull;
        return (double)(s >> 11) / 9007199254740992.0;
    };
    for (int k = 0; k < G_NLAYER + G_NTYPE; k++) {
        const int fi = layer_in(k), fo = layer_out(g.get(), k);
        const double a = sqrt(6.0 / (fi + fo)) * (k >= G_NLAYER ? 0.1 : 1.0);
        for (long long i = 0; i < (long long)fi * fo; i++) h[g->woff[k] + i] = (float)((2.0 * rnd() - 1.0) * a);
    }
    if (cudaMalloc(&g->W, sizeof(float) * o) != cudaSuccess || cudaMalloc(&g->G, sizeof(float) * o) != cudaSuccess ||
        cudaMalloc(&g->Mo, sizeof(float) * o) != cudaSuccess || cudaMalloc(&g->Vo, sizeof(float) * o) != cudaSuccess ||
        cudaMalloc(&g->Wb, sizeof(__nv_bfloat16) * o) != cudaSuccess) {
        cudaGetLastError();
        pimd_guess_destroy(g.release());
        return PIMD_ENOMEM;
    }
    cudaMemcpy(g->W, h.data(), sizeof(float) * o, cudaMemcpyHostToDevice);
    cudaMemset(g->Mo, 0, sizeof(float) * o);
    cudaMemset(g->Vo, 0, sizeof(float) * o);
    to_bf16_kernel<<<ew(o), 256>>>(g->W, g->Wb, o);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        pimd_guess_destroy(g.release());
        return PIMD_ECUDA;
    }
    *out = g.release();
    return PIMD_OK;
}

extern "C" long long pimd_guess_nparam(const pimd_guess* g) { return g ? g->nparam : -1; }
extern "C" long long pimd_guess_ndata(const pimd_guess* g) { return g ? g->ndata : -1; }
extern "C" void pimd_guess_clear_data(pimd_guess* g)
{
    if (!g) return;
    g->data.clear();
    g->ndata = 0;
}

namespace pimd {

// converged densities d_D of nrep replicas -> one training row set
int guess_collect_device(pimd_guess* g, int nrep, const int* natom_of, const int* Zc,
                         const std::vector<int>& atom_f0, const double* d_xyz, const int* d_Z, const int* d_atom0,
                         const RepMat* d_rm, double* d_D, cudaStream_t st)
{
    std::unique_ptr<GuessRows> wk(new GuessRows());
    GK(rows_setup(g, *wk, nrep, natom_of, Zc, atom_f0, {}, d_xyz, d_Z, d_atom0, st));
    const int n = wk->npair;
    GK(wk->alloc(&wk->Y, wk->nout));
    GK(wk->alloc(&wk->w, n));
    if (n > 0)
        block_rotate_kernel<<<(n + 63) / 64, 64, 0, st>>>(wk->d_pairs, n, wk->frames, g->es, d_Z, d_rm, d_D, wk->Y,
                                                           wk->within, 1);
    std::vector<int> within(n);
    if (n > 0 && cudaMemcpyAsync(within.data(), wk->within, sizeof(int) * n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return PIMD_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return PIMD_ECUDA;
    std::vector<float> w(n);
    long long nent = 0;
    for (int i = 0; i < n; i++) {
        w[i] = within[i] ? 1.f : 0.f;
        if (within[i]) nent += g->out_dim[wk->pairs[i].type];
    }
    wk->inv_n = 1.0 / (double)std::max<long long>(nent, 1);
    if (n > 0 && cudaMemcpyAsync(wk->w, w.data(), sizeof(float) * n, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return PIMD_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return PIMD_ECUDA;
    g->ndata += wk->nrep;
    g->data.push_back(std::move(wk));
    return PIMD_OK;
}

// predicted densities of the replicas in mask into d_D (through d_tmp, mtot
// doubles of scratch), scaled to tr(D S) = number of electrons
int guess_predict_device(pimd_guess* g, int nrep, const int* natom_of, const int* Zc,
                         const std::vector<int>& atom_f0, const std::vector<int>& mask, const double* d_xyz,
                         const int* d_Z, const int* d_atom0, const RepMat* d_rm, const int* d_mask, const double* d_S,
                         double* d_tmp, long long mtot, double* d_D, cudaStream_t st)
{
    GuessRows wk;
    GK(rows_setup(g, wk, nrep, natom_of, Zc, atom_f0, mask, d_xyz, d_Z, d_atom0, st));
    GK(g->scr.ensure(wk.npair, wk.nout));
    if (cudaMemsetAsync(d_tmp, 0, sizeof(double) * mtot, st) != cudaSuccess) return PIMD_ECUDA;
    if (wk.npair > 0) {
        guess_forward(g, wk, g->scr, st);
        block_rotate_kernel<<<(wk.npair + 63) / 64, 64, 0, st>>>(wk.d_pairs, wk.npair, wk.frames, g->es, d_Z, d_rm,
                                                                  d_tmp, g->scr.Out, wk.within, 0);
    }
    electron_scale_kernel<<<nrep, 256, 0, st>>>(d_rm, nrep, d_tmp, d_S, d_mask);
    launch_copy_mats(d_rm, nrep, d_tmp, d_D, d_mask, st);
    // the row set is freed on return: wait for the kernels that read it
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return PIMD_ECUDA;
    return umma_status(st);
}

}  // namespace pimd

// one pass over the training set: per row set a forward and backward pass
// and (update) an Adam step; *loss = replica-weighted mean of the losses
static int guess_pass(pimd_guess* g, int update, float lr, double* loss)
{
    cudaStream_t st = 0;
    double tot = 0.0;
    long long rows = 0, outs = 0;
    for (auto& d : g->data) {
        rows = std::max<long long>(rows, d->npair);
        outs = std::max<long long>(outs, d->nout);
    }
    GK(g->scr.ensure(rows, outs));
    for (auto& d : g->data) {
        if (d->npair == 0) continue;
        guess_forward(g, *d, g->scr, st);
        GK(guess_backward(g, *d, g->scr, st));
        double l = 0.0;
        if (cudaMemcpyAsync(&l, g->scr.d_loss, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return PIMD_ECUDA;
        if (update) guess_adam(g, lr, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return PIMD_ECUDA;
        tot += l * (double)d->nrep;
    }
    if (loss) *loss = g->ndata > 0 ? tot / (double)g->ndata : 0.0;
    if (cudaGetLastError() != cudaSuccess) return PIMD_ECUDA;
    return umma_status(st);
}

extern "C" int pimd_guess_train(pimd_guess* g, int epochs, double lr, double* loss_history)
{
    if (!g || epochs < 0 || !(lr > 0) || g->data.empty()) return PIMD_EINVAL;
    if (cudaSetDevice(g->device) != cudaSuccess) return PIMD_ECUDA;
    for (int ep = 0; ep < epochs; ep++) {
        double l = 0.0;
        GK(guess_pass(g, 1, (float)lr, &l));
        if (loss_history) loss_history[ep] = l;
    }
    return PIMD_OK;
}

extern "C" int pimd_guess_loss(pimd_guess* g, double* loss)
{
    if (!g || !loss || g->data.empty()) return PIMD_EINVAL;
    if (cudaSetDevice(g->device) != cudaSuccess) return PIMD_ECUDA;
    return guess_pass(g, 0, 0.f, loss);
}

// ---------------------------------------------------------------- test hooks
extern "C" int pimd_guess_mlp_grad(pimd_guess* g, int n, int type, const float* X, const float* Y, double* loss,
                                   float* params_out, float* grads_out)
{
    if (!g || n <= 0 || type < 0 || type >= G_NTYPE || !X || !Y || !loss) return PIMD_EINVAL;
    if (cudaSetDevice(g->device) != cudaSuccess) return PIMD_ECUDA;
    cudaStream_t st = 0;
    GuessRows wk;
    wk.npair = n;
    wk.nrep = 1;
    wk.type_start.assign(G_NTYPE + 1, 0);
    for (int t = type + 1; t <= G_NTYPE; t++) wk.type_start[t] = n;
    wk.pairs.assign(n, GuessPair{0, 0, 0, type, 0, 0, 0});
    for (int i = 0; i < n; i++) wk.pairs[i].out_off = (long long)i * g->out_dim[type];
    wk.nout = (long long)n * g->out_dim[type];
    wk.inv_n = 1.0 / (double)wk.nout;
    float* Xf;
    GK(wk.alloc(&Xf, (size_t)n * G_NF));
    GK(wk.alloc(&wk.X, (size_t)n * G_NF));
    GK(wk.alloc(&wk.Y, wk.nout));
    GK(wk.alloc(&wk.w, n));
    GuessScratch s;
    GK(s.ensure(n, wk.nout));
    cudaMemcpy(Xf, X, sizeof(float) * n * G_NF, cudaMemcpyHostToDevice);
    to_bf16_kernel<<<ew((long long)n * G_NF), 256>>>(Xf, wk.X, (long long)n * G_NF);
    cudaMemcpy(wk.Y, Y, sizeof(float) * wk.nout, cudaMemcpyHostToDevice);
    std::vector<float> w(n, 1.f);
    cudaMemcpy(wk.w, w.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
    guess_forward(g, wk, s, st);
    GK(guess_backward(g, wk, s, st));
    if (cudaDeviceSynchronize() != cudaSuccess) return PIMD_ECUDA;
    GK(umma_status(st));
    cudaMemcpy(loss, s.d_loss, sizeof(double), cudaMemcpyDeviceToHost);
    if (params_out) cudaMemcpy(params_out, g->W, sizeof(float) * g->nparam, cudaMemcpyDeviceToHost);
    if (grads_out) cudaMemcpy(grads_out, g->G, sizeof(float) * g->nparam, cudaMemcpyDeviceToHost);
    return cudaGetLastError() == cudaSuccess ? PIMD_OK : PIMD_ECUDA;
}

extern "C" int pimd_guess_pair_data(pimd_guess* g, int natom, const int* Z, const double* coords, const double* D,
                                    const float* local_in, int npair_max, long long nout_max, int* npair_out,
                                    int* pair_AB, long long* block_off, float* feats, double* frames,
                                    float* local_out, double* D_out)
{
    if (!g || natom <= 0 || !Z || !coords || !npair_out) return PIMD_EINVAL;
    if (cudaSetDevice(g->device) != cudaSuccess) return PIMD_ECUDA;
    cudaStream_t st = 0;
    std::vector<int> atom_f0(natom);
    int N = 0, nel = 0;
    for (int i = 0; i < natom; i++) {
        const int nb = guess_elem_nbf(g, Z[i]);
        if (nb < 0) return PIMD_EINVAL;
        atom_f0[i] = N;
        N += nb;
        nel += Z[i];
    }
    DevOwned mem;
    double *d_xyz, *d_D;
    int *d_Z, *d_atom0;
    RepMat* d_rm;
    GK(mem.alloc(&d_xyz, (size_t)natom * 3));
    GK(mem.alloc(&d_Z, natom));
    GK(mem.alloc(&d_atom0, 2));
    GK(mem.alloc(&d_rm, 1));
    GK(mem.alloc(&d_D, (size_t)N * N));
    const int atom0[2] = {0, natom};
    const RepMat rm{N, nel / 2, 0};
    cudaMemcpy(d_xyz, coords, sizeof(double) * natom * 3, cudaMemcpyHostToDevice);
    cudaMemcpy(d_Z, Z, sizeof(int) * natom, cudaMemcpyHostToDevice);
    cudaMemcpy(d_atom0, atom0, sizeof(atom0), cudaMemcpyHostToDevice);
    cudaMemcpy(d_rm, &rm, sizeof(rm), cudaMemcpyHostToDevice);
    GuessRows wk;
    GK(rows_setup(g, wk, 1, &natom, Z, atom_f0, {}, d_xyz, d_Z, d_atom0, st));
    *npair_out = wk.npair;
    if (wk.npair > npair_max || wk.nout > nout_max) return PIMD_EINVAL;
    const int n = wk.npair;
    float *Xf, *blk;
    GK(mem.alloc(&Xf, (size_t)n * G_NF));
    GK(mem.alloc(&blk, wk.nout));
    featurize_kernel<<<(n + 127) / 128, 128, 0, st>>>(wk.d_pairs, n, d_xyz, d_Z, d_atom0, wk.X, Xf, wk.frames,
                                                      wk.within);
    if (D && local_out) {
        cudaMemcpy(d_D, D, sizeof(double) * N * N, cudaMemcpyHostToDevice);
        block_rotate_kernel<<<(n + 63) / 64, 64, 0, st>>>(wk.d_pairs, n, wk.frames, g->es, d_Z, d_rm, d_D, blk,
                                                           wk.within, 1);
        cudaMemcpy(local_out, blk, sizeof(float) * wk.nout, cudaMemcpyDeviceToHost);
    }
    if (local_in && D_out) {
        cudaMemset(d_D, 0, sizeof(double) * N * N);
        cudaMemcpy(blk, local_in, sizeof(float) * wk.nout, cudaMemcpyHostToDevice);
        block_rotate_kernel<<<(n + 63) / 64, 64, 0, st>>>(wk.d_pairs, n, wk.frames, g->es, d_Z, d_rm, d_D, blk,
                                                           wk.within, 0);
        cudaMemcpy(D_out, d_D, sizeof(double) * N * N, cudaMemcpyDeviceToHost);
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return PIMD_ECUDA;
    for (int i = 0; i < n; i++) {
        if (pair_AB) {
            pair_AB[2 * i] = wk.pairs[i].A;
            pair_AB[2 * i + 1] = wk.pairs[i].B;
        }
        if (block_off) block_off[i] = wk.pairs[i].out_off;
    }
    if (feats) cudaMemcpy(feats, Xf, sizeof(float) * (size_t)n * G_NF, cudaMemcpyDeviceToHost);
    if (frames) cudaMemcpy(frames, wk.frames, sizeof(double) * (size_t)n * 9, cudaMemcpyDeviceToHost);
    return cudaGetLastError() == cudaSuccess ? PIMD_OK : PIMD_ECUDA;
}

// BF16 GEMM test hook (the network's tensor-core GEMM alone)
extern "C" int pimd_bf16_gemm_dev(int M, int N, int K, const void* A, int lda, int ta, const void* B, int ldb, int tb,
                                  float* C, int ldc, void* stream)
{
    if (M <= 0 || N <= 0 || K <= 0 || !A || !B || !C) return PIMD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    gemm_bf16(M, N, K, (const __nv_bfloat16*)A, lda, ta, (const __nv_bfloat16*)B, ldb, tb, C, ldc, 0.f, st);
    if (cudaGetLastError() != cudaSuccess) return PIMD_ECUDA;
    return umma_status(st);
}

// ---------------------------------------------------------------- save / load
extern "C" int pimd_guess_save(const pimd_guess* g, const char* path)
{
    if (!g || !path) return PIMD_EINVAL;
    std::vector<float> h(g->nparam);
    if (cudaMemcpy(h.data(), g->W, sizeof(float) * g->nparam, cudaMemcpyDeviceToHost) != cudaSuccess) return PIMD_ECUDA;
    FILE* f = fopen(path, "wb");
    if (!f) return PIMD_EINVAL;
    const char magic[8] = {'P', 'I', 'M', 'D', 'G', 'S', '0', '1'};
    const long long n = g->nparam;
    bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(&n, sizeof(n), 1, f) == 1 &&
              fwrite(g->out_dim, sizeof(int), G_NTYPE, f) == (size_t)G_NTYPE &&
              fwrite(h.data(), sizeof(float), n, f) == (size_t)n;
    ok = (fclose(f) == 0) && ok;
    return ok ? PIMD_OK : PIMD_EINVAL;
}

extern "C" int pimd_guess_load(pimd_guess* g, const char* path)
{
    if (!g || !path) return PIMD_EINVAL;
    FILE* f = fopen(path, "rb");
    if (!f) return PIMD_EINVAL;
    char magic[8];
    long long n = 0;
    int od[G_NTYPE];
    std::vector<float> h;
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "PIMDGS01", 8) == 0 && fread(&n, sizeof(n), 1, f) == 1 &&
              n == g->nparam && fread(od, sizeof(int), G_NTYPE, f) == (size_t)G_NTYPE &&
              memcmp(od, g->out_dim, sizeof(od)) == 0;
    if (ok) {
        h.resize(n);
        ok = fread(h.data(), sizeof(float), n, f) == (size_t)n;
    }
    fclose(f);
    if (!ok) return PIMD_EINVAL;
    if (cudaSetDevice(g->device) != cudaSuccess) return PIMD_ECUDA;
    cudaMemcpy(g->W, h.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
    cudaMemset(g->Mo, 0, sizeof(float) * n);
    cudaMemset(g->Vo, 0, sizeof(float) * n);
    g->step = 0;
    to_bf16_kernel<<<ew(n), 256>>>(g->W, g->Wb, n);
    return cudaDeviceSynchronize() == cudaSuccess ? PIMD_OK : PIMD_ECUDA;
}
