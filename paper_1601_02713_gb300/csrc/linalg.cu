// Dense per-replica linear algebra of the SCF in FP64: batched GEMM, a
// batched one-sided (Hestenes) Jacobi eigensolver, Pulay DIIS, and the small
// element-wise / reduction steps (Fock assembly, energy, commutator norm).
// Every kernel covers all replicas of a call in one launch; replicas whose
// SCF has finished are skipped through the active mask.
#include <math.h>

#include <algorithm>

#include <cooperative_groups.h>

#include "internal.h"
#include "pimdgb.h"

namespace cg = cooperative_groups;

namespace pimd {

namespace {

// C = alpha op(A) op(B) + beta C, row-major; op(X) = X or X^T. 64x64 tiles,
// 256 threads, 4x4 outputs per thread. grid = (tilesN, tilesM, ndesc).
constexpr int TB = 64, TK = 16;

__global__ void __launch_bounds__(256) gemm_kernel(const GemmDesc* __restrict__ descs, const int* active)
{
    const GemmDesc d = descs[blockIdx.z];
    if (d.rep >= 0 && active && !active[d.rep]) return;
    const int m0 = blockIdx.y * TB, n0 = blockIdx.x * TB;
    if (m0 >= d.M || n0 >= d.N) return;
    __shared__ double As[TK][TB + 1];
    __shared__ double Bs[TK][TB + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < d.K; k0 += TK) {
        for (int e = threadIdx.x; e < TK * TB; e += 256) {
            const int kk = e / TB, mm = e % TB;
            const int m = m0 + mm, k = k0 + kk;
            double va = 0.0;
            if (m < d.M && k < d.K) va = d.ta ? d.A[(size_t)k * d.lda + m] : d.A[(size_t)m * d.lda + k];
            As[kk][mm] = va;
            const int n = n0 + mm;
            double vb = 0.0;
            if (n < d.N && k < d.K) vb = d.tb ? d.B[(size_t)n * d.ldb + k] : d.B[(size_t)k * d.ldb + n];
            Bs[kk][mm] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; kk++) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int m = m0 + ty * 4 + i;
        if (m >= d.M) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int n = n0 + tx * 4 + j;
            if (n >= d.N) continue;
            double* c = d.C + (size_t)m * d.ldc + n;
            *c = d.alpha * acc[i][j] + (d.beta != 0.0 ? d.beta * *c : 0.0);
        }
    }
}

// ---------------------------------------------------------------------------
// One-sided Jacobi (Hestenes): the columns of G = A + sigma I (SPD) are
// rotated pairwise until mutually orthogonal; then G = V diag(lambda + sigma)
// and each eigenvector is a normalised column. Pairs follow the round-robin
// (circle) schedule, n/2 disjoint pairs per round handled by the warps of one
// block per replica. For each pair (p, q): alpha = |g_p|^2, beta = |g_q|^2,
// gamma = g_p . g_q; zeta = (beta - alpha) / (2 gamma),
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1 + t^2), s = c t,
// g_p <- c g_p - s g_q, g_q <- s g_p + c g_q.
// ---------------------------------------------------------------------------
constexpr int JAC_THREADS = 512;
constexpr int JAC_PER = 24;   // largest column length per lane: n <= 768
constexpr int JAC_MAXSWEEP = 60;
constexpr int JAC_CLUSTER = 8;   // CTAs (SMs) per matrix of 128 or more rows

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// PER = column elements held per lane (n <= 32 PER): the kernel is FP64-bound,
// so PER is the smallest instantiated length that fits the batch's largest
// matrix (padding lanes would be FP64 work on zeros).
// CS = CTAs per matrix: 1, or a thread-block cluster of CS CTAs on CS SMs.
// The n/2 column pairs of a round are independent, so the CTAs of the
// cluster split every round and meet at a cluster barrier (hardware, no spin)
// after it; the columns live in global memory (L2), each written by one CTA
// per round. Every CTA computes the shift and the column norms of the
// eigenvalue step itself (O(n^2), small); the rotation flag of a sweep is
// or-ed into CTA 0's shared memory (distributed shared memory).
// notconv (may be NULL): notconv[r] = 1 when matrix r is still rotating after
// JAC_MAXSWEEP sweeps (its eigenpairs are then not converged)
template <int CS>
__device__ __forceinline__ void jac_cluster_sync()
{
    if constexpr (CS > 1) {
        __threadfence();
        cg::this_cluster().sync();
    } else {
        __syncthreads();
    }
}

template <int PER, int CS>
__global__ void __launch_bounds__(JAC_THREADS) jacobi_kernel(const RepMat* __restrict__ rms, const double* A,
                                                             double* V, double* evals, int ldE, double* work,
                                                             const int* active, int shift_to_spd, int* notconv)
{
    const int r = blockIdx.x / CS, cr = blockIdx.x % CS;
    if (active && !active[r]) return;   // the whole cluster (one matrix) leaves together
    const RepMat rm = rms[r];
    const int n = rm.N;
    if (n == 0) return;
    const double* a = A + rm.off;
    double* G = work + rm.off;     // column-major: G[col * n + row]
    double* v = V + rm.off;
    double* ev = evals + (size_t)r * ldE;
    __shared__ double s_red[JAC_THREADS / 32];
    __shared__ double s_shift;
    __shared__ int s_rot[3];       // CTA 0's copy: rotation flags of sweeps s mod 3
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = JAC_THREADS / 32;
    int* rot0 = s_rot;             // CTA 0's flags
    if constexpr (CS > 1) rot0 = cg::this_cluster().map_shared_rank(s_rot, 0);
    // Gershgorin lower bound for the shift
    double lo = 1e300;
    for (int i = threadIdx.x; i < n; i += JAC_THREADS) {
        double off = 0.0;
        for (int j = 0; j < n; j++)
            if (j != i) off += fabs(a[(size_t)i * n + j]);
        lo = fmin(lo, a[(size_t)i * n + i] - off);
    }
    for (int o = 16; o > 0; o >>= 1) lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    if (lane == 0) s_red[warp] = lo;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 1e300;
        for (int w = 0; w < nw; w++) m = fmin(m, s_red[w]);
        s_shift = shift_to_spd ? (m < 1.0 ? 1.0 - m : 0.0) : 0.0;
        s_rot[0] = s_rot[1] = s_rot[2] = 0;
    }
    __syncthreads();
    const double shift = s_shift;
    for (int e = cr * JAC_THREADS + threadIdx.x; e < n * n; e += CS * JAC_THREADS) {
        const int i = e / n, j = e % n;
        G[(size_t)j * n + i] = a[e] + (i == j ? shift : 0.0);
    }
    jac_cluster_sync<CS>();
    const int M = (n + 1) & ~1;  // even number of players; index n is a dummy when n is odd
    const double tol = 4e-16 * (n > 8 ? n : 8);
    bool settled = false;
    for (int sweep = 0; sweep < JAC_MAXSWEEP; sweep++) {
        // the next sweep's flag is cleared now: it was last read at the end of
        // sweep - 2, and every CTA has passed a barrier of sweep - 1 since
        if (cr == 0 && threadIdx.x == 0) s_rot[(sweep + 1) % 3] = 0;
        int rotated = 0;
        for (int rd = 0; rd < M - 1; rd++) {
            for (int k = warp * CS + cr; k < M / 2; k += nw * CS) {
                int p, q;
                if (k == 0) {
                    p = rd;
                    q = M - 1;
                } else {
                    p = (rd + k) % (M - 1);
                    q = (rd - k + (M - 1)) % (M - 1);
                }
                if (p >= n || q >= n) continue;
                double* gp = G + (size_t)p * n;
                double* gq = G + (size_t)q * n;
                // both columns in registers (all loads in flight at once)
                double x[PER], y[PER];
#pragma unroll
                for (int k = 0; k < PER; k++) {
                    const int i = lane + 32 * k;
                    x[k] = i < n ? gp[i] : 0.0;
                    y[k] = i < n ? gq[i] : 0.0;
                }
                double al = 0.0, be = 0.0, ga = 0.0;
#pragma unroll
                for (int k = 0; k < PER; k++) {
                    al = fma(x[k], x[k], al);
                    be = fma(y[k], y[k], be);
                    ga = fma(x[k], y[k], ga);
                }
                al = warp_sum(al);
                be = warp_sum(be);
                ga = warp_sum(ga);
                if (fabs(ga) > tol * sqrt(al * be) && ga != 0.0) {
                    rotated = 1;
                    const double zeta = (be - al) / (2.0 * ga);
                    const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
#pragma unroll
                    for (int k = 0; k < PER; k++) {
                        const int i = lane + 32 * k;
                        if (i < n) {
                            gp[i] = c * x[k] - s * y[k];
                            gq[i] = s * x[k] + c * y[k];
                        }
                    }
                }
            }
            jac_cluster_sync<CS>();
        }
        if (rotated && lane == 0) atomicOr(rot0 + sweep % 3, 1);
        jac_cluster_sync<CS>();
        if (!*(volatile int*)(rot0 + sweep % 3)) {
            settled = true;
            break;
        }
    }
    if (!settled && notconv && cr == 0 && threadIdx.x == 0) notconv[r] = 1;
    // eigenvalues (column norms minus the shift), ascending order by rank;
    // every CTA has all norms, each writes its share of the vectors
    extern __shared__ double s_lam[];
    for (int j = threadIdx.x; j < n; j += JAC_THREADS) {
        double nn = 0.0;
        for (int i = 0; i < n; i++) nn += G[(size_t)j * n + i] * G[(size_t)j * n + i];
        s_lam[j] = sqrt(nn);
    }
    __syncthreads();
    for (int j = cr * JAC_THREADS + threadIdx.x; j < n; j += CS * JAC_THREADS) {
        const double lj = s_lam[j];
        int rank = 0;
        for (int k = 0; k < n; k++) {
            const double lk = s_lam[k];
            rank += (lk < lj) || (lk == lj && k < j);
        }
        ev[rank] = lj - shift;
        const double inv = lj > 0.0 ? 1.0 / lj : 0.0;
        for (int i = 0; i < n; i++) v[(size_t)i * n + rank] = G[(size_t)j * n + i] * inv;
    }
    // no CTA of the cluster may leave while another can still address its
    // shared memory (the flag reads above)
    if constexpr (CS > 1) cg::this_cluster().sync();
}

template <int PER>
static void jacobi_launch(int nmat, cudaStream_t st, size_t sm, const RepMat* rm, const double* A, double* V,
                          double* evals, int ldE, double* work, const int* active, int shift, int* notconv)
{
    // matrices of 128 or more rows: a cluster of JAC_CLUSTER CTAs (SMs) each
    if (PER >= 4) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(nmat * JAC_CLUSTER);
        cfg.blockDim = dim3(JAC_THREADS);
        cfg.dynamicSmemBytes = sm;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = JAC_CLUSTER;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, jacobi_kernel<PER, JAC_CLUSTER>, rm, A, V, evals, ldE, work, active, shift,
                           notconv);
    } else {
        jacobi_kernel<PER, 1><<<nmat, JAC_THREADS, sm, st>>>(rm, A, V, evals, ldE, work, active, shift, notconv);
    }
}

// one block (or cluster) per matrix; nmax = the largest n of the batch (<= 32 JAC_PER)
static void jacobi_dispatch(int nmat, int nmax, cudaStream_t st, const RepMat* rm, const double* A, double* V,
                            double* evals, int ldE, double* work, const int* active, int shift, int* notconv)
{
    const size_t sm = sizeof(double) * nmax;
    if (nmax <= 32 * 2)
        jacobi_launch<2>(nmat, st, sm, rm, A, V, evals, ldE, work, active, shift, notconv);
    else if (nmax <= 32 * 4)
        jacobi_launch<4>(nmat, st, sm, rm, A, V, evals, ldE, work, active, shift, notconv);
    else if (nmax <= 32 * 6)
        jacobi_launch<6>(nmat, st, sm, rm, A, V, evals, ldE, work, active, shift, notconv);
    else if (nmax <= 32 * 8)
        jacobi_launch<8>(nmat, st, sm, rm, A, V, evals, ldE, work, active, shift, notconv);
    else if (nmax <= 32 * 12)
        jacobi_launch<12>(nmat, st, sm, rm, A, V, evals, ldE, work, active, shift, notconv);
    else if (nmax <= 32 * 16)
        jacobi_launch<16>(nmat, st, sm, rm, A, V, evals, ldE, work, active, shift, notconv);
    else
        jacobi_launch<JAC_PER>(nmat, st, sm, rm, A, V, evals, ldE, work, active, shift, notconv);
}

__global__ void fock_assemble_kernel(const RepMat* rms, const double* h, const double* G, double* F,
                                     const int* active)
{
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    const RepMat rm = rms[r];
    const int n = rm.N;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
        const int i = e / n, j = e % n;
        F[rm.off + e] = h[rm.off + e] + G[rm.off + e] + G[rm.off + (size_t)j * n + i];
    }
}

__device__ __forceinline__ double block_sum(double v, double* red)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) s += red[k];
    __syncthreads();
    return s;
}

// E = 1/2 sum D (h + F) + V_nn (one block per replica)
__global__ void energy_kernel(const RepMat* rms, const double* D, const double* h, const double* F,
                              const double* enn, double* E, const int* active)
{
    const int r = blockIdx.x;
    if (active && !active[r]) return;
    const RepMat rm = rms[r];
    __shared__ double red[32];
    double s = 0.0;
    for (int e = threadIdx.x; e < rm.N * rm.N; e += blockDim.x)
        s += D[rm.off + e] * (h[rm.off + e] + F[rm.off + e]);
    s = block_sum(s, red);
    if (threadIdx.x == 0) E[r] = 0.5 * s + enn[r];
}

__global__ void antisym_kernel(const RepMat* rms, const double* M, double* E, const int* active)
{
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    const RepMat rm = rms[r];
    const int n = rm.N;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
        const int i = e / n, j = e % n;
        E[rm.off + e] = M[rm.off + e] - M[rm.off + (size_t)j * n + i];
    }
}

__global__ void maxabs_kernel(const RepMat* rms, const double* A, double* out, const int* active)
{
    const int r = blockIdx.x;
    if (active && !active[r]) return;
    const RepMat rm = rms[r];
    __shared__ double red[32];
    double m = 0.0;
    for (int e = threadIdx.x; e < rm.N * rm.N; e += blockDim.x) m = fmax(m, fabs(A[rm.off + e]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mm = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) mm = fmax(mm, red[k]);
        out[r] = mm;
    }
}

// X = U diag(s^{-1/2}) U^T
__global__ void orth_kernel(const RepMat* rms, const double* U, const double* s, int ldE, double* X)
{
    const int r = blockIdx.y;
    const RepMat rm = rms[r];
    const int n = rm.N;
    const double* u = U + rm.off;
    const double* sv = s + (size_t)r * ldE;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
        const int i = e / n, j = e % n;
        double acc = 0.0;
        for (int k = 0; k < n; k++) acc += u[(size_t)i * n + k] * u[(size_t)j * n + k] / sqrt(sv[k]);
        X[rm.off + e] = acc;
    }
}

// out[i][k] = C[i][k] * evals[k] for k < nocc (other columns zero)
__global__ void scale_cols_kernel(const RepMat* rms, const double* C, const double* ev, int ldE, double* out,
                                  const int* mask)
{
    const int r = blockIdx.y;
    if (mask && !mask[r]) return;
    const RepMat rm = rms[r];
    const int n = rm.N;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
        const int k = e % n;
        out[rm.off + e] = k < rm.nocc ? C[rm.off + e] * ev[(size_t)r * ldE + k] : 0.0;
    }
}

__global__ void copy_mats_kernel(const RepMat* rms, const double* src, double* dst, const int* mask)
{
    const int r = blockIdx.y;
    if (mask && !mask[r]) return;
    const RepMat rm = rms[r];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rm.N * rm.N; e += gridDim.x * blockDim.x)
        dst[rm.off + e] = src[rm.off + e];
}

// DIIS history: Fh/Eh[(rep * hist + slot) * stride + e] with stride = max N^2
__global__ void diis_store_kernel(const RepMat* rms, const double* F, const double* E, double* Fh, double* Eh,
                                  const int* slot, int hist, long long stride, const int* active)
{
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    const RepMat rm = rms[r];
    const size_t base = ((size_t)r * hist + slot[r]) * stride;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rm.N * rm.N; e += gridDim.x * blockDim.x) {
        Fh[base + e] = F[rm.off + e];
        Eh[base + e] = E[rm.off + e];
    }
}

// B[rep][slot][j] = <e_slot, e_j> for the stored j (one block per (j, rep))
__global__ void diis_dots_kernel(const RepMat* rms, const double* Eh, const int* slot, const int* count, int hist,
                                 long long stride, double* B, const int* active)
{
    const int r = blockIdx.y, j = blockIdx.x;
    if (active && !active[r]) return;
    if (j >= count[r]) return;
    const RepMat rm = rms[r];
    const int s = slot[r];
    const double* ea = Eh + ((size_t)r * hist + s) * stride;
    const double* eb = Eh + ((size_t)r * hist + j) * stride;
    __shared__ double red[32];
    double acc = 0.0;
    for (int e = threadIdx.x; e < rm.N * rm.N; e += blockDim.x) acc += ea[e] * eb[e];
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) {
        B[((size_t)r * hist + s) * hist + j] = acc;
        B[((size_t)r * hist + j) * hist + s] = acc;
    }
}

// Pulay: minimise |sum c_i e_i| subject to sum c_i = 1:
// [B 1; 1 0] [c; -lambda] = [0; 1], Gaussian elimination with partial pivoting;
// an ill-conditioned system drops the oldest vectors first.
__global__ void diis_solve_kernel(int nrep, const double* B, const int* slot, const int* count, int hist,
                                  double* coef, const int* active)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrep) return;
    if (active && !active[r]) return;
    const int m_all = count[r];
    double* c = coef + (size_t)r * hist;
    for (int j = 0; j < hist; j++) c[j] = 0.0;
    // chronological order of the stored slots: oldest first
    int order[16];
    for (int k = 0; k < m_all; k++) order[k] = (slot[r] - (m_all - 1) + k + 2 * hist) % hist;
    for (int drop = 0; drop < m_all; drop++) {
        const int m = m_all - drop;
        if (m < 2) break;
        double a[17][18];
        for (int i = 0; i < m; i++) {
            for (int j = 0; j < m; j++) a[i][j] = B[((size_t)r * hist + order[drop + i]) * hist + order[drop + j]];
            a[i][m] = 1.0;
            a[i][m + 1] = 0.0;
        }
        for (int j = 0; j < m; j++) a[m][j] = 1.0;
        a[m][m] = 0.0;
        a[m][m + 1] = 1.0;
        const int n = m + 1;
        double scale = 0.0;
        for (int i = 0; i < m; i++) scale = fmax(scale, fabs(a[i][i]));
        bool ok = true;
        for (int col = 0; col < n && ok; col++) {
            int piv = col;
            for (int i = col + 1; i < n; i++)
                if (fabs(a[i][col]) > fabs(a[piv][col])) piv = i;
            if (fabs(a[piv][col]) <= 1e-14 * fmax(scale, 1e-300)) {
                ok = false;
                break;
            }
            if (piv != col)
                for (int j = 0; j <= n; j++) {
                    const double t = a[col][j];
                    a[col][j] = a[piv][j];
                    a[piv][j] = t;
                }
            for (int i = col + 1; i < n; i++) {
                const double f = a[i][col] / a[col][col];
                for (int j = col; j <= n; j++) a[i][j] -= f * a[col][j];
            }
        }
        if (!ok) continue;
        double x[17];
        for (int i = n - 1; i >= 0; i--) {
            double s = a[i][n];
            for (int j = i + 1; j < n; j++) s -= a[i][j] * x[j];
            x[i] = s / a[i][i];
        }
        for (int i = 0; i < m; i++) c[order[drop + i]] = x[i];
        return;
    }
    c[slot[r]] = 1.0;
}

__global__ void diis_combine_kernel(const RepMat* rms, const double* Fh, const double* coef, int hist,
                                    long long stride, const double* F, double* Fbar, const int* diis_on,
                                    const int* active)
{
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    const RepMat rm = rms[r];
    const bool on = diis_on[r];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rm.N * rm.N; e += gridDim.x * blockDim.x) {
        if (!on) {
            Fbar[rm.off + e] = F[rm.off + e];
            continue;
        }
        double acc = 0.0;
        for (int j = 0; j < hist; j++) {
            const double cj = coef[(size_t)r * hist + j];
            if (cj != 0.0) acc += cj * Fh[((size_t)r * hist + j) * stride + e];
        }
        Fbar[rm.off + e] = acc;
    }
}

__global__ void identity_kernel(const RepMat* rms, double* A, const int* mask)
{
    const int r = blockIdx.y;
    if (mask && !mask[r]) return;
    const RepMat rm = rms[r];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rm.N * rm.N; e += gridDim.x * blockDim.x)
        A[rm.off + e] = (e / rm.N == e % rm.N) ? 1.0 : 0.0;
}

__global__ void gather_xyz_kernel(const double* ax, const int* sa, int n, double* sx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int x = 0; x < 3; x++) sx[3 * i + x] = ax[3 * sa[i] + x];
}

__global__ void add_mats_kernel(const RepMat* rms, const double* A, const double* B, double* C)
{
    const int r = blockIdx.y;
    const RepMat rm = rms[r];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rm.N * rm.N; e += gridDim.x * blockDim.x)
        C[rm.off + e] = A[rm.off + e] + B[rm.off + e];
}

__global__ void shell_bounds_kernel(Shells S, Reps R, const double* M, double* Dsh, const int* mask)
{
    const int r = blockIdx.y;
    if (mask && !mask[r]) return;
    const int n = R.nsh[r];
    const int a = blockIdx.x;
    if (a >= n) return;
    const int N = R.nbf[r];
    const double* m = M + R.moff[r];
    const int ga = R.sh0[r] + a;
    const int fa = S.bf[ga], na = nsph(S.l[ga]);
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        const int gb = R.sh0[r] + b;
        const int fb = S.bf[gb], nb = nsph(S.l[gb]);
        double mx = 0.0;
        for (int i = 0; i < na; i++)
            for (int j = 0; j < nb; j++) mx = fmax(mx, fabs(m[(size_t)(fa + i) * N + fb + j]));
        Dsh[R.dsoff[r] + (size_t)a * n + b] = mx;
    }
}

__global__ void delta_density_kernel(const RepMat* rms, const double* D, double* Dprev, double* dD, double* G,
                                     const int* mode)
{
    const int r = blockIdx.y;
    const int md = mode[r];
    if (md == 0) return;
    const RepMat rm = rms[r];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rm.N * rm.N; e += gridDim.x * blockDim.x) {
        const double d = D[rm.off + e];
        dD[rm.off + e] = md == 1 ? d - Dprev[rm.off + e] : d;
        Dprev[rm.off + e] = d;
        if (md == 2) G[rm.off + e] = 0.0;
    }
}

}  // namespace


void launch_shell_bounds(const Shells& S, const Reps& R, int nrep, int maxsh, const double* M, double* Dsh,
                         const int* mask, cudaStream_t st)
{
    if (nrep == 0 || maxsh == 0) return;
    shell_bounds_kernel<<<dim3(maxsh, nrep), 128, 0, st>>>(S, R, M, Dsh, mask);
}

void launch_delta_density(const RepMat* rm, int nrep, const double* D, double* Dprev, double* dD, double* G,
                          const int* mode, cudaStream_t st)
{
    delta_density_kernel<<<dim3(64, nrep), 256, 0, st>>>(rm, D, Dprev, dD, G, mode);
}

__global__ void to_fixed_kernel(double* a, long long n, double fxs)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        ((long long*)a)[i] = __double2ll_rn(a[i] * fxs);
}

__global__ void from_fixed_kernel(double* a, long long n, double fxs)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] = (double)((const long long*)a)[i] / fxs;
}

void launch_double_to_fixed(double* a, long long n, double fxs, cudaStream_t st)
{
    if (n > 0) to_fixed_kernel<<<(int)std::min<long long>((n + 255) / 256, 4096), 256, 0, st>>>(a, n, fxs);
}

void launch_fixed_to_double(double* a, long long n, double fxs, cudaStream_t st)
{
    if (n > 0) from_fixed_kernel<<<(int)std::min<long long>((n + 255) / 256, 4096), 256, 0, st>>>(a, n, fxs);
}

void gather_xyz(const double* atom_xyz, const int* shell_atom, int nshell, double* shell_xyz, cudaStream_t st)
{
    if (nshell == 0) return;
    gather_xyz_kernel<<<(nshell + 127) / 128, 128, 0, st>>>(atom_xyz, shell_atom, nshell, shell_xyz);
}

// ---------------------------------------------------------------------------
// Eigensolver entry point that allocates nothing. Some callers cannot call
// cudaMalloc: code whose device memory is owned by another allocator (a
// framework's caching pool that has already reserved the GPU), and loops that
// must not pay the implicit device synchronisation of cudaMalloc/cudaFree
// between launches. For them the solver's workspace and its per-matrix
// descriptors live in file-scope device arrays of fixed size, which every GPU
// that loads the library keeps until the process exits.
// ---------------------------------------------------------------------------
#define PIMD_EIGH_NOALLOC_MAX_DOUBLES (1 << 21)  // 16 MiB: nmat * n * n <= 2,097,152
#define PIMD_EIGH_NOALLOC_MAX_MATS 1024

static __device__ __align__(256) double g_eigh_work[PIMD_EIGH_NOALLOC_MAX_DOUBLES];
static __device__ __align__(256) RepMat g_eigh_desc[PIMD_EIGH_NOALLOC_MAX_MATS];

// device addresses of the two arrays, resolved once per device (the names
// above are host-side stand-ins and must never be passed to a kernel)
static double* g_eigh_work_ptr[64];
static RepMat* g_eigh_desc_ptr[64];

// descriptors of nmat consecutive n x n matrices, written on the device (no
// host staging buffer, so the call only enqueues work on its stream)
__global__ void eigh_desc_kernel(RepMat* desc, int nmat, int n)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nmat; r += gridDim.x * blockDim.x)
        desc[r] = RepMat{n, 0, (long long)r * n * n};
}

void launch_identity(const RepMat* rm, int nrep, double* A, const int* mask, cudaStream_t st)
{
    identity_kernel<<<dim3(64, nrep), 256, 0, st>>>(rm, A, mask);
}

void add_mats(const RepMat* rm, int nrep, const double* A, const double* B, double* C, cudaStream_t st)
{
    add_mats_kernel<<<dim3(64, nrep), 256, 0, st>>>(rm, A, B, C);
}

void launch_gemm(const GemmDesc* d_desc, int ndesc, int maxM, int maxN, const int* active, cudaStream_t st)
{
    if (ndesc == 0 || maxM == 0 || maxN == 0) return;
    dim3 grid((maxN + TB - 1) / TB, (maxM + TB - 1) / TB, ndesc);
    gemm_kernel<<<grid, 256, 0, st>>>(d_desc, active);
}

void launch_jacobi(const RepMat* d_rm, int nrep, const double* A, double* V, double* evals, int ldE, double* work,
                   const int* active, int shift_to_spd, cudaStream_t st, int* notconv)
{
    // ldE is the largest n of the batch; the kernel holds 32 * JAC_PER column elements per warp
    if (ldE > 32 * JAC_PER) return;
    if (nrep == 0) return;
    jacobi_dispatch(nrep, ldE, st, d_rm, A, V, evals, ldE, work, active, shift_to_spd, notconv);
}

static dim3 elem_grid(int nrep) { return dim3(64, nrep); }

void launch_fock_assemble(const RepMat* rm, int nrep, const double* h, const double* G, double* F,
                          const int* active, cudaStream_t st)
{
    fock_assemble_kernel<<<elem_grid(nrep), 256, 0, st>>>(rm, h, G, F, active);
}

void launch_energy(const RepMat* rm, int nrep, const double* D, const double* h, const double* F,
                   const double* enn, double* E, const int* active, cudaStream_t st)
{
    energy_kernel<<<nrep, 256, 0, st>>>(rm, D, h, F, enn, E, active);
}

void launch_antisym(const RepMat* rm, int nrep, const double* M, double* E, const int* active, cudaStream_t st)
{
    antisym_kernel<<<elem_grid(nrep), 256, 0, st>>>(rm, M, E, active);
}

void launch_maxabs(const RepMat* rm, int nrep, const double* A, double* out, const int* active, cudaStream_t st)
{
    maxabs_kernel<<<nrep, 256, 0, st>>>(rm, A, out, active);
}

void launch_orth_from_eig(const RepMat* rm, int nrep, const double* U, const double* s, int ldE, double* X,
                          cudaStream_t st)
{
    orth_kernel<<<elem_grid(nrep), 256, 0, st>>>(rm, U, s, ldE, X);
}

void launch_scale_cols(const RepMat* rm, int nrep, const double* C, const double* evals, int ldE, double* out,
                       const int* mask, cudaStream_t st)
{
    scale_cols_kernel<<<elem_grid(nrep), 256, 0, st>>>(rm, C, evals, ldE, out, mask);
}

void launch_copy_mats(const RepMat* rm, int nrep, const double* src, double* dst, const int* mask,
                      cudaStream_t st)
{
    copy_mats_kernel<<<elem_grid(nrep), 256, 0, st>>>(rm, src, dst, mask);
}

// one block per descriptor {rep, f0, n, off}: an n x n diagonal block of D[rep]
__global__ void place_blocks_kernel(const RepMat* rms, const int* desc, int nblk, const double* src, double* D)
{
    const int b = blockIdx.x;
    if (b >= nblk) return;
    const int rep = desc[4 * b], f0 = desc[4 * b + 1], n = desc[4 * b + 2], off = desc[4 * b + 3];
    const RepMat rm = rms[rep];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x)
        D[rm.off + (size_t)(f0 + e / n) * rm.N + f0 + e % n] = src[(size_t)off + e];
}

void launch_place_blocks(const RepMat* rm, const int* desc4, int nblk, const double* src, double* D,
                         cudaStream_t st)
{
    if (nblk > 0) place_blocks_kernel<<<nblk, 128, 0, st>>>(rm, desc4, nblk, src, D);
}


void launch_diis_store(const RepMat* rm, int nrep, const double* F, const double* E, double* Fh, double* Eh,
                       const int* slot, int hist, long long stride, const int* active, cudaStream_t st)
{
    diis_store_kernel<<<elem_grid(nrep), 256, 0, st>>>(rm, F, E, Fh, Eh, slot, hist, stride, active);
}

void launch_diis_dots(const RepMat* rm, int nrep, const double* Eh, const int* slot, const int* count, int hist,
                      long long stride, double* B, const int* active, cudaStream_t st)
{
    diis_dots_kernel<<<dim3(hist, nrep), 256, 0, st>>>(rm, Eh, slot, count, hist, stride, B, active);
}

void launch_diis_solve(int nrep, const double* B, const int* slot, const int* count, int hist, double* coef,
                       const int* active, cudaStream_t st)
{
    diis_solve_kernel<<<(nrep + 31) / 32, 32, 0, st>>>(nrep, B, slot, count, hist, coef, active);
}

void launch_diis_combine(const RepMat* rm, int nrep, const double* Fh, const double* coef, int hist,
                         long long stride, const double* F, double* Fbar, const int* diis_on, const int* active,
                         cudaStream_t st)
{
    diis_combine_kernel<<<elem_grid(nrep), 256, 0, st>>>(rm, Fh, coef, hist, stride, F, Fbar, diis_on,
                                                         active);
}

int eigh_noalloc(int nmat, int n, const double* A, double* V, double* evals, cudaStream_t st)
{
    if (nmat <= 0 || n <= 0 || !A || !V || !evals) return PIMD_EINVAL;
    if (nmat > PIMD_EIGH_NOALLOC_MAX_MATS || (long long)nmat * n * n > PIMD_EIGH_NOALLOC_MAX_DOUBLES ||
        n > 32 * JAC_PER)
        return PIMD_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PIMD_ECUDA;
    if (!g_eigh_work_ptr[dev]) {
        // set-up on the first call on this device
        void* w = nullptr;
        void* d = nullptr;
        if (cudaGetSymbolAddress(&w, g_eigh_work) != cudaSuccess) return PIMD_ECUDA;
        if (cudaGetSymbolAddress(&d, g_eigh_desc) != cudaSuccess) return PIMD_ECUDA;
        g_eigh_desc_ptr[dev] = (RepMat*)d;
        g_eigh_work_ptr[dev] = (double*)w;
    }
    eigh_desc_kernel<<<(nmat + 127) / 128, 128, 0, st>>>(g_eigh_desc_ptr[dev], nmat, n);
    jacobi_dispatch(nmat, n, st, g_eigh_desc_ptr[dev], A, V, evals, n, g_eigh_work_ptr[dev], nullptr, 1, nullptr);
    if (cudaGetLastError() != cudaSuccess) return PIMD_ECUDA;
    return PIMD_OK;
}

}  // namespace pimd

// C ABI (declared in include/pimdgb.h)
extern "C" int pimd_eigh_noalloc(int nmat, int n, const double* A_dev, double* V_dev, double* evals_dev, void* stream)
{
    return pimd::eigh_noalloc(nmat, n, A_dev, V_dev, evals_dev, (cudaStream_t)stream);
}
