// Shell-quartet ERI kernels: Coulomb/exchange (Fock) build, Schwarz factors
// and the two-electron part of the analytic RHF gradient.
//
// One thread evaluates one contracted shell quartet (ab|cd) of one replica:
// the primitive loop runs the generated Obara-Saika vertical recursion into
// contracted [e0|f0] accumulators, then the generated Head-Gordon-Pople
// horizontal recursion gives the Cartesian block, which is turned into real
// spherical d functions and contracted with the density on the fly.
// A block shares one bra pair (staged in shared memory) and walks a tile of
// 32, 64 or 128 ket pairs of the same class (one thread each; the width is
// chosen per class pair by the autotuner), so the code path is uniform across
// the block. Every replica of the call is covered by the same launch.
//
// Quartets are the canonical ones (a >= b, c >= d, ab >= cd); each is
// scattered to its 8 permutations with weight f = 1/|stabiliser| into a
// non-symmetric G' with F = h + G' + G'^T, where (per element)
//   G'_ab += 2f D_cd v,  G'_cd += 2f D_ab v,
//   G'_ac -= f/2 D_bd v, G'_bc -= f/2 D_ad v, G'_ad -= f/2 D_bc v, G'_bd -= f/2 D_ac v,
// which reproduces F = h + J - K/2 with J_mn = sum D_ls (mn|ls) and
// K_mn = sum D_ls (ml|ns) for a symmetric density.
#pragma once
#include "boys.cuh"
#include "pimd_dev.cuh"

namespace pimd {

constexpr double kSqrt3 = 1.7320508075688772935;

// in[N0][ncart(L)][N2] -> out[N0][nsph(L)][N2]; spherical d order m = -2..2:
// sqrt3 xy, sqrt3 yz, zz - (xx + yy)/2, sqrt3 xz, sqrt3/2 (xx - yy)
template <int N0, int L, int N2, typename T>
__device__ __forceinline__ void sph_index(const T* __restrict__ in, T* __restrict__ out)
{
    if constexpr (L < 2) {
#pragma unroll
        for (int i = 0; i < N0 * ncart(L) * N2; i++) out[i] = in[i];
    } else {
#pragma unroll
        for (int i0 = 0; i0 < N0; i0++)
#pragma unroll
            for (int i2 = 0; i2 < N2; i2++) {
                const T* s = in + i0 * 6 * N2 + i2;
                T* d = out + i0 * 5 * N2 + i2;
                const T xx = s[0], xy = s[N2], xz = s[2 * N2], yy = s[3 * N2], yz = s[4 * N2], zz = s[5 * N2];
                d[0] = T(kSqrt3) * xy;
                d[N2] = T(kSqrt3) * yz;
                d[2 * N2] = zz - T(0.5) * (xx + yy);
                d[3 * N2] = T(kSqrt3) * xz;
                d[4 * N2] = T(0.5 * kSqrt3) * (xx - yy);
            }
    }
}

// transpose of sph_index: in[N0][nsph(L)][N2] -> out[N0][ncart(L)][N2]
template <int N0, int L, int N2, typename T>
__device__ __forceinline__ void sph_index_t(const T* __restrict__ in, T* __restrict__ out)
{
    if constexpr (L < 2) {
#pragma unroll
        for (int i = 0; i < N0 * ncart(L) * N2; i++) out[i] = in[i];
    } else {
#pragma unroll
        for (int i0 = 0; i0 < N0; i0++)
#pragma unroll
            for (int i2 = 0; i2 < N2; i2++) {
                const T* s = in + i0 * 5 * N2 + i2;
                T* d = out + i0 * 6 * N2 + i2;
                const T m2 = s[0], m1 = s[N2], m0 = s[2 * N2], p1 = s[3 * N2], p2 = s[4 * N2];
                d[0] = T(-0.5) * m0 + T(0.5 * kSqrt3) * p2;
                d[N2] = T(kSqrt3) * m2;
                d[2 * N2] = T(kSqrt3) * p1;
                d[3 * N2] = T(-0.5) * m0 - T(0.5 * kSqrt3) * p2;
                d[4 * N2] = T(kSqrt3) * m1;
                d[5 * N2] = m0;
            }
    }
}

// Cartesian (ab|cd) block -> spherical block
template <int LA, int LB, int LC, int LD, typename T>
__device__ __forceinline__ void cart_to_sph4(T* __restrict__ buf, T* __restrict__ tmp)
{
    constexpr int ca = ncart(LA), cb = ncart(LB), cc = ncart(LC), cd = ncart(LD);
    constexpr int sa = nsph(LA), sb = nsph(LB), sc = nsph(LC);
    sph_index<1, LA, cb * cc * cd>(buf, tmp);
    sph_index<sa, LB, cc * cd>(tmp, buf);
    sph_index<sa * sb, LC, cd>(buf, tmp);
    sph_index<sa * sb * sc, LD, 1>(tmp, buf);
}

template <int LA, int LB, int LC, int LD, typename T>
__device__ __forceinline__ void sph_to_cart4_t(T* __restrict__ buf, T* __restrict__ tmp)
{
    constexpr int ca = ncart(LA), cb = ncart(LB), cc = ncart(LC);
    constexpr int sb = nsph(LB), sc = nsph(LC), sd = nsph(LD);
    sph_index_t<1, LA, sb * sc * sd>(buf, tmp);
    sph_index_t<ca, LB, sc * sd>(tmp, buf);
    sph_index_t<ca * cb, LC, sd>(buf, tmp);
    sph_index_t<ca * cb * cc, LD, 1>(tmp, buf);
}

// Per-primitive-quartet quantities of the Obara-Saika recursion.
template <typename R>
struct PrimQ {
    R PA[3], WP[3], QC[3], WQ[3];
    R o2p, o2pr, o2q, o2qr, o2pq, T, theta;
};
typedef PrimQ<double> PrimQuartet;

// 1/sqrt(x) for normal positive x with |log2 x| < 126 (p + q of two Gaussian
// exponents): a single-precision estimate from the hardware approximation
// (operand and result moved between the formats with integer operations on
// the exponent and mantissa fields), then one Newton step for f(y) = y^-2 - x
// carried to second order: with e = 1 - x y0^2, y = y0 (1 + e/2 + 3e^2/8), so
// the relative error goes from |e| < 2^-20 to about (5/16) e^3 < 2^-61.
__device__ __forceinline__ double rsqrt_r(double x)
{
    const int hi = __double2hiint(x), lo = __double2loint(x);
    // float with the top 23 mantissa bits of x (exponent rebias 1023 -> 127)
    const float xf = __int_as_float(((hi - (896 << 20)) << 3) | ((unsigned)lo >> 29));
    const int yb = __float_as_int(rsqrtf(xf));
    const double y0 = __hiloint2double((yb >> 3) + (896 << 20), yb << 29);
    const double t = x * y0;
    const double e = fma(-t, y0, 1.0);
    const double c = fma(0.375, e, 0.5);
    return fma(y0 * e, c, y0);
}
__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }

// bra/ket: the first PP_NERI primitive-pair fields (p, P, K, P - A, 1/(2p), 1/(2p^2))
template <typename R>
__device__ __forceinline__ void prim_quartet(const R* bra, const R* ket, PrimQ<R>& g)
{
    const R p = bra[PP_P], q = ket[PP_P];
    const R rs = rsqrt_r(p + q);
    const R ipq = rs * rs;
    const R qi = q * ipq, pi = p * ipq;
    const R rho = p * qi;
    const R PQx = bra[PP_PX] - ket[PP_PX], PQy = bra[PP_PY] - ket[PP_PY], PQz = bra[PP_PZ] - ket[PP_PZ];
    // W - P = -q/(p+q) (P - Q), W - Q = p/(p+q) (P - Q)
    g.WP[0] = -qi * PQx;
    g.WP[1] = -qi * PQy;
    g.WP[2] = -qi * PQz;
    g.WQ[0] = pi * PQx;
    g.WQ[1] = pi * PQy;
    g.WQ[2] = pi * PQz;
    g.PA[0] = bra[PP_PAX];
    g.PA[1] = bra[PP_PAY];
    g.PA[2] = bra[PP_PAZ];
    g.QC[0] = ket[PP_PAX];
    g.QC[1] = ket[PP_PAY];
    g.QC[2] = ket[PP_PAZ];
    g.T = rho * fma(PQx, PQx, fma(PQy, PQy, PQz * PQz));
    g.o2p = bra[PP_O2P];
    g.o2pr = rho * bra[PP_O2PP];
    g.o2q = ket[PP_O2P];
    g.o2qr = rho * ket[PP_O2PP];
    g.o2pq = R(0.5) * ipq;
    g.theta = bra[PP_K] * ket[PP_K] * rs;
}


// J'_ab of a tile: every lane of the warp holds a quartet with the same bra
// pair (ab), so the bra-side Coulomb block sum_cd 2f D_cd (ab|cd) is summed
// over the warp with shuffles and added to G' with one atomic per element
// (lanes without a quartet contribute zero; all 32 lanes must call this).
template <int LA, int LB, int LC, int LD, typename R>
__device__ __forceinline__ void bra_coulomb_warp(const R* __restrict__ I, double f, bool work, int fa, int fb,
                                                 int fc, int fd, int N, const R* __restrict__ D,
                                                 double* __restrict__ G, double fxs)
{
    constexpr int na = nsph(LA), nb = nsph(LB), nc = nsph(LC), nd = nsph(LD);
    R Dcd[nc * nd];
#pragma unroll
    for (int i = 0; i < nc; i++)
#pragma unroll
        for (int j = 0; j < nd; j++) Dcd[i * nd + j] = work ? __ldg(D + (size_t)(fc + i) * N + fd + j) : R(0);
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int a = 0; a < na; a++) {
#pragma unroll
        for (int b = 0; b < nb; b++) {
            R s = R(0);
#pragma unroll
            for (int c = 0; c < nc; c++)
#pragma unroll
                for (int d = 0; d < nd; d++) s += Dcd[c * nd + d] * I[((a * nb + b) * nc + c) * nd + d];
            double v = work ? 2.0 * f * (double)s : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0 && v != 0.0) det_add(G + (size_t)(fa + a) * N + fb + b, v, fxs);
        }
    }
}

// Contract a spherical block with the density and scatter into G' (the
// contraction in the block's precision R, the accumulation in FP64): J'_cd
// and the four exchange blocks; with bra_j, also J'_ab (else the caller adds
// it with bra_coulomb_warp).
template <int LA, int LB, int LC, int LD, typename R>
__device__ __forceinline__ void scatter_jk(const R* __restrict__ I, double f, int fa, int fb, int fc, int fd,
                                           int N, const R* __restrict__ D, double* __restrict__ G, double fxs,
                                           bool bra_j = true)
{
    constexpr int na = nsph(LA), nb = nsph(LB), nc = nsph(LC), nd = nsph(LD);
    R Dab[na * nb], Dcd[nc * nd], Dac[na * nc], Dad[na * nd], Dbc[nb * nc], Dbd[nb * nd];
#pragma unroll
    for (int i = 0; i < na; i++)
#pragma unroll
        for (int j = 0; j < nb; j++) Dab[i * nb + j] = __ldg(D + (size_t)(fa + i) * N + fb + j);
#pragma unroll
    for (int i = 0; i < nc; i++)
#pragma unroll
        for (int j = 0; j < nd; j++) Dcd[i * nd + j] = __ldg(D + (size_t)(fc + i) * N + fd + j);
#pragma unroll
    for (int i = 0; i < na; i++)
#pragma unroll
        for (int j = 0; j < nc; j++) Dac[i * nc + j] = __ldg(D + (size_t)(fa + i) * N + fc + j);
#pragma unroll
    for (int i = 0; i < na; i++)
#pragma unroll
        for (int j = 0; j < nd; j++) Dad[i * nd + j] = __ldg(D + (size_t)(fa + i) * N + fd + j);
#pragma unroll
    for (int i = 0; i < nb; i++)
#pragma unroll
        for (int j = 0; j < nc; j++) Dbc[i * nc + j] = __ldg(D + (size_t)(fb + i) * N + fc + j);
#pragma unroll
    for (int i = 0; i < nb; i++)
#pragma unroll
        for (int j = 0; j < nd; j++) Dbd[i * nd + j] = __ldg(D + (size_t)(fb + i) * N + fd + j);

    // J'_ab (rows of the bra)
    if (bra_j) {
#pragma unroll
        for (int a = 0; a < na; a++) {
#pragma unroll
            for (int b = 0; b < nb; b++) {
                R s = R(0);
#pragma unroll
                for (int c = 0; c < nc; c++)
#pragma unroll
                    for (int d = 0; d < nd; d++) s += Dcd[c * nd + d] * I[((a * nb + b) * nc + c) * nd + d];
                det_add(G + (size_t)(fa + a) * N + fb + b, 2.0 * f * (double)s, fxs);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < nc; c++)
#pragma unroll
        for (int d = 0; d < nd; d++) {
            R s = R(0);
#pragma unroll
            for (int a = 0; a < na; a++)
#pragma unroll
                for (int b = 0; b < nb; b++) s += Dab[a * nb + b] * I[((a * nb + b) * nc + c) * nd + d];
            det_add(G + (size_t)(fc + c) * N + fd + d, 2.0 * f * (double)s, fxs);
        }
#pragma unroll
    for (int a = 0; a < na; a++)
#pragma unroll
        for (int c = 0; c < nc; c++) {
            R s = R(0);
#pragma unroll
            for (int b = 0; b < nb; b++)
#pragma unroll
                for (int d = 0; d < nd; d++) s += Dbd[b * nd + d] * I[((a * nb + b) * nc + c) * nd + d];
            det_add(G + (size_t)(fa + a) * N + fc + c, -0.5 * f * (double)s, fxs);
        }
#pragma unroll
    for (int b = 0; b < nb; b++)
#pragma unroll
        for (int c = 0; c < nc; c++) {
            R s = R(0);
#pragma unroll
            for (int a = 0; a < na; a++)
#pragma unroll
                for (int d = 0; d < nd; d++) s += Dad[a * nd + d] * I[((a * nb + b) * nc + c) * nd + d];
            det_add(G + (size_t)(fb + b) * N + fc + c, -0.5 * f * (double)s, fxs);
        }
#pragma unroll
    for (int a = 0; a < na; a++)
#pragma unroll
        for (int d = 0; d < nd; d++) {
            R s = R(0);
#pragma unroll
            for (int b = 0; b < nb; b++)
#pragma unroll
                for (int c = 0; c < nc; c++) s += Dbc[b * nc + c] * I[((a * nb + b) * nc + c) * nd + d];
            det_add(G + (size_t)(fa + a) * N + fd + d, -0.5 * f * (double)s, fxs);
        }
#pragma unroll
    for (int b = 0; b < nb; b++)
#pragma unroll
        for (int d = 0; d < nd; d++) {
            R s = R(0);
#pragma unroll
            for (int a = 0; a < na; a++)
#pragma unroll
                for (int c = 0; c < nc; c++) s += Dac[a * nc + c] * I[((a * nb + b) * nc + c) * nd + d];
            det_add(G + (size_t)(fb + b) * N + fd + d, -0.5 * f * (double)s, fxs);
        }
}

// first nf primitive-pair fields of pair g, primitive pair k
__device__ __forceinline__ void load_ppn(const Pairs& P, int g, int k, double* out, int nf)
{
    const size_t n = P.n;
#pragma unroll
    for (int f = 0; f < nf; f++) out[f] = __ldg(P.pp + ((size_t)f * PIMD_MAXPP + k) * n + g);
}
__device__ __forceinline__ void load_ppn(const Pairs& P, int g, int k, float* out, int nf)
{
    const size_t n = P.n;
#pragma unroll
    for (int f = 0; f < nf; f++) out[f] = __ldg(P.ppf + ((size_t)f * PIMD_MAXPP + k) * n + g);
}
__device__ __forceinline__ const double* pp_base(const Pairs& P, double) { return P.pp; }
__device__ __forceinline__ const float* pp_base(const Pairs& P, float) { return P.ppf; }

// contracted Cartesian block of one quartet via the generated recursion.
// Primitive screening: primitive quartet (i|j) is skipped when
// qp_i qp_j < qthr (qthr = the primitive cutoff over the quartet's density
// bound; qthr <= 0 keeps every primitive); both primitive lists are in
// descending order of qp, so the quartets that survive form a staircase: for
// ket primitive j the bra primitives i < imax(j), imax non-increasing. The
// loop walks that staircase as one flat sequence of `total` primitive
// quartets, and runs `kmax` iterations (kmax >= total, the longest sequence
// of the warp), so that a warp executes the recursion once per position of
// its longest lane instead of once per primitive quartet that any lane needs.
// Returns the number of primitive quartets evaluated.
__device__ __forceinline__ int stair_width(const float* sqp, int nbra, float qj, float qthr)
{
    int n = 0;
    while (n < nbra && sqp[n] * qj >= qthr) n++;
    return n;
}

__device__ __forceinline__ int stair_total(const float* sqp, int nbra, const Pairs& P, int cd, float qthr)
{
    const int nket = P.npp[cd];
    if (qthr <= 0.0f) return nbra * nket;
    int total = 0;
    for (int j = 0; j < nket; j++) {
        const int w = stair_width(sqp, nbra, __ldg(P.qp + (size_t)j * P.n + cd), qthr);
        if (w == 0) break;
        total += w;
    }
    return total;
}

template <class C, typename R>
__device__ __forceinline__ int quartet_cart(const R (*sbra)[PIMD_MAXPP], const float* sqp, int nbra, const Pairs& P,
                                            int cd, const double A[3], const double B[3], const double Cc[3],
                                            const double Dd[3], const R* __restrict__ boys, float qthr, int total,
                                            int kmax, R* cart)
{
    R acc[C::NE * C::NF];
#pragma unroll
    for (int i = 0; i < C::NE * C::NF; i++) acc[i] = R(0);
    const int nket = P.npp[cd];
    int i = 0, j = 0;
    int w = total > 0 ? (qthr > 0.0f ? stair_width(sqp, nbra, __ldg(P.qp + cd), qthr) : nbra) : 0;
    R ket[PP_NERI];
    for (int k = 0; k < kmax; k++) {
        if (k < total) {
            if (i == 0) load_ppn(P, cd, j, ket, PP_NERI);
            R bra[PP_NERI];
#pragma unroll
            for (int f = 0; f < PP_NERI; f++) bra[f] = sbra[f][i];
            PrimQ<R> g;
            prim_quartet<R>(bra, ket, g);
            R F[C::L + 1];
            boys_eval<C::L>(g.T, boys, g.theta, F);
            C::template vrr<R>(F, g.PA[0], g.PA[1], g.PA[2], g.WP[0], g.WP[1], g.WP[2], g.QC[0], g.QC[1], g.QC[2],
                               g.WQ[0], g.WQ[1], g.WQ[2], g.o2p, g.o2pr, g.o2q, g.o2qr, g.o2pq, acc);
            if (++i == w) {
                i = 0;
                if (++j < nket)
                    w = qthr > 0.0f ? stair_width(sqp, nbra, __ldg(P.qp + (size_t)j * P.n + cd), qthr) : nbra;
            }
        }
    }
    C::template hrr<R>(acc, R(A[0] - B[0]), R(A[1] - B[1]), R(A[2] - B[2]), R(Cc[0] - Dd[0]), R(Cc[1] - Dd[1]),
                       R(Cc[2] - Dd[2]), cart);
    return total;
}

// tau_prim: primitive quartets whose bound qp_i qp_j (density bound) is below
// it are skipped (0 keeps every primitive quartet). fxs > 0: G' accumulated as
// fixed-point integers (det_add).
template <class C, typename R>
__global__ void __launch_bounds__(128) jk_kernel(Pairs P, Shells S, Reps R_, const Tile* __restrict__ tiles,
                                                 const R* __restrict__ Dall, double* __restrict__ Gall,
                                                 const R* __restrict__ boys, double tau_lo, double tau_hi,
                                                 const double* __restrict__ Dsh, unsigned long long* __restrict__ cnt,
                                                 double tau_prim, double fxs)
{
    __shared__ R sbra[PP_NERI][PIMD_MAXPP];
    __shared__ float sqp[PIMD_MAXPP];
    const Tile t = tiles[blockIdx.x];
    if (!R_.active[t.rep]) return;
    const int ab = t.ab;
    for (int e = threadIdx.x; e < PP_NERI * PIMD_MAXPP; e += blockDim.x) {
        const int f = e / PIMD_MAXPP, k = e % PIMD_MAXPP;
        sbra[f][k] = pp_base(P, R(0))[((size_t)f * PIMD_MAXPP + k) * P.n + ab];
    }
    if (threadIdx.x < PIMD_MAXPP) sqp[threadIdx.x] = P.qp[(size_t)threadIdx.x * P.n + ab];
    __syncthreads();
    const int r = t.rep;
    const int nbra = P.npp[ab];
    // screening of ket pair c0 + k: density-weighted Schwarz bound (every
    // contribution of the quartet to G' is at most 2 |(ab|cd)| times one of
    // the six density blocks) and the primitive cutoff over that bound
    auto screen = [&](int k, int& cd, int& sc, int& sd, float& qthr) -> bool {
        cd = t.c0 + k;
        sc = sd = 0;
        qthr = 0.0f;
        if (cd >= t.c1) return false;
        const int sa = P.sa[ab], sb = P.sb[ab];
        sc = P.sa[cd];
        sd = P.sb[cd];
        const double dq = fmax(fmax(fmax(shell_bound(R_, Dsh, r, sa, sb), shell_bound(R_, Dsh, r, sc, sd)),
                                    fmax(shell_bound(R_, Dsh, r, sa, sc), shell_bound(R_, Dsh, r, sa, sd))),
                               fmax(shell_bound(R_, Dsh, r, sb, sc), shell_bound(R_, Dsh, r, sb, sd)));
        const double bound = P.Q[ab] * P.Q[cd] * dq;
        qthr = (float)(tau_prim / dq);
        return bound >= tau_lo && bound < tau_hi;
    };
    int cd, sc, sd;
    float qthr;
    bool work = screen(threadIdx.x, cd, sc, sd, qthr);
    if (tau_prim > 0.0 && blockDim.x > 32) {
        // Lanes stop their primitive loops at their own cutoff, and a warp
        // issues for all its lanes: the block's quartets are regrouped by the
        // number of primitive quartets that survive (descending, bitonic sort
        // over the block), so that a warp holds quartets of similar length.
        __shared__ int skey[128], sidx[128];
        const int est = work ? stair_total(sqp, nbra, P, cd, qthr) : -1;
        const int tid = threadIdx.x, bd = blockDim.x;
        skey[tid] = est;
        sidx[tid] = tid;
        __syncthreads();
        for (int k = 2; k <= bd; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                const int o = tid ^ j;
                if (o > tid) {
                    const bool desc = (tid & k) == 0;
                    const int a = skey[tid], b = skey[o];
                    if (desc ? a < b : a > b) {
                        skey[tid] = b;
                        skey[o] = a;
                        const int x = sidx[tid];
                        sidx[tid] = sidx[o];
                        sidx[o] = x;
                    }
                }
                __syncthreads();
            }
        work = screen(sidx[tid], cd, sc, sd, qthr);
    }
    const int sa = P.sa[ab], sb = P.sb[ab];
    // a warp with no quartet left leaves; otherwise every lane stays for the
    // warp-wide J'_ab sum (the block's warps share the bra pair)
    if (__all_sync(0xffffffffu, !work)) return;
    constexpr int NCART = ncart(C::LA) * ncart(C::LB) * ncart(C::LC) * ncart(C::LD);
    R cart[NCART], tmp[NCART];
    double f = 0.0;
    int nprim = 0;
    const int total = work ? stair_total(sqp, nbra, P, cd, qthr) : 0;
    const int kmax = __reduce_max_sync(0xffffffffu, (unsigned)total);
    if (work) {
        double A[3], B[3], Cc[3], Dd[3];
#pragma unroll
        for (int x = 0; x < 3; x++) {
            A[x] = S.xyz[3 * sa + x];
            B[x] = S.xyz[3 * sb + x];
            Cc[x] = S.xyz[3 * sc + x];
            Dd[x] = S.xyz[3 * sd + x];
        }
        nprim = quartet_cart<C, R>(sbra, sqp, nbra, P, cd, A, B, Cc, Dd, boys, qthr, total, kmax, cart);
        cart_to_sph4<C::LA, C::LB, C::LC, C::LD>(cart, tmp);
        f = 1.0;
        if (sa == sb) f *= 0.5;
        if (sc == sd) f *= 0.5;
        if (ab == cd) f *= 0.5;
    }
    const unsigned nq = __reduce_add_sync(0xffffffffu, work ? 1u : 0u);
    const unsigned np = __reduce_add_sync(0xffffffffu, (unsigned)nprim);
    if ((threadIdx.x & 31) == 0 && nq) {
        atomicAdd(cnt, (unsigned long long)nq);
        atomicAdd(cnt + 1, (unsigned long long)np);
        atomicAdd(R_.qrep + 2 * r + (sizeof(R) == 4 ? 1 : 0), (unsigned long long)nq);
    }
    const int N = R_.nbf[r];
    const size_t off = R_.moff[r];
    bra_coulomb_warp<C::LA, C::LB, C::LC, C::LD, R>(cart, f, work, S.bf[P.sa[ab]], S.bf[P.sb[ab]], S.bf[sc],
                                                     S.bf[sd], N, Dall + off, Gall + off, fxs);
    if (work)
        scatter_jk<C::LA, C::LB, C::LC, C::LD, R>(cart, f, S.bf[sa], S.bf[sb], S.bf[sc], S.bf[sd], N, Dall + off,
                                                  Gall + off, fxs, false);
}

// Schwarz factors: Q_ab = sqrt(max over functions of (mn|mn)), one thread per pair
template <class C>
__global__ void __launch_bounds__(128) schwarz_kernel(Pairs P, Shells S, const int* __restrict__ list, int n,
                                                      const double* __restrict__ boys, double* __restrict__ Qout)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int ab = list[idx];
    const int sa = P.sa[ab], sb = P.sb[ab];
    double sbra_l[PP_NERI][PIMD_MAXPP];
    const int np = P.npp[ab];
    for (int k = 0; k < np; k++)
        for (int f = 0; f < PP_NERI; f++) sbra_l[f][k] = P.pp[((size_t)f * PIMD_MAXPP + k) * P.n + ab];
    double A[3], B[3];
#pragma unroll
    for (int x = 0; x < 3; x++) {
        A[x] = S.xyz[3 * sa + x];
        B[x] = S.xyz[3 * sb + x];
    }
    constexpr int NCART = ncart(C::LA) * ncart(C::LB) * ncart(C::LC) * ncart(C::LD);
    double cart[NCART], tmp[NCART];
    const float qone[PIMD_MAXPP] = {1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f};
    quartet_cart<C, double>(sbra_l, qone, np, P, ab, A, B, A, B, boys, 0.0f, np * P.npp[ab], np * P.npp[ab], cart);
    cart_to_sph4<C::LA, C::LB, C::LC, C::LD>(cart, tmp);
    constexpr int na = nsph(C::LA), nb = nsph(C::LB);
    double m = 0.0;
#pragma unroll
    for (int i = 0; i < na; i++)
#pragma unroll
        for (int j = 0; j < nb; j++) m = fmax(m, fabs(cart[((i * nb + j) * na + i) * nb + j]));
    Qout[ab] = sqrt(m);
}

// Primitive-pair Schwarz factors: for every primitive pair k of shell pair ab
// (one thread per pair), qp_k = sqrt(max over functions of |(kk|kk)|) with
// the contraction coefficients included, so that |(ij|kl)| <= qp_i qp_l for
// any primitive quartet (Cauchy-Schwarz for the two charge distributions).
// The pair's primitive data are then reordered by descending qp (every field,
// in place) and qp is stored in that order.
template <class C>
__global__ void __launch_bounds__(128) prim_schwarz_kernel(Pairs P, Shells S, const int* __restrict__ list, int n,
                                                           const double* __restrict__ boys, double* pp, float* qp,
                                                           float* qg)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int ab = list[idx];
    const int sa = P.sa[ab], sb = P.sb[ab];
    const int np = P.npp[ab];
    const size_t N = P.n;
    double A[3], B[3];
#pragma unroll
    for (int x = 0; x < 3; x++) {
        A[x] = S.xyz[3 * sa + x];
        B[x] = S.xyz[3 * sb + x];
    }
    constexpr int na = nsph(C::LA), nb = nsph(C::LB);
    constexpr int NCART = ncart(C::LA) * ncart(C::LB) * ncart(C::LC) * ncart(C::LD);
    float q[PIMD_MAXPP];
    int perm[PIMD_MAXPP];
    for (int k = 0; k < np; k++) {
        double v[PP_NERI];
        for (int f = 0; f < PP_NERI; f++) v[f] = pp[((size_t)f * PIMD_MAXPP + k) * N + ab];
        double acc[C::NE * C::NF];
        for (int i = 0; i < C::NE * C::NF; i++) acc[i] = 0.0;
        PrimQ<double> g;
        prim_quartet<double>(v, v, g);
        double F[C::L + 1];
        boys_eval<C::L>(g.T, boys, g.theta, F);
        C::template vrr<double>(F, g.PA[0], g.PA[1], g.PA[2], g.WP[0], g.WP[1], g.WP[2], g.QC[0], g.QC[1],
                                g.QC[2], g.WQ[0], g.WQ[1], g.WQ[2], g.o2p, g.o2pr, g.o2q, g.o2qr, g.o2pq, acc);
        double cart[NCART], tmp[NCART];
        C::template hrr<double>(acc, A[0] - B[0], A[1] - B[1], A[2] - B[2], A[0] - B[0], A[1] - B[1], A[2] - B[2],
                                cart);
        cart_to_sph4<C::LA, C::LB, C::LC, C::LD>(cart, tmp);
        double m = 0.0;
        for (int i = 0; i < na; i++)
            for (int j = 0; j < nb; j++) m = fmax(m, fabs(cart[((i * nb + j) * na + i) * nb + j]));
        // rounded up so that the float bound stays an upper bound
        q[k] = __double2float_ru(sqrt(m) * (1.0 + 1e-6));
        perm[k] = k;
    }
    // insertion sort of the primitive pairs, descending qp (stable)
    for (int k = 1; k < np; k++) {
        const int pk = perm[k];
        int j = k - 1;
        while (j >= 0 && q[perm[j]] < q[pk]) {
            perm[j + 1] = perm[j];
            j--;
        }
        perm[j + 1] = pk;
    }
    for (int f = 0; f < PP_NF; f++) {
        double v[PIMD_MAXPP];
        for (int k = 0; k < np; k++) v[k] = pp[((size_t)f * PIMD_MAXPP + k) * N + ab];
        for (int k = 0; k < np; k++) pp[((size_t)f * PIMD_MAXPP + k) * N + ab] = v[perm[k]];
    }
    for (int k = 0; k < PIMD_MAXPP; k++) {
        float g = 0.0f;
        if (k < np) {
            const double ea = pp[((size_t)PP_EA * PIMD_MAXPP + k) * N + ab];
            const double eb = pp[((size_t)PP_EB * PIMD_MAXPP + k) * N + ab];
            g = q[perm[k]] * __double2float_ru(2.0 * sqrt(2.0 * fmax(ea, eb)));
        }
        qp[(size_t)k * N + ab] = k < np ? q[perm[k]] : 0.0f;
        qg[(size_t)k * N + ab] = g;
    }
}

}  // namespace pimd
