// Two-electron part of the analytic RHF gradient from derivative ERIs.
//
//   g_X += sum_{mnls} [ 1/2 D_mn D_ls - 1/4 D_ml D_ns ] d(mn|ls)/dX
//
// summed over canonical quartets with weight f = 1/|stabiliser|; the bracket
// summed over the 8 index permutations is Gamma = 4 D_ab D_cd - D_ac D_bd -
// D_ad D_bc. Derivatives of a Cartesian Gaussian with respect to its centre,
//   d/dA_i g_a = 2 alpha g_{a+1_i} - a_i g_{a-1_i},
// are taken for centres A, B and C from one shared Obara-Saika recursion whose
// primitives are accumulated four times (unweighted and weighted by 2 alpha,
// 2 beta, 2 gamma); centre D follows from translational invariance,
// dD = -(dA + dB + dC). Gamma is built in the spherical basis and taken back to
// Cartesian components with the transpose of the spherical transform.
#pragma once
#include "eri_kernels.cuh"

namespace pimd {

// Cartesian exponents of component idx of a shell of angular momentum l
__device__ __forceinline__ void cart_of(int l, int idx, int& lx, int& ly, int& lz)
{
    int n = 0;
    for (int x = l; x >= 0; x--)
        for (int y = l - x; y >= 0; y--) {
            if (n == idx) {
                lx = x;
                ly = y;
                lz = l - x - y;
                return;
            }
            n++;
        }
    lx = ly = lz = 0;
}

__device__ __forceinline__ int cidx(int lx, int ly, int lz)
{
    const int l = lx + ly + lz;
    return (l - lx) * (l - lx + 1) / 2 + lz;
}

// Gamma of one quartet in Cartesian components: Gc[((a*nb+b)*nc+c)*nd+d]
template <int LA, int LB, int LC, int LD, typename R = double>
__device__ __forceinline__ void gamma_cart(double f, int fa, int fb, int fc, int fd, int N,
                                           const double* __restrict__ D, R* Gc, R* tmp)
{
    constexpr int na = nsph(LA), nb = nsph(LB), nc = nsph(LC), nd = nsph(LD);
    for (int a = 0; a < na; a++)
        for (int b = 0; b < nb; b++) {
            const double dab = __ldg(D + (size_t)(fa + a) * N + fb + b);
            for (int c = 0; c < nc; c++) {
                const double dac = __ldg(D + (size_t)(fa + a) * N + fc + c);
                const double dbc = __ldg(D + (size_t)(fb + b) * N + fc + c);
                for (int d = 0; d < nd; d++) {
                    const double dcd = __ldg(D + (size_t)(fc + c) * N + fd + d);
                    const double dbd = __ldg(D + (size_t)(fb + b) * N + fd + d);
                    const double dad = __ldg(D + (size_t)(fa + a) * N + fd + d);
                    Gc[((a * nb + b) * nc + c) * nd + d] = R(f * (4.0 * dab * dcd - dac * dbd - dad * dbc));
                }
            }
        }
    sph_to_cart4_t<LA, LB, LC, LD>(Gc, tmp);
}

// sum_{abcd} Gc * d(ab|cd)/dX_i for X at position POS (0: A, 1: B, 2: C), given
// accessors for the raised (l+1) and lowered (l-1) blocks of that position.
template <int LA, int LB, int LC, int LD, int POS, class Up, class Dn, typename R = double>
__device__ __forceinline__ void contract_deriv(const R* Gc, Up up, Dn dn, R g[3])
{
    constexpr int L[4] = {LA, LB, LC, LD};
    constexpr int n[4] = {ncart(LA), ncart(LB), ncart(LC), ncart(LD)};
    int nu[4] = {n[0], n[1], n[2], n[3]};
    int ndn[4] = {n[0], n[1], n[2], n[3]};
    nu[POS] = ncart(L[POS] + 1);
    ndn[POS] = L[POS] > 0 ? ncart(L[POS] - 1) : 1;
    g[0] = g[1] = g[2] = R(0);
    for (int i0 = 0; i0 < n[0]; i0++)
        for (int i1 = 0; i1 < n[1]; i1++)
            for (int i2 = 0; i2 < n[2]; i2++)
                for (int i3 = 0; i3 < n[3]; i3++) {
                    const R gm = Gc[((i0 * n[1] + i1) * n[2] + i2) * n[3] + i3];
                    int idx[4] = {i0, i1, i2, i3};
                    int e[3];
                    cart_of(L[POS], idx[POS], e[0], e[1], e[2]);
#pragma unroll
                    for (int x = 0; x < 3; x++) {
                        int eu[3] = {e[0], e[1], e[2]};
                        eu[x]++;
                        int ju[4] = {i0, i1, i2, i3};
                        ju[POS] = cidx(eu[0], eu[1], eu[2]);
                        R v = up(((ju[0] * nu[1] + ju[1]) * nu[2] + ju[2]) * nu[3] + ju[3]);
                        if (e[x] > 0) {
                            int ed[3] = {e[0], e[1], e[2]};
                            ed[x]--;
                            int jd[4] = {i0, i1, i2, i3};
                            jd[POS] = cidx(ed[0], ed[1], ed[2]);
                            v -= e[x] * dn(((jd[0] * ndn[1] + jd[1]) * ndn[2] + jd[2]) * ndn[3] + jd[3]);
                        }
                        g[x] += gm * v;
                    }
                }
}

template <typename R = double>
struct ArrAcc {
    const R* p;
    __device__ __forceinline__ R operator()(int i) const { return p[i]; }
};


template <typename R>
__device__ __forceinline__ void scatter_grad(double* grad, const Shells& S, int sa, int sb, int sc, int sd,
                                             const R gA[3], const R gB[3], const R gC[3], double fxs)
{
    const int aa = S.atom[sa], ab = S.atom[sb], ac = S.atom[sc], ad = S.atom[sd];
#pragma unroll
    for (int x = 0; x < 3; x++) {
        const double a = gA[x], b = gB[x], c = gC[x];
        det_add(grad + 3 * aa + x, a, fxs);
        det_add(grad + 3 * ab + x, b, fxs);
        det_add(grad + 3 * ac + x, c, fxs);
        det_add(grad + 3 * ad + x, -(a + b + c), fxs);
    }
}

// bound of |Gamma| over a quartet from the shell-pair density bounds
__device__ __forceinline__ double gamma_bound(const Reps& R, const double* Dsh, int r, int sa, int sb, int sc, int sd)
{
    const double j = shell_bound(R, Dsh, r, sa, sb) * shell_bound(R, Dsh, r, sc, sd);
    const double k1 = shell_bound(R, Dsh, r, sa, sc) * shell_bound(R, Dsh, r, sb, sd);
    const double k2 = shell_bound(R, Dsh, r, sa, sd) * shell_bound(R, Dsh, r, sb, sc);
    return 4.0 * j + k1 + k2;
}

// Straight-line gradient kernel (generated VRR/HRR) in precision R for the
// quartets whose bound Q_ab Q_cd |Gamma| lies in [tau_lo, tau_hi).
// blockDim.x >= the tile's ket width.
// Primitive screening: primitive quartet (i|j) is skipped when
// (qg_i qp_j + qp_i qg_j) |Gamma| < tau_prim (qg: the derivative scale of a
// primitive pair); tau_prim = 0 keeps every primitive quartet.
template <class G, typename R>
__global__ void __launch_bounds__(128) grad2e_kernel(Pairs P, Shells S, Reps Rp, const Tile* __restrict__ tiles,
                                                     const double* __restrict__ Dall, double* __restrict__ grad,
                                                     const R* __restrict__ boys, double tau_lo, double tau_hi,
                                                     const double* __restrict__ Dsh,
                                                     unsigned long long* __restrict__ cnt, double tau_prim,
                                                     double fxs)
{
    constexpr int LA = G::LA, LB = G::LB, LC = G::LC, LD = G::LD;
    __shared__ R sbra[PP_NF][PIMD_MAXPP];
    __shared__ float sqp[PIMD_MAXPP], sqg[PIMD_MAXPP];
    const Tile t = tiles[blockIdx.x];
    const int ab = t.ab;
    for (int e = threadIdx.x; e < PP_NF * PIMD_MAXPP; e += blockDim.x) {
        const int f = e / PIMD_MAXPP, k = e % PIMD_MAXPP;
        sbra[f][k] = pp_base(P, R(0))[((size_t)f * PIMD_MAXPP + k) * P.n + ab];
    }
    if (threadIdx.x < PIMD_MAXPP) {
        sqp[threadIdx.x] = P.qp[(size_t)threadIdx.x * P.n + ab];
        sqg[threadIdx.x] = P.qg[(size_t)threadIdx.x * P.n + ab];
    }
    __syncthreads();
    const int sa = P.sa[ab], sb = P.sb[ab];
    const int nbra = P.npp[ab];
    // screening of ket pair c0 + k (quartet bound Q_ab Q_cd |Gamma|) and the
    // primitive cutoff over |Gamma|
    auto screen = [&](int k, int& cd, double& gam, float& gthr) -> bool {
        cd = t.c0 + k;
        gam = 0.0;
        gthr = 0.0f;
        if (cd >= t.c1) return false;
        gam = gamma_bound(Rp, Dsh, t.rep, sa, sb, P.sa[cd], P.sb[cd]);
        const double bound = P.Q[ab] * P.Q[cd] * gam;
        gthr = (float)(tau_prim / gam);
        return bound >= tau_lo && bound < tau_hi;
    };
    int cd;
    double gam;
    float gthr;
    bool work = screen(threadIdx.x, cd, gam, gthr);
    if (tau_prim > 0.0 && blockDim.x > 32) {
        // regroup the block's quartets by their number of surviving primitive
        // quartets (bitonic sort, descending): lanes stop at their own cutoff
        // and a warp issues for all its lanes
        __shared__ int skey[128], sidx[128];
        int est = -1;
        if (work) {
            est = 0;
            const int nket = P.npp[cd];
            for (int j = 0; j < nket; j++) {
                const float qpj = __ldg(P.qp + (size_t)j * P.n + cd), qgj = __ldg(P.qg + (size_t)j * P.n + cd);
                for (int i = 0; i < nbra; i++) est += sqg[i] * qpj + sqp[i] * qgj >= gthr;
            }
        }
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
        work = screen(sidx[tid], cd, gam, gthr);
    }
    // the lane's surviving primitive quartets, walked as one flat sequence
    // (row-major over (j, i)) for kmax steps, kmax the longest of the warp
    auto survives = [&](int i, float qpj, float qgj) { return sqg[i] * qpj + sqp[i] * qgj >= gthr; };
    int total = 0;
    if (work) {
        const int nk = P.npp[cd];
        for (int j = 0; j < nk; j++) {
            const float qpj = __ldg(P.qp + (size_t)j * P.n + cd), qgj = __ldg(P.qg + (size_t)j * P.n + cd);
            for (int i = 0; i < nbra; i++) total += survives(i, qpj, qgj);
        }
    }
    const int kmax = __reduce_max_sync(0xffffffffu, (unsigned)total);
    {
        // executed quartets and primitive quartets (one atomic pair per warp)
        const unsigned nq = __reduce_add_sync(0xffffffffu, work ? 1u : 0u);
        const unsigned np = __reduce_add_sync(0xffffffffu, (unsigned)total);
        if ((threadIdx.x & 31) == 0 && nq) {
            atomicAdd(cnt, (unsigned long long)nq);
            atomicAdd(cnt + 1, (unsigned long long)np);
        }
    }
    if (!work) return;
    const int sc = P.sa[cd], sd = P.sb[cd];
    double A[3], B[3], Cc[3], Dd[3];
#pragma unroll
    for (int x = 0; x < 3; x++) {
        A[x] = S.xyz[3 * sa + x];
        B[x] = S.xyz[3 * sb + x];
        Cc[x] = S.xyz[3 * sc + x];
        Dd[x] = S.xyz[3 * sd + x];
    }
    R accU[G::N_accU], accA[G::N_accA], accB[G::N_accB], accC[G::N_accC];
    for (int i = 0; i < G::N_accU; i++) accU[i] = R(0);
    for (int i = 0; i < G::N_accA; i++) accA[i] = R(0);
    for (int i = 0; i < G::N_accB; i++) accB[i] = R(0);
    for (int i = 0; i < G::N_accC; i++) accC[i] = R(0);
    const int nket = P.npp[cd];
    int i = 0, j = 0, jl = -1;
    float qpj = __ldg(P.qp + cd), qgj = __ldg(P.qg + cd);
    R ket[PP_NF];
    for (int k = 0; k < kmax; k++) {
        if (k < total) {
            // advance to the next surviving primitive quartet (one exists: k < total)
            while (!survives(i, qpj, qgj)) {
                if (++i == nbra) {
                    i = 0;
                    ++j;
                    qpj = __ldg(P.qp + (size_t)j * P.n + cd);
                    qgj = __ldg(P.qg + (size_t)j * P.n + cd);
                }
            }
            if (j != jl) {
                load_ppn(P, cd, j, ket, PP_NF);
                jl = j;
            }
            R bra[PP_NERI];
#pragma unroll
            for (int f = 0; f < PP_NERI; f++) bra[f] = sbra[f][i];
            PrimQ<R> g;
            prim_quartet<R>(bra, ket, g);
            R F[G::L + 1];
            boys_eval<G::L>(g.T, boys, g.theta, F);
            G::template vrr<R>(F, g.PA[0], g.PA[1], g.PA[2], g.WP[0], g.WP[1], g.WP[2], g.QC[0], g.QC[1], g.QC[2],
                               g.WQ[0], g.WQ[1], g.WQ[2], g.o2p, g.o2pr, g.o2q, g.o2qr, g.o2pq, accU, accA, accB,
                               accC, R(2) * sbra[PP_EA][i], R(2) * sbra[PP_EB][i], R(2) * ket[PP_EA]);
            if (++i == nbra && j + 1 < nket) {
                i = 0;
                ++j;
                qpj = __ldg(P.qp + (size_t)j * P.n + cd);
                qgj = __ldg(P.qg + (size_t)j * P.n + cd);
            }
        }
    }
    const R AB0 = R(A[0] - B[0]), AB1 = R(A[1] - B[1]), AB2 = R(A[2] - B[2]);
    const R CD0 = R(Cc[0] - Dd[0]), CD1 = R(Cc[1] - Dd[1]), CD2 = R(Cc[2] - Dd[2]);
    constexpr int NC = ncart(LA) * ncart(LB) * ncart(LC) * ncart(LD);
    R Gc[NC], tmp[NC];
    double f = 1.0;
    if (sa == sb) f *= 0.5;
    if (sc == sd) f *= 0.5;
    if (ab == cd) f *= 0.5;
    const int r = t.rep;
    gamma_cart<LA, LB, LC, LD, R>(f, S.bf[sa], S.bf[sb], S.bf[sc], S.bf[sd], Rp.nbf[r], Dall + Rp.moff[r], Gc,
                                  tmp);
    R gA[3], gB[3], gC[3];
    {
        R up[ncart(LA + 1) * ncart(LB) * ncart(LC) * ncart(LD)];
        G::template hrrAp<R>(accA, AB0, AB1, AB2, CD0, CD1, CD2, up);
        if constexpr (LA > 0) {
            R dn[ncart(LA > 0 ? LA - 1 : 0) * ncart(LB) * ncart(LC) * ncart(LD)];
            G::template hrrAm<R>(accU, AB0, AB1, AB2, CD0, CD1, CD2, dn);
            contract_deriv<LA, LB, LC, LD, 0>(Gc, ArrAcc<R>{up}, ArrAcc<R>{dn}, gA);
        } else {
            contract_deriv<LA, LB, LC, LD, 0>(Gc, ArrAcc<R>{up}, ArrAcc<R>{up}, gA);
        }
    }
    {
        R up[ncart(LA) * ncart(LB + 1) * ncart(LC) * ncart(LD)];
        G::template hrrBp<R>(accB, AB0, AB1, AB2, CD0, CD1, CD2, up);
        if constexpr (LB > 0) {
            R dn[ncart(LA) * ncart(LB > 0 ? LB - 1 : 0) * ncart(LC) * ncart(LD)];
            G::template hrrBm<R>(accU, AB0, AB1, AB2, CD0, CD1, CD2, dn);
            contract_deriv<LA, LB, LC, LD, 1>(Gc, ArrAcc<R>{up}, ArrAcc<R>{dn}, gB);
        } else {
            contract_deriv<LA, LB, LC, LD, 1>(Gc, ArrAcc<R>{up}, ArrAcc<R>{up}, gB);
        }
    }
    {
        R up[ncart(LA) * ncart(LB) * ncart(LC + 1) * ncart(LD)];
        G::template hrrCp<R>(accC, AB0, AB1, AB2, CD0, CD1, CD2, up);
        if constexpr (LC > 0) {
            R dn[ncart(LA) * ncart(LB) * ncart(LC > 0 ? LC - 1 : 0) * ncart(LD)];
            G::template hrrCm<R>(accU, AB0, AB1, AB2, CD0, CD1, CD2, dn);
            contract_deriv<LA, LB, LC, LD, 2>(Gc, ArrAcc<R>{up}, ArrAcc<R>{dn}, gC);
        } else {
            contract_deriv<LA, LB, LC, LD, 2>(Gc, ArrAcc<R>{up}, ArrAcc<R>{up}, gC);
        }
    }
    scatter_grad(grad, S, sa, sb, sc, sd, gA, gB, gC, fxs);
}

}  // namespace pimd
