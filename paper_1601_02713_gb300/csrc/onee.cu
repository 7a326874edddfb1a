// One-electron integrals (overlap, kinetic, nuclear attraction), their
// derivatives for the analytic gradient, primitive-pair data, the nuclear
// repulsion, and the Boys table.
//
// Obara-Saika recursions (Obara & Saika, J. Chem. Phys. 84, 3963 (1986)),
// one direction at a time for the overlap,
//   S(i+1, j) = PA S(i, j) + [i S(i-1, j) + j S(i, j-1)] / (2p),
//   S(i, j+1) = PB S(i, j) + [i S(i-1, j) + j S(i, j-1)] / (2p),
// the kinetic energy as (1/2) <grad a | grad b>,
//   T(i, j) = 1/2 [ i j S(i-1,j-1) - 2a j S(i+1,j-1) - 2b i S(i-1,j+1) + 4ab S(i+1,j+1) ],
// and the nuclear attraction with auxiliary orders m,
//   V^m(a+1_i, b) = PA_i V^m(a,b) - PC_i V^{m+1}(a,b)
//                   + a_i/(2p) [V^m(a-1_i,b) - V^{m+1}(a-1_i,b)] + b_i/(2p) [V^m(a,b-1_i) - V^{m+1}(a,b-1_i)],
//   V^m(0,0) = (2 pi / p) K F_m(p |PC|^2)     (and the same rule for b+1_i with PB).
#include <math.h>

#include "boys.cuh"
#include "internal.h"

namespace pimd {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int NA1 = 20;   // Cartesian components of levels 0..3
constexpr int NB1 = 10;   // levels 0..2
constexpr int NM1 = 6;

__device__ __forceinline__ int loff(int l) { return l * (l + 1) * (l + 2) / 6; }
__device__ __forceinline__ int gidx(int x, int y, int z)
{
    const int l = x + y + z;
    return loff(l) + (l - x) * (l - x + 1) / 2 + z;
}

__device__ __forceinline__ int cidx_host_dev(const int* e)
{
    const int l = e[0] + e[1] + e[2];
    return (l - e[0]) * (l - e[0] + 1) / 2 + e[2];
}

__device__ __forceinline__ void cart_of_d(int l, int idx, int* e)
{
    int n = 0;
    for (int x = l; x >= 0; x--)
        for (int y = l - x; y >= 0; y--) {
            if (n == idx) {
                e[0] = x;
                e[1] = y;
                e[2] = l - x - y;
                return;
            }
            n++;
        }
}

__device__ __forceinline__ int dir_of(const int* e)
{
    return (e[0] >= e[1] && e[0] >= e[2]) ? 0 : (e[1] >= e[2] ? 1 : 2);
}

// V^m(a, b) tables for a levels 0..la, b levels 0..lb (m = 0 of levels la, lb
// are the attraction integrals). Vt[(m * NA1 + ia) * NB1 + ib].
__device__ void os_nuclear(int la, int lb, double p, const double* PA, const double* PB, const double* PC,
                           const double* F, double pref, double* Vt)
{
    const int Lt = la + lb;
    const double o2p = 0.5 / p;
    for (int m = 0; m <= Lt; m++) Vt[(m * NA1 + 0) * NB1 + 0] = pref * F[m];
    for (int l = 1; l <= la; l++) {
        for (int c = 0; c < (l + 1) * (l + 2) / 2; c++) {
            int e[3];
            cart_of_d(l, c, e);
            const int i = dir_of(e);
            int e1[3] = {e[0], e[1], e[2]};
            e1[i]--;
            const int ia = gidx(e[0], e[1], e[2]), i1 = gidx(e1[0], e1[1], e1[2]);
            int i2 = -1;
            if (e1[i] > 0) {
                int e2[3] = {e1[0], e1[1], e1[2]};
                e2[i]--;
                i2 = gidx(e2[0], e2[1], e2[2]);
            }
            for (int m = 0; m <= Lt - l; m++) {
                double v = PA[i] * Vt[(m * NA1 + i1) * NB1] - PC[i] * Vt[((m + 1) * NA1 + i1) * NB1];
                if (i2 >= 0) v += e1[i] * o2p * (Vt[(m * NA1 + i2) * NB1] - Vt[((m + 1) * NA1 + i2) * NB1]);
                Vt[(m * NA1 + ia) * NB1] = v;
            }
        }
    }
    for (int lbb = 1; lbb <= lb; lbb++) {
        for (int cb = 0; cb < (lbb + 1) * (lbb + 2) / 2; cb++) {
            int f[3];
            cart_of_d(lbb, cb, f);
            const int i = dir_of(f);
            int f1[3] = {f[0], f[1], f[2]};
            f1[i]--;
            const int ib = gidx(f[0], f[1], f[2]), j1 = gidx(f1[0], f1[1], f1[2]);
            int j2 = -1;
            if (f1[i] > 0) {
                int f2[3] = {f1[0], f1[1], f1[2]};
                f2[i]--;
                j2 = gidx(f2[0], f2[1], f2[2]);
            }
            for (int l = 0; l <= la; l++)
                for (int c = 0; c < (l + 1) * (l + 2) / 2; c++) {
                    int e[3];
                    cart_of_d(l, c, e);
                    const int ia = gidx(e[0], e[1], e[2]);
                    int ia1 = -1;
                    if (e[i] > 0) {
                        int e1[3] = {e[0], e[1], e[2]};
                        e1[i]--;
                        ia1 = gidx(e1[0], e1[1], e1[2]);
                    }
                    for (int m = 0; m <= Lt - l - lbb; m++) {
                        double v = PB[i] * Vt[(m * NA1 + ia) * NB1 + j1] - PC[i] * Vt[((m + 1) * NA1 + ia) * NB1 + j1];
                        if (ia1 >= 0)
                            v += e[i] * o2p * (Vt[(m * NA1 + ia1) * NB1 + j1] - Vt[((m + 1) * NA1 + ia1) * NB1 + j1]);
                        if (j2 >= 0)
                            v += f1[i] * o2p * (Vt[(m * NA1 + ia) * NB1 + j2] - Vt[((m + 1) * NA1 + ia) * NB1 + j2]);
                        Vt[(m * NA1 + ia) * NB1 + ib] = v;
                    }
                }
        }
    }
}

// 1-D overlap table S[i][j], i <= imax, j <= jmax (without the (pi/p)^{1/2} K factor)
__device__ void os_overlap_1d(int imax, int jmax, double PA, double PB, double p, double S[6][5])
{
    const double o2p = 0.5 / p;
    S[0][0] = 1.0;
    for (int i = 0; i <= imax; i++)
        for (int j = 0; j <= jmax; j++) {
            if (i == 0 && j == 0) continue;
            double v;
            if (i > 0) {
                v = PA * S[i - 1][j];
                if (i > 1) v += (i - 1) * o2p * S[i - 2][j];
                if (j > 0) v += j * o2p * S[i - 1][j - 1];
            } else {
                v = PB * S[i][j - 1];
                if (j > 1) v += (j - 1) * o2p * S[i][j - 2];
            }
            S[i][j] = v;
        }
}

__device__ __forceinline__ double kin_1d(const double S[6][5], int i, int j, double a, double b)
{
    double t = 4.0 * a * b * S[i + 1][j + 1];
    if (i > 0 && j > 0) t += i * j * S[i - 1][j - 1];
    if (j > 0) t -= 2.0 * a * j * S[i + 1][j - 1];
    if (i > 0) t -= 2.0 * b * i * S[i - 1][j + 1];
    return 0.5 * t;
}

// 2-index Cartesian -> spherical transform of block[na_c][nb_c] in place
__device__ void sph2(int la, int lb, double* blk)
{
    const double s3 = 1.7320508075688772935;
    const int nac = (la + 1) * (la + 2) / 2, nbc = (lb + 1) * (lb + 2) / 2;
    double tmp[36];
    int nas = nac;
    if (la == 2) {
        for (int j = 0; j < nbc; j++) {
            const double xx = blk[0 * nbc + j], xy = blk[1 * nbc + j], xz = blk[2 * nbc + j], yy = blk[3 * nbc + j],
                         yz = blk[4 * nbc + j], zz = blk[5 * nbc + j];
            tmp[0 * nbc + j] = s3 * xy;
            tmp[1 * nbc + j] = s3 * yz;
            tmp[2 * nbc + j] = zz - 0.5 * (xx + yy);
            tmp[3 * nbc + j] = s3 * xz;
            tmp[4 * nbc + j] = 0.5 * s3 * (xx - yy);
        }
        nas = 5;
        for (int k = 0; k < nas * nbc; k++) blk[k] = tmp[k];
    }
    if (lb == 2) {
        for (int i = 0; i < nas; i++) {
            const double* r = blk + i * 6;
            const double xx = r[0], xy = r[1], xz = r[2], yy = r[3], yz = r[4], zz = r[5];
            tmp[i * 5 + 0] = s3 * xy;
            tmp[i * 5 + 1] = s3 * yz;
            tmp[i * 5 + 2] = zz - 0.5 * (xx + yy);
            tmp[i * 5 + 3] = s3 * xz;
            tmp[i * 5 + 4] = 0.5 * s3 * (xx - yy);
        }
        for (int k = 0; k < nas * 5; k++) blk[k] = tmp[k];
    }
}

// spherical block [na_s][nb_s] -> Cartesian-component weights [na_c][nb_c]
// (transpose transform: sum_sph X_s I_s = sum_cart X_c I_c)
__device__ void sph2_t(int la, int lb, const double* in, double* out)
{
    const double s3 = 1.7320508075688772935;
    const int nac = (la + 1) * (la + 2) / 2, nbc = (lb + 1) * (lb + 2) / 2;
    const int nas = la == 2 ? 5 : nac, nbs = lb == 2 ? 5 : nbc;
    double tmp[36];
    // first index
    for (int j = 0; j < nbs; j++) {
        if (la == 2) {
            const double m2 = in[0 * nbs + j], m1 = in[1 * nbs + j], m0 = in[2 * nbs + j], p1 = in[3 * nbs + j],
                         p2 = in[4 * nbs + j];
            tmp[0 * nbs + j] = -0.5 * m0 + 0.5 * s3 * p2;
            tmp[1 * nbs + j] = s3 * m2;
            tmp[2 * nbs + j] = s3 * p1;
            tmp[3 * nbs + j] = -0.5 * m0 - 0.5 * s3 * p2;
            tmp[4 * nbs + j] = s3 * m1;
            tmp[5 * nbs + j] = m0;
        } else {
            for (int i = 0; i < nac; i++) tmp[i * nbs + j] = in[i * nbs + j];
        }
    }
    for (int i = 0; i < nac; i++) {
        if (lb == 2) {
            const double* r = tmp + i * 5;
            const double m2 = r[0], m1 = r[1], m0 = r[2], p1 = r[3], p2 = r[4];
            double* o = out + i * 6;
            o[0] = -0.5 * m0 + 0.5 * s3 * p2;
            o[1] = s3 * m2;
            o[2] = s3 * p1;
            o[3] = -0.5 * m0 - 0.5 * s3 * p2;
            o[4] = s3 * m1;
            o[5] = m0;
        } else {
            for (int j = 0; j < nbc; j++) out[i * nbc + j] = tmp[i * nbc + j];
        }
    }
}

__global__ void pair_data_kernel(Pairs P, int* npp, double* pp, Shells S, BasisPrimDev B)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P.n) return;
    const int a = P.sa[g], b = P.sb[g];
    const int pa = B.sprim[a], pb = B.sprim[b], na = B.snprim[a], nb = B.snprim[b];
    double AB2 = 0.0;
    double A[3], Bc[3];
    for (int x = 0; x < 3; x++) {
        A[x] = S.xyz[3 * a + x];
        Bc[x] = S.xyz[3 * b + x];
        AB2 += (A[x] - Bc[x]) * (A[x] - Bc[x]);
    }
    const double c0 = 1.4142135623730950488 * pow(kPi, 1.25);
    // primitive pairs whose prefactor is below 1e-17 of the pair's largest
    // one are dropped (their share of any integral is below double rounding)
    double kmax = 0.0;
    for (int i = 0; i < na; i++)
        for (int j = 0; j < nb; j++) {
            const double ea = B.exps[pa + i], eb = B.exps[pb + j];
            kmax = fmax(kmax, fabs(B.coefs[pa + i] * B.coefs[pb + j] * exp(-ea * eb / (ea + eb) * AB2) / (ea + eb)));
        }
    int k = 0;
    for (int i = 0; i < na; i++)
        for (int j = 0; j < nb; j++) {
            const double ea = B.exps[pa + i], eb = B.exps[pb + j];
            const double p = ea + eb, ip = 1.0 / p;
            const double kij = B.coefs[pa + i] * B.coefs[pb + j] * exp(-ea * eb * ip * AB2) * ip;
            if (fabs(kij) < 1e-17 * kmax) continue;
            const double Px = (ea * A[0] + eb * Bc[0]) * ip, Py = (ea * A[1] + eb * Bc[1]) * ip,
                         Pz = (ea * A[2] + eb * Bc[2]) * ip;
            const double vals[PP_NF] = {p,  Px, Py, Pz, c0 * kij, Px - A[0], Py - A[1], Pz - A[2],
                                        0.5 * ip, 0.5 * ip * ip, ea, eb};
            for (int f = 0; f < PP_NF; f++) pp[((size_t)f * PIMD_MAXPP + k) * P.n + g] = vals[f];
            k++;
        }
    npp[g] = k;
}

// Cartesian S, T, V blocks of bra shell a (raised by dla with weight 2 alpha if
// wa) and ket shell b, contracted. The nuclear attraction is summed over the
// nuclei [c0, c1) unless single >= 0 (then only nucleus `single`).
__device__ void one_e_blocks(int sa, int sb, int la, int lb, const Shells& S, const BasisPrimDev& B,
                             const AtomsDev& At, int c0, int c1, const double* boys, double* Sb, double* Tb,
                             double* Vb, bool want_st)
{
    const int nac = (la + 1) * (la + 2) / 2, nbc = (lb + 1) * (lb + 2) / 2;
    for (int k = 0; k < nac * nbc; k++) {
        if (want_st) {
            Sb[k] = 0.0;
            Tb[k] = 0.0;
        }
        Vb[k] = 0.0;
    }
    double A[3], Bc[3], AB2 = 0.0;
    for (int x = 0; x < 3; x++) {
        A[x] = S.xyz[3 * sa + x];
        Bc[x] = S.xyz[3 * sb + x];
        AB2 += (A[x] - Bc[x]) * (A[x] - Bc[x]);
    }
    const int pa = B.sprim[sa], pb = B.sprim[sb];
    for (int i = 0; i < B.snprim[sa]; i++)
        for (int j = 0; j < B.snprim[sb]; j++) {
            const double a = B.exps[pa + i], b = B.exps[pb + j];
            const double p = a + b;
            const double K = B.coefs[pa + i] * B.coefs[pb + j] * exp(-a * b / p * AB2);
            double P[3], PA[3], PB[3];
            for (int x = 0; x < 3; x++) {
                P[x] = (a * A[x] + b * Bc[x]) / p;
                PA[x] = P[x] - A[x];
                PB[x] = P[x] - Bc[x];
            }
            if (want_st) {
                double S1[3][6][5];
                for (int x = 0; x < 3; x++) os_overlap_1d(la + 1, lb + 1, PA[x], PB[x], p, S1[x]);
                const double pre = K * pow(kPi / p, 1.5);
                for (int ia = 0; ia < nac; ia++) {
                    int e[3];
                    cart_of_d(la, ia, e);
                    for (int ib = 0; ib < nbc; ib++) {
                        int f[3];
                        cart_of_d(lb, ib, f);
                        const double sx = S1[0][e[0]][f[0]], sy = S1[1][e[1]][f[1]], sz = S1[2][e[2]][f[2]];
                        const double tx = kin_1d(S1[0], e[0], f[0], a, b), ty = kin_1d(S1[1], e[1], f[1], a, b),
                                     tz = kin_1d(S1[2], e[2], f[2], a, b);
                        Sb[ia * nbc + ib] += pre * sx * sy * sz;
                        Tb[ia * nbc + ib] += pre * (tx * sy * sz + sx * ty * sz + sx * sy * tz);
                    }
                }
            }
            double Vt[NM1 * NA1 * NB1];
            for (int c = c0; c < c1; c++) {
                double PC[3], PC2 = 0.0;
                for (int x = 0; x < 3; x++) {
                    PC[x] = P[x] - At.xyz[3 * c + x];
                    PC2 += PC[x] * PC[x];
                }
                double F[NM1];
                boys_eval_n(la + lb, p * PC2, boys, 1.0, F);
                os_nuclear(la, lb, p, PA, PB, PC, F, -At.Z[c] * 2.0 * kPi / p * K, Vt);
                for (int ia = 0; ia < nac; ia++) {
                    int e[3];
                    cart_of_d(la, ia, e);
                    const int ga = gidx(e[0], e[1], e[2]);
                    for (int ib = 0; ib < nbc; ib++) {
                        int f[3];
                        cart_of_d(lb, ib, f);
                        Vb[ia * nbc + ib] += Vt[(0 * NA1 + ga) * NB1 + gidx(f[0], f[1], f[2])];
                    }
                }
            }
        }
}

__global__ void one_e_kernel(Pairs P, Shells S, BasisPrimDev B, AtomsDev At, Reps R, double* Sm, double* Tm,
                             double* Vm, const double* boys)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P.n) return;
    const int sa = P.sa[g], sb = P.sb[g];
    const int la = S.l[sa], lb = S.l[sb];
    const int r = S.rep[sa];
    double Sb[36], Tb[36], Vb[36];
    one_e_blocks(sa, sb, la, lb, S, B, At, At.rep_atom0[r], At.rep_atom0[r + 1], boys, Sb, Tb, Vb, true);
    sph2(la, lb, Sb);
    sph2(la, lb, Tb);
    sph2(la, lb, Vb);
    const int na = nsph(la), nb = nsph(lb);
    const int N = R.nbf[r];
    const size_t off = R.moff[r];
    const int fa = S.bf[sa], fb = S.bf[sb];
    for (int i = 0; i < na; i++)
        for (int j = 0; j < nb; j++) {
            const size_t u = off + (size_t)(fa + i) * N + fb + j, v = off + (size_t)(fb + j) * N + fa + i;
            Sm[u] = Sb[i * nb + j];
            Sm[v] = Sb[i * nb + j];
            Tm[u] = Tb[i * nb + j];
            Tm[v] = Tb[i * nb + j];
            Vm[u] = Vb[i * nb + j];
            Vm[v] = Vb[i * nb + j];
        }
}

// derivative of the bra Gaussian: d/dA_x g_a = 2 alpha g_{a+1_x} - a_x g_{a-1_x}
// One thread per (pair, orientation).
__global__ void grad_1e_kernel(Pairs P, Shells S, BasisPrimDev B, AtomsDev At, Reps R, const double* D,
                               const double* W, double* grad, const double* boys, double fxs)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * P.n) return;
    const int g = t >> 1, orient = t & 1;
    int sa = P.sa[g], sb = P.sb[g];
    if (orient) {
        if (sa == sb) return;
        const int tmp = sa;
        sa = sb;
        sb = tmp;
    }
    const int la = S.l[sa], lb = S.l[sb];
    const int r = S.rep[sa];
    const int N = R.nbf[r];
    const size_t off = R.moff[r];
    const int fa = S.bf[sa], fb = S.bf[sb];
    const int nas = nsph(la), nbs = nsph(lb);
    const int nac = ncart(la), nbc = ncart(lb);
    // density and energy-weighted density blocks in Cartesian-component form
    double Ds[25], Ws[25], Dc[36], Wc[36];
    for (int i = 0; i < nas; i++)
        for (int j = 0; j < nbs; j++) {
            Ds[i * nbs + j] = D[off + (size_t)(fa + i) * N + fb + j];
            Ws[i * nbs + j] = W[off + (size_t)(fa + i) * N + fb + j];
        }
    sph2_t(la, lb, Ds, Dc);
    sph2_t(la, lb, Ws, Wc);
    const int c0 = At.rep_atom0[r], c1 = At.rep_atom0[r + 1];
    const int atom_a = S.atom[sa];
    double ga[3] = {0.0, 0.0, 0.0};
    // raised and lowered bra blocks of one bra primitive (the weight 2 alpha
    // is per primitive): S, T summed over nuclei, V per nucleus
    double Su[60], Tu[60], Vu[60], Sd[18], Td[18], Vd[18];
    const int pa = B.sprim[sa];
    const int ncu = ncart(la + 1), ncd = la > 0 ? ncart(la - 1) : 0;
    // S and T derivative parts
    {
        double dS[3][36], dT[3][36];
        for (int x = 0; x < 3; x++)
            for (int k = 0; k < nac * nbc; k++) dS[x][k] = dT[x][k] = 0.0;
        for (int i = 0; i < B.snprim[sa]; i++) {
            const double a = B.exps[pa + i];
            // raised
            {
                double A[3], Bc[3], AB2 = 0.0;
                for (int x = 0; x < 3; x++) {
                    A[x] = S.xyz[3 * sa + x];
                    Bc[x] = S.xyz[3 * sb + x];
                    AB2 += (A[x] - Bc[x]) * (A[x] - Bc[x]);
                }
                const int pb = B.sprim[sb];
                for (int k = 0; k < ncu * nbc; k++) Su[k] = Tu[k] = 0.0;
                for (int k = 0; k < ncd * nbc; k++) Sd[k] = Td[k] = 0.0;
                for (int j = 0; j < B.snprim[sb]; j++) {
                    const double b = B.exps[pb + j];
                    const double p = a + b;
                    const double K = B.coefs[pa + i] * B.coefs[pb + j] * exp(-a * b / p * AB2);
                    double PA[3], PB[3];
                    for (int x = 0; x < 3; x++) {
                        const double Px = (a * A[x] + b * Bc[x]) / p;
                        PA[x] = Px - A[x];
                        PB[x] = Px - Bc[x];
                    }
                    double S1[3][6][5];
                    for (int x = 0; x < 3; x++) os_overlap_1d(la + 2, lb + 1, PA[x], PB[x], p, S1[x]);
                    const double pre = K * pow(kPi / p, 1.5);
                    for (int lev = 0; lev < 2; lev++) {
                        const int lq = lev == 0 ? la + 1 : la - 1;
                        if (lq < 0) continue;
                        const int nq = ncart(lq);
                        for (int ia = 0; ia < nq; ia++) {
                            int e[3];
                            cart_of_d(lq, ia, e);
                            for (int ib = 0; ib < nbc; ib++) {
                                int f[3];
                                cart_of_d(lb, ib, f);
                                const double sx = S1[0][e[0]][f[0]], sy = S1[1][e[1]][f[1]], sz = S1[2][e[2]][f[2]];
                                const double tx = kin_1d(S1[0], e[0], f[0], a, b),
                                             ty = kin_1d(S1[1], e[1], f[1], a, b),
                                             tz = kin_1d(S1[2], e[2], f[2], a, b);
                                const double s = pre * sx * sy * sz;
                                const double tk = pre * (tx * sy * sz + sx * ty * sz + sx * sy * tz);
                                if (lev == 0) {
                                    Su[ia * nbc + ib] += s;
                                    Tu[ia * nbc + ib] += tk;
                                } else {
                                    Sd[ia * nbc + ib] += s;
                                    Td[ia * nbc + ib] += tk;
                                }
                            }
                        }
                    }
                }
                for (int ia = 0; ia < nac; ia++) {
                    int e[3];
                    cart_of_d(la, ia, e);
                    for (int x = 0; x < 3; x++) {
                        int eu[3] = {e[0], e[1], e[2]};
                        eu[x]++;
                        const int iu = cidx_host_dev(eu);
                        for (int ib = 0; ib < nbc; ib++) {
                            double vs = 2.0 * a * Su[iu * nbc + ib], vt = 2.0 * a * Tu[iu * nbc + ib];
                            if (e[x] > 0) {
                                int ed[3] = {e[0], e[1], e[2]};
                                ed[x]--;
                                const int id = cidx_host_dev(ed);
                                vs -= e[x] * Sd[id * nbc + ib];
                                vt -= e[x] * Td[id * nbc + ib];
                            }
                            dS[x][ia * nbc + ib] += vs;
                            dT[x][ia * nbc + ib] += vt;
                        }
                    }
                }
            }
        }
        for (int x = 0; x < 3; x++) {
            double s = 0.0;
            for (int k = 0; k < nac * nbc; k++) s += 2.0 * (Dc[k] * dT[x][k] - Wc[k] * dS[x][k]);
            ga[x] += s;
        }
    }
    // nuclear attraction, nucleus by nucleus: basis-function term on the bra
    // atom and, by translational invariance of the three-centre integral
    // (dA + dB + dC = 0, the ket term equal to the bra term by symmetry), the
    // operator term -2 sum D dV^C/dA on nucleus C itself.
    for (int c = c0; c < c1; c++) {
        double dV[3][36];
        for (int x = 0; x < 3; x++)
            for (int k = 0; k < nac * nbc; k++) dV[x][k] = 0.0;
        for (int i = 0; i < B.snprim[sa]; i++) {
            const double a = B.exps[pa + i];
            double A[3], Bc[3], AB2 = 0.0;
            for (int x = 0; x < 3; x++) {
                A[x] = S.xyz[3 * sa + x];
                Bc[x] = S.xyz[3 * sb + x];
                AB2 += (A[x] - Bc[x]) * (A[x] - Bc[x]);
            }
            const int pb = B.sprim[sb];
            for (int k = 0; k < ncu * nbc; k++) Vu[k] = 0.0;
            for (int k = 0; k < ncd * nbc; k++) Vd[k] = 0.0;
            for (int j = 0; j < B.snprim[sb]; j++) {
                const double b = B.exps[pb + j];
                const double p = a + b;
                const double K = B.coefs[pa + i] * B.coefs[pb + j] * exp(-a * b / p * AB2);
                double PA[3], PB[3], PC[3], PC2 = 0.0;
                for (int x = 0; x < 3; x++) {
                    const double Px = (a * A[x] + b * Bc[x]) / p;
                    PA[x] = Px - A[x];
                    PB[x] = Px - Bc[x];
                    PC[x] = Px - At.xyz[3 * c + x];
                    PC2 += PC[x] * PC[x];
                }
                double F[NM1];
                boys_eval_n(la + 1 + lb, p * PC2, boys, 1.0, F);
                double Vt[NM1 * NA1 * NB1];
                os_nuclear(la + 1, lb, p, PA, PB, PC, F, -At.Z[c] * 2.0 * kPi / p * K, Vt);
                for (int lev = 0; lev < 2; lev++) {
                    const int lq = lev == 0 ? la + 1 : la - 1;
                    if (lq < 0) continue;
                    for (int ia = 0; ia < ncart(lq); ia++) {
                        int e[3];
                        cart_of_d(lq, ia, e);
                        const int gq = gidx(e[0], e[1], e[2]);
                        for (int ib = 0; ib < nbc; ib++) {
                            int f[3];
                            cart_of_d(lb, ib, f);
                            const double v = Vt[(0 * NA1 + gq) * NB1 + gidx(f[0], f[1], f[2])];
                            if (lev == 0)
                                Vu[ia * nbc + ib] += v;
                            else
                                Vd[ia * nbc + ib] += v;
                        }
                    }
                }
            }
            for (int ia = 0; ia < nac; ia++) {
                int e[3];
                cart_of_d(la, ia, e);
                for (int x = 0; x < 3; x++) {
                    int eu[3] = {e[0], e[1], e[2]};
                    eu[x]++;
                    const int iu = cidx_host_dev(eu);
                    for (int ib = 0; ib < nbc; ib++) {
                        double v = 2.0 * a * Vu[iu * nbc + ib];
                        if (e[x] > 0) {
                            int ed[3] = {e[0], e[1], e[2]};
                            ed[x]--;
                            v -= e[x] * Vd[cidx_host_dev(ed) * nbc + ib];
                        }
                        dV[x][ia * nbc + ib] += v;
                    }
                }
            }
        }
        for (int x = 0; x < 3; x++) {
            double s = 0.0;
            for (int k = 0; k < nac * nbc; k++) s += 2.0 * Dc[k] * dV[x][k];
            ga[x] += s;
            det_add(grad + 3 * c + x, -s, fxs);
        }
    }
    for (int x = 0; x < 3; x++) det_add(grad + 3 * atom_a + x, ga[x], fxs);
}

__global__ void vnn_kernel(AtomsDev At, int natom, const int* atom_rep, double* enn, double* grad, double fxs)
{
    const int A = blockIdx.x * blockDim.x + threadIdx.x;
    if (A >= natom) return;
    const int r = atom_rep[A];
    const int c0 = At.rep_atom0[r], c1 = At.rep_atom0[r + 1];
    double e = 0.0, g[3] = {0.0, 0.0, 0.0};
    for (int Bi = c0; Bi < c1; Bi++) {
        if (Bi == A) continue;
        double d[3], r2 = 0.0;
        for (int x = 0; x < 3; x++) {
            d[x] = At.xyz[3 * A + x] - At.xyz[3 * Bi + x];
            r2 += d[x] * d[x];
        }
        const double rr = sqrt(r2);
        const double zz = At.Z[A] * At.Z[Bi];
        e += 0.5 * zz / rr;
        for (int x = 0; x < 3; x++) g[x] -= zz * d[x] / (rr * r2);
    }
    det_add(enn + r, e, fxs);
    if (grad)
        for (int x = 0; x < 3; x++) det_add(grad + 3 * A + x, g[x], fxs);
}

__global__ void boys_eval_kernel(int n, int m, const double* T, double* F, const double* boys)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double t = T[i];
    // the table covers T >= 0 only: a negative or non-finite argument gives NaN
    if (!(t >= 0.0) || !isfinite(t)) {
        F[i] = nan("");
        return;
    }
    double f[BOYS_MMAX + 1];
    boys_eval_n(m, t, boys, 1.0, f);
    F[i] = f[m];
}

// FP32 evaluation of the mixed-precision quartets: variant 0 the
// compile-time-order form of the straight-line kernels, 1 the runtime-order
// form of the cooperative kernels
template <int L>
__device__ __forceinline__ float boys_f32_fixed(float t, const float* boysf)
{
    float f[L + 1];
    boys_eval<L>(t, boysf, 1.0f, f);
    return f[L];
}

__global__ void boys_eval_f32_kernel(int n, int m, const float* T, float* F, const float* boysf, int variant)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float t = T[i];
    if (!(t >= 0.0f) || !isfinite(t)) {
        F[i] = nanf("");
        return;
    }
    if (variant == 1) {
        float f[BOYS_MMAX + 1];
        boys_eval_n(m, t, boysf, 1.0f, f);
        F[i] = f[m];
        return;
    }
    float v = 0.0f;
    switch (m) {
    case 0: v = boys_f32_fixed<0>(t, boysf); break;
    case 1: v = boys_f32_fixed<1>(t, boysf); break;
    case 2: v = boys_f32_fixed<2>(t, boysf); break;
    case 3: v = boys_f32_fixed<3>(t, boysf); break;
    case 4: v = boys_f32_fixed<4>(t, boysf); break;
    case 5: v = boys_f32_fixed<5>(t, boysf); break;
    case 6: v = boys_f32_fixed<6>(t, boysf); break;
    case 7: v = boys_f32_fixed<7>(t, boysf); break;
    case 8: v = boys_f32_fixed<8>(t, boysf); break;
    case 9: v = boys_f32_fixed<9>(t, boysf); break;
    case 10: v = boys_f32_fixed<10>(t, boysf); break;
    case 11: v = boys_f32_fixed<11>(t, boysf); break;
    default: v = boys_f32_fixed<12>(t, boysf); break;
    }
    F[i] = v;
}

}  // namespace

void launch_boys_eval_f32(int n, int m, const float* T, float* F, const float* boysf, int variant, cudaStream_t st)
{
    if (n == 0) return;
    boys_eval_f32_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, m, T, F, boysf, variant);
}

void launch_pair_data(const Pairs& P, int* npp, double* pp, const Shells& S, const BasisPrimDev& B,
                      cudaStream_t st)
{
    if (P.n == 0) return;
    pair_data_kernel<<<(P.n + 127) / 128, 128, 0, st>>>(P, npp, pp, S, B);
}

void launch_one_electron(const Pairs& P, const Shells& S, const BasisPrimDev& B, const AtomsDev& At,
                         const Reps& R, double* Sm, double* Tm, double* Vm, const double* boys, cudaStream_t st)
{
    if (P.n == 0) return;
    one_e_kernel<<<(P.n + 63) / 64, 64, 0, st>>>(P, S, B, At, R, Sm, Tm, Vm, boys);
}

void launch_grad_1e(const Pairs& P, const Shells& S, const BasisPrimDev& B, const AtomsDev& At, const Reps& R,
                    const double* D, const double* W, double* grad, const double* boys, double fxs,
                    cudaStream_t st)
{
    if (P.n == 0) return;
    grad_1e_kernel<<<(2 * P.n + 63) / 64, 64, 0, st>>>(P, S, B, At, R, D, W, grad, boys, fxs);
}

void launch_vnn(const AtomsDev& At, int natom_total, const int* atom_rep, double* enn, double* grad,
                cudaStream_t st, double fxs)
{
    if (natom_total == 0) return;
    vnn_kernel<<<(natom_total + 127) / 128, 128, 0, st>>>(At, natom_total, atom_rep, enn, grad, fxs);
}

void launch_boys_eval(int n, int m, const double* T, double* F, const double* boys, cudaStream_t st)
{
    if (n == 0) return;
    boys_eval_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, m, T, F, boys);
}

// F_m(T) = e^{-T} sum_i (2T)^i / ((2m+1)(2m+3)...(2m+2i+1)), a sum of positive
// terms evaluated in long double; stored as F_{m+j}(T_k) / j! and e^{-T_k}.
void boys_fill_table(double* tab)
{
    const int NM = BOYS_MT + BOYS_NTAYLOR;
    long double F[BOYS_MT + BOYS_NTAYLOR];
    for (int k = 0; k < BOYS_NT; k++) {
        const long double T = (long double)k / BOYS_GRID;
        for (int m = 0; m < NM; m++) {
            long double term = 1.0L / (2 * m + 1), sum = term;
            for (int i = 1; i < 2000; i++) {
                term *= 2.0L * T / (2 * m + 2 * i + 1);
                sum += term;
                if (term < 1e-22L * sum) break;
            }
            F[m] = expl(-T) * sum;
        }
        long double fact = 1.0L;
        for (int j = 0; j < BOYS_NTAYLOR; j++) {
            if (j > 0) fact *= j;
            for (int m = 0; m < BOYS_MT; m++)
                tab[((size_t)k * BOYS_MT + m) * BOYS_NTAYLOR + j] = (double)(F[m + j] / fact);
        }
    }
    for (int k = 0; k < BOYS_NE; k++) tab[BOYS_EXP_OFF + k] = (double)expl(-(long double)k / BOYS_GRID);
}

void boys_table_upload(double** dev_tab, float** dev_tabf)
{
    static double host[BOYS_TAB_DOUBLES];
    static float hostf[BOYS_TAB_FLOATS];
    static bool filled = false;
    if (!filled) {
        boys_fill_table(host);
        for (int k = 0; k < BOYS_NT; k++) {
            for (int m = 0; m < BOYS_MT; m++)
                for (int j = 0; j < BOYS_NTAYLOR_F; j++)
                    hostf[((size_t)k * BOYS_MT + m) * BOYS_NTAYLOR_F + j] =
                        (float)host[((size_t)k * BOYS_MT + m) * BOYS_NTAYLOR + j];
            hostf[(size_t)BOYS_NT * BOYS_MT * BOYS_NTAYLOR_F + k] = (float)host[(size_t)BOYS_NT * BOYS_MT * BOYS_NTAYLOR + k];
        }
        filled = true;
    }
    cudaMalloc(dev_tab, sizeof(host));
    cudaMemcpy(*dev_tab, host, sizeof(host), cudaMemcpyHostToDevice);
    cudaMalloc(dev_tabf, sizeof(hostf));
    cudaMemcpy(*dev_tabf, hostf, sizeof(hostf), cudaMemcpyHostToDevice);
}

__global__ void to_float_kernel(const double* src, float* dst, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

void launch_to_float(const double* src, float* dst, long long n, cudaStream_t st)
{
    if (n <= 0) return;
    to_float_kernel<<<256, 256, 0, st>>>(src, dst, n);
}

}  // namespace pimd
