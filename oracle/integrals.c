/*
 * Oracle: plain FP64 Gaussian-integral code for the RHF energy and gradient.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call
 * this file; only the tests, the package's smoke check and the CPU-baseline leg
 * of the benchmark use it. It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * The paper states the workload (RHF-type Born-Oppenheimer energies and forces
 * of every replica, Sec. 2; integral cutoff 1e-12, Sec. 3.1) but no integral
 * algorithm. This file writes the textbook McMurchie-Davidson scheme out
 * literally: Hermite expansion coefficients E^{ij}_t, Hermite Coulomb
 * integrals R^{(n)}_{tuv} from the Boys function F_n(T), and
 *   (ab|cd) = 2 pi^{5/2} / (p q sqrt(p+q))
 *             sum_{tuv} E^{ab}_{tuv} sum_{tau nu phi} (-1)^{tau+nu+phi}
 *             E^{cd}_{tau nu phi} R_{t+tau, u+nu, v+phi}(alpha, P-Q).
 * Integral derivatives come from differentiating the Gaussians,
 *   d/dA_x [x_A^i e^{-a x_A^2}] = 2a x_A^{i+1} e^{..} - i x_A^{i-1} e^{..},
 * applied to every centre explicitly (translational invariance is not used, so
 * it stays a test). The Hellmann-Feynman term uses dR_{tuv}/dC_x = -R_{t+1,u,v}.
 *
 * Basis conventions (shared definition, implemented independently elsewhere):
 * cartesian components of a shell of angular momentum l are ordered
 * lx = l..0, ly = l-lx..0, lz = l-lx-ly (p: x,y,z; d: xx,xy,xz,yy,yz,zz).
 * Contraction coefficients passed in already carry the normalisation of the
 * axis-aligned component x^l. Spherical d functions (m = -2..2) are
 *   sqrt3 xy, sqrt3 yz, zz - (xx+yy)/2, sqrt3 xz, sqrt3/2 (xx-yy).
 * With spherical == 0 every cartesian component is normalised on its own.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define LMAX_SHELL 3          /* d shells raised by one for derivatives */
#define LMAX_E (LMAX_SHELL + 2)  /* kinetic integrals need j + 2 */
#define LMAX_R 10             /* d quartet raised by one: 2+2+2+3 = 9 */
#define NCART(l) (((l) + 1) * ((l) + 2) / 2)

/* ------------------------------------------------------------------------- */
/* Boys function F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt                        */
/* T < 30: the series F_m(T) = e^{-T} sum_i (2T)^i / ((2m+1)(2m+3)...(2m+2i+1))  */
/* T >= 30: F_0 = (1/2) sqrt(pi/T) erf(sqrt T) and the upward recursion          */
/*          F_{m+1} = ((2m+1) F_m - e^{-T}) / (2T), stable for T >> m.          */
/* ------------------------------------------------------------------------- */
double oracle_boys(int m, double T)
{
    if (T < 30.0) {
        double term = 1.0 / (2 * m + 1);
        double sum = term;
        for (int i = 1; i < 1000; i++) {
            term *= 2.0 * T / (2 * m + 2 * i + 1);
            sum += term;
            if (term < 1e-18 * sum) break;
        }
        return exp(-T) * sum;
    }
    double et = exp(-T);
    double f = 0.5 * sqrt(M_PI / T) * erf(sqrt(T));
    for (int k = 0; k < m; k++) f = ((2 * k + 1) * f - et) / (2.0 * T);
    return f;
}

/* all F_0..F_n at one T: top value from oracle_boys, then the downward
 * recursion F_m = (2T F_{m+1} + e^{-T}) / (2m+1) (stable for all T). */
static void boys_all(int n, double T, double *F)
{
    F[n] = oracle_boys(n, T);
    double et = exp(-T);
    for (int m = n - 1; m >= 0; m--) F[m] = (2.0 * T * F[m + 1] + et) / (2 * m + 1);
}

/* cartesian component list of a shell */
static int cart_list(int l, int (*c)[3])
{
    int n = 0;
    for (int lx = l; lx >= 0; lx--)
        for (int ly = l - lx; ly >= 0; ly--) {
            c[n][0] = lx; c[n][1] = ly; c[n][2] = l - lx - ly; n++;
        }
    return n;
}

static double dfact(int n) /* (n)!! with (-1)!! = 1 */
{
    double r = 1.0;
    for (int k = n; k > 1; k -= 2) r *= k;
    return r;
}

/* ------------------------------------------------------------------------- */
/* Hermite expansion coefficients E^{ij}_t for one Cartesian direction        */
/* E[i][j][t], i <= imax, j <= jmax, t <= i + j                                */
/* ------------------------------------------------------------------------- */
typedef double Etab[LMAX_E + 1][LMAX_E + 1][2 * LMAX_E + 2];

static void hermite_E(int imax, int jmax, double a, double b, double XAB, Etab E)
{
    double p = a + b, mu = a * b / p;
    double XPA = -b / p * XAB, XPB = a / p * XAB;
    E[0][0][0] = exp(-mu * XAB * XAB);
    for (int i = 0; i <= imax; i++) {
        for (int j = 0; j <= jmax; j++) {
            if (i == 0 && j == 0) continue;
            for (int t = 0; t <= i + j; t++) {
                double v;
                if (i > 0) {
                    v = t <= i - 1 + j ? XPA * E[i - 1][j][t] : 0.0;
                    if (t > 0) v += E[i - 1][j][t - 1] / (2 * p);
                    if (t + 1 <= i - 1 + j) v += (t + 1) * E[i - 1][j][t + 1];
                } else {
                    v = t <= i + j - 1 ? XPB * E[i][j - 1][t] : 0.0;
                    if (t > 0) v += E[i][j - 1][t - 1] / (2 * p);
                    if (t + 1 <= i + j - 1) v += (t + 1) * E[i][j - 1][t + 1];
                }
                E[i][j][t] = v;
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Hermite Coulomb integrals R_{tuv} = R^{(0)}_{tuv}(alpha, X, Y, Z), t+u+v<=L  */
/* ------------------------------------------------------------------------- */
typedef double Rtab[LMAX_R + 1][LMAX_R + 1][LMAX_R + 1];

static void hermite_R(int L, double alpha, double X, double Y, double Z, Rtab R0)
{
    static __thread double Rn[LMAX_R + 1][LMAX_R + 1][LMAX_R + 1][LMAX_R + 1];
    double F[LMAX_R + 1];
    double T = alpha * (X * X + Y * Y + Z * Z);
    boys_all(L, T, F);
    double fac = 1.0;
    for (int n = 0; n <= L; n++) {
        Rn[n][0][0][0] = fac * F[n];
        fac *= -2.0 * alpha;
    }
    for (int k = 1; k <= L; k++)
        for (int t = 0; t <= k; t++)
            for (int u = 0; u <= k - t; u++) {
                int v = k - t - u;
                for (int n = 0; n <= L - k; n++) {
                    double r;
                    if (t > 0) {
                        r = X * Rn[n + 1][t - 1][u][v];
                        if (t > 1) r += (t - 1) * Rn[n + 1][t - 2][u][v];
                    } else if (u > 0) {
                        r = Y * Rn[n + 1][t][u - 1][v];
                        if (u > 1) r += (u - 1) * Rn[n + 1][t][u - 2][v];
                    } else {
                        r = Z * Rn[n + 1][t][u][v - 1];
                        if (v > 1) r += (v - 1) * Rn[n + 1][t][u][v - 2];
                    }
                    Rn[n][t][u][v] = r;
                }
            }
    for (int t = 0; t <= L; t++)
        for (int u = 0; u <= L - t; u++)
            for (int v = 0; v <= L - t - u; v++) R0[t][u][v] = Rn[0][t][u][v];
}

/* ------------------------------------------------------------------------- */
/* Hermite data of one primitive pair: exponent sum, centre, E tables         */
/* ------------------------------------------------------------------------- */
typedef struct {
    double p, P[3], w;
    Etab E[3];
} primpair_t;

static void make_primpair(int la, int lb, double a, double b, const double *A, const double *B,
                          double w, primpair_t *pp)
{
    pp->p = a + b;
    pp->w = w;
    for (int x = 0; x < 3; x++) {
        pp->P[x] = (a * A[x] + b * B[x]) / pp->p;
        hermite_E(la, lb, a, b, A[x] - B[x], pp->E[x]);
    }
}

/* ------------------------------------------------------------------------- */
/* primitive cartesian ERIs for shells of angular momentum la,lb,lc,ld,       */
/* accumulated with weight w into out[((ia*nb + ib)*nc + ic)*nd + id]:        */
/*   X_{tuv}(cd) = sum_{tau nu phi} (-1)^{tau+nu+phi} E^{cd}_{tau nu phi}     */
/*                 R_{t+tau,u+nu,v+phi}                                      */
/*   (ab|cd)     = pre * sum_{tuv} E^{ab}_{tuv} X_{tuv}(cd)                   */
/* ------------------------------------------------------------------------- */
static void eri_prim_acc(int la, int lb, int lc, int ld, const primpair_t *ab, const primpair_t *cd,
                         double w, double *out)
{
    static __thread Rtab R;
    static __thread double X[2 * LMAX_SHELL + 1][2 * LMAX_SHELL + 1][2 * LMAX_SHELL + 1];
    int ca[NCART(LMAX_SHELL)][3], cb[NCART(LMAX_SHELL)][3], cc[NCART(LMAX_SHELL)][3], cdd[NCART(LMAX_SHELL)][3];
    int na = cart_list(la, ca), nb = cart_list(lb, cb), nc = cart_list(lc, cc), nd = cart_list(ld, cdd);
    double p = ab->p, q = cd->p, alpha = p * q / (p + q);
    int L = la + lb + lc + ld, Lab = la + lb;
    hermite_R(L, alpha, ab->P[0] - cd->P[0], ab->P[1] - cd->P[1], ab->P[2] - cd->P[2], R);
    double pre = w * 2.0 * pow(M_PI, 2.5) / (p * q * sqrt(p + q));
    for (int ic = 0; ic < nc; ic++)
    for (int id = 0; id < nd; id++) {
        const int *xc = cc[ic], *xd = cdd[id];
        for (int t = 0; t <= Lab; t++)
        for (int u = 0; u <= Lab - t; u++)
        for (int v = 0; v <= Lab - t - u; v++) {
            double s2 = 0.0;
            for (int tau = 0; tau <= xc[0] + xd[0]; tau++)
            for (int nu = 0; nu <= xc[1] + xd[1]; nu++)
            for (int phi = 0; phi <= xc[2] + xd[2]; phi++) {
                double sgn = ((tau + nu + phi) & 1) ? -1.0 : 1.0;
                s2 += sgn * cd->E[0][xc[0]][xd[0]][tau] * cd->E[1][xc[1]][xd[1]][nu] * cd->E[2][xc[2]][xd[2]][phi]
                      * R[t + tau][u + nu][v + phi];
            }
            X[t][u][v] = s2;
        }
        for (int ia = 0; ia < na; ia++)
        for (int ib = 0; ib < nb; ib++) {
            const int *xa = ca[ia], *xb = cb[ib];
            double sum = 0.0;
            for (int t = 0; t <= xa[0] + xb[0]; t++)
            for (int u = 0; u <= xa[1] + xb[1]; u++)
            for (int v = 0; v <= xa[2] + xb[2]; v++)
                sum += ab->E[0][xa[0]][xb[0]][t] * ab->E[1][xa[1]][xb[1]][u] * ab->E[2][xa[2]][xb[2]][v] * X[t][u][v];
            out[((ia * nb + ib) * nc + ic) * nd + id] += pre * sum;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* basis description passed from Python                                      */
/* ------------------------------------------------------------------------- */
typedef struct {
    int nshell;
    const int *l, *nprim, *poff;   /* per shell: l, number of primitives, offset */
    const double *exps, *coefs;    /* per primitive (coefs normalised for x^l) */
    const double *cen;             /* [nshell][3] */
    const int *atom;               /* [nshell] */
    int spherical;
} basis_t;

static int shell_nbf(const basis_t *bs, int s)
{
    int l = bs->l[s];
    return bs->spherical && l >= 2 ? 2 * l + 1 : NCART(l);
}

static void shell_offsets(const basis_t *bs, int *off)
{
    int o = 0;
    for (int s = 0; s < bs->nshell; s++) { off[s] = o; o += shell_nbf(bs, s); }
    off[bs->nshell] = o;
}

/* rows: basis functions of the shell, cols: cartesian components */
static int cart_to_basis(const basis_t *bs, int l, double *T)
{
    int nc = NCART(l);
    if (bs->spherical && l == 2) {
        const double s3 = sqrt(3.0);
        double M[5][6] = {
            {0, s3, 0, 0, 0, 0},               /* sqrt3 xy */
            {0, 0, 0, 0, s3, 0},               /* sqrt3 yz */
            {-0.5, 0, 0, -0.5, 0, 1.0},        /* zz - (xx+yy)/2 */
            {0, 0, s3, 0, 0, 0},               /* sqrt3 xz */
            {0.5 * s3, 0, 0, -0.5 * s3, 0, 0}, /* sqrt3/2 (xx - yy) */
        };
        memcpy(T, M, sizeof(M));
        return 5;
    }
    if (bs->spherical && l > 2) return -1;
    int c[NCART(LMAX_SHELL)][3];
    cart_list(l, c);
    memset(T, 0, sizeof(double) * nc * nc);
    for (int i = 0; i < nc; i++) {
        /* per-component normalisation relative to x^l */
        T[i * nc + i] = sqrt(dfact(2 * l - 1) / (dfact(2 * c[i][0] - 1) * dfact(2 * c[i][1] - 1) * dfact(2 * c[i][2] - 1)));
    }
    return nc;
}

/* transform one index of a 4-index block: in[n0][nc][n2] -> out[n0][nf][n2] */
static void transform_index(const double *in, double *out, int n0, int nc, int n2, const double *T, int nf)
{
    for (int i = 0; i < n0; i++)
        for (int f = 0; f < nf; f++)
            for (int k = 0; k < n2; k++) {
                double s = 0.0;
                for (int c = 0; c < nc; c++) s += T[f * nc + c] * in[(i * nc + c) * n2 + k];
                out[(i * nf + f) * n2 + k] = s;
            }
}

/* cartesian block [na_c][nb_c][nc_c][nd_c] -> basis block [na][nb][nc][nd] */
static void block_to_basis(const basis_t *bs, int la, int lb, int lc, int ld, double *blk, double *tmp)
{
    int ls[4] = {la, lb, lc, ld};
    int n[4] = {NCART(la), NCART(lb), NCART(lc), NCART(ld)};
    double T[36 * 2];
    for (int k = 0; k < 4; k++) {
        int nf = cart_to_basis(bs, ls[k], T);
        int n0 = 1, n2 = 1;
        for (int j = 0; j < k; j++) n0 *= n[j];
        for (int j = k + 1; j < 4; j++) n2 *= n[j];
        transform_index(blk, tmp, n0, n[k], n2, T, nf);
        n[k] = nf;
        memcpy(blk, tmp, sizeof(double) * n0 * nf * n2);
    }
}

#define MAXC 10 /* NCART(3) */
#define BLK (MAXC * MAXC * MAXC * MAXC)

/* contracted cartesian block of (ab|cd) with raised/lowered angular momentum
 * dl[k] on centre k and primitive weights: each primitive quartet is scaled by
 * prod_k (wexp[k] ? 2*alpha_k : 1). */
static void eri_contracted_cart(const basis_t *bs, const int sh[4], const int dl[4], const int wexp[4], double *out)
{
    static __thread primpair_t bra[64], ket[64];
    int l[4];
    int n = 1;
    for (int k = 0; k < 4; k++) { l[k] = bs->l[sh[k]] + dl[k]; n *= NCART(l[k]); }
    memset(out, 0, sizeof(double) * n);
    int nbra = 0, nket = 0;
    for (int side = 0; side < 2; side++) {
        int s0 = sh[2 * side], s1 = sh[2 * side + 1];
        for (int i = 0; i < bs->nprim[s0]; i++)
            for (int j = 0; j < bs->nprim[s1]; j++) {
                int pi = bs->poff[s0] + i, pj = bs->poff[s1] + j;
                double a = bs->exps[pi], b = bs->exps[pj];
                double w = bs->coefs[pi] * bs->coefs[pj];
                if (wexp[2 * side]) w *= 2 * a;
                if (wexp[2 * side + 1]) w *= 2 * b;
                primpair_t *pp = side == 0 ? &bra[nbra++] : &ket[nket++];
                make_primpair(l[2 * side], l[2 * side + 1], a, b, bs->cen + 3 * s0, bs->cen + 3 * s1, w, pp);
            }
    }
    for (int i = 0; i < nbra; i++)
        for (int j = 0; j < nket; j++)
            eri_prim_acc(l[0], l[1], l[2], l[3], &bra[i], &ket[j], bra[i].w * ket[j].w, out);
}

/* contracted basis-function block (ab|cd), layout [na][nb][nc][nd] */
static void eri_block(const basis_t *bs, int a, int b, int c, int d, double *out)
{
    int sh[4] = {a, b, c, d}, dl[4] = {0, 0, 0, 0}, w[4] = {0, 0, 0, 0};
    double tmp[BLK];
    eri_contracted_cart(bs, sh, dl, w, out);
    block_to_basis(bs, bs->l[a], bs->l[b], bs->l[c], bs->l[d], out, tmp);
}

#define BASIS_ARGS int nshell, const int *l, const int *nprim, const int *poff, const double *exps, \
    const double *coefs, const double *cen, const int *atom, int spherical
#define MAKE_BASIS basis_t bs = {nshell, l, nprim, poff, exps, coefs, cen, atom, spherical}

void oracle_eri_block(BASIS_ARGS, int a, int b, int c, int d, double *out)
{
    MAKE_BASIS;
    double blk[BLK];
    eri_block(&bs, a, b, c, d, blk);
    int n = shell_nbf(&bs, a) * shell_nbf(&bs, b) * shell_nbf(&bs, c) * shell_nbf(&bs, d);
    memcpy(out, blk, sizeof(double) * n);
}

/* Schwarz factors Q_ab = sqrt(max |(ab|ab)|) over the functions of the pair */
void oracle_schwarz(BASIS_ARGS, double *Q)
{
    MAKE_BASIS;
    int ns = bs.nshell;
#pragma omp parallel for schedule(dynamic)
    for (int a = 0; a < ns; a++)
        for (int b = 0; b <= a; b++) {
            double blk[BLK];
            eri_block(&bs, a, b, a, b, blk);
            int na = shell_nbf(&bs, a), nb = shell_nbf(&bs, b);
            double m = 0.0;
            for (int i = 0; i < na; i++)
                for (int j = 0; j < nb; j++) {
                    double v = fabs(blk[((i * nb + j) * na + i) * nb + j]);
                    if (v > m) m = v;
                }
            Q[a * ns + b] = Q[b * ns + a] = sqrt(m);
        }
}

/* full ERI tensor (tiny systems only), layout [N][N][N][N] */
void oracle_eri_full(BASIS_ARGS, double *out)
{
    MAKE_BASIS;
    int ns = bs.nshell;
    int *off = malloc(sizeof(int) * (ns + 1));
    shell_offsets(&bs, off);
    int N = off[ns];
    double blk[BLK];
    for (int a = 0; a < ns; a++)
    for (int b = 0; b < ns; b++)
    for (int c = 0; c < ns; c++)
    for (int d = 0; d < ns; d++) {
        eri_block(&bs, a, b, c, d, blk);
        int na = shell_nbf(&bs, a), nb = shell_nbf(&bs, b), nc = shell_nbf(&bs, c), nd = shell_nbf(&bs, d);
        for (int i = 0; i < na; i++) for (int j = 0; j < nb; j++)
        for (int k = 0; k < nc; k++) for (int m = 0; m < nd; m++)
            out[(((size_t)(off[a] + i) * N + off[b] + j) * N + off[c] + k) * N + off[d] + m] =
                blk[((i * nb + j) * nc + k) * nd + m];
    }
    free(off);
}

/* ------------------------------------------------------------------------- */
/* Coulomb and exchange matrices                                              */
/*   J_mn = sum_ls D_ls (mn|ls),  K_mn = sum_ls D_ls (ml|ns)                  */
/* over canonical shell quartets a>=b, c>=d, (ab)>=(cd), Schwarz-screened at  */
/* Q_ab Q_cd >= tau (density independent), each scattered to its 8            */
/* permutations with weight 1/|stabiliser| so that the full sum is recovered. */
/* ------------------------------------------------------------------------- */
long long oracle_jk(BASIS_ARGS, const double *D, double tau, double *J, double *K)
{
    MAKE_BASIS;
    int ns = bs.nshell;
    int *off = malloc(sizeof(int) * (ns + 1));
    shell_offsets(&bs, off);
    int N = off[ns];
    double *Q = malloc(sizeof(double) * ns * ns);
    oracle_schwarz(nshell, l, nprim, poff, exps, coefs, cen, atom, spherical, Q);
    memset(J, 0, sizeof(double) * N * N);
    memset(K, 0, sizeof(double) * N * N);
    long long nq = 0;
    int npair = ns * (ns + 1) / 2;
#pragma omp parallel reduction(+ : nq)
    {
        double *Jt = calloc((size_t)N * N, sizeof(double));
        double *Kt = calloc((size_t)N * N, sizeof(double));
        double blk[BLK];
#pragma omp for schedule(dynamic)
        for (int pab = 0; pab < npair; pab++) {
            int a = (int)((sqrt(8.0 * pab + 1) - 1) / 2);
            while (a * (a + 1) / 2 > pab) a--;
            while ((a + 1) * (a + 2) / 2 <= pab) a++;
            int b = pab - a * (a + 1) / 2;
            for (int pcd = 0; pcd <= pab; pcd++) {
                int c = (int)((sqrt(8.0 * pcd + 1) - 1) / 2);
                while (c * (c + 1) / 2 > pcd) c--;
                while ((c + 1) * (c + 2) / 2 <= pcd) c++;
                int d = pcd - c * (c + 1) / 2;
                if (Q[a * ns + b] * Q[c * ns + d] < tau) continue;
                nq++;
                eri_block(&bs, a, b, c, d, blk);
                double f = 1.0;
                if (a == b) f *= 0.5;
                if (c == d) f *= 0.5;
                if (pab == pcd) f *= 0.5;
                int na = shell_nbf(&bs, a), nb = shell_nbf(&bs, b), nc = shell_nbf(&bs, c), nd = shell_nbf(&bs, d);
                for (int i = 0; i < na; i++) for (int j = 0; j < nb; j++)
                for (int k = 0; k < nc; k++) for (int m = 0; m < nd; m++) {
                    double v = f * blk[((i * nb + j) * nc + k) * nd + m];
                    int p = off[a] + i, qq = off[b] + j, r = off[c] + k, s = off[d] + m;
                    /* the 8 index permutations (pq|rs), (qp|rs), (pq|sr), (qp|sr),
                     * (rs|pq), (sr|pq), (rs|qp), (sr|qp); for each (ij|kl):
                     * J_ij += D_kl v, K_ik += D_jl v */
                    int perm[8][4] = {{p, qq, r, s}, {qq, p, r, s}, {p, qq, s, r}, {qq, p, s, r},
                                      {r, s, p, qq}, {s, r, p, qq}, {r, s, qq, p}, {s, r, qq, p}};
                    for (int g = 0; g < 8; g++) {
                        int i1 = perm[g][0], j1 = perm[g][1], k1 = perm[g][2], l1 = perm[g][3];
                        Jt[i1 * N + j1] += D[k1 * N + l1] * v;
                        Kt[i1 * N + k1] += D[j1 * N + l1] * v;
                    }
                }
            }
        }
#pragma omp critical
        {
            for (size_t x = 0; x < (size_t)N * N; x++) { J[x] += Jt[x]; K[x] += Kt[x]; }
        }
        free(Jt);
        free(Kt);
    }
    free(Q);
    free(off);
    return nq;
}

/* ------------------------------------------------------------------------- */
/* two-electron gradient                                                      */
/*   g_A += sum_{mnls} [ 1/2 D_mn D_ls - kx/4 D_ml D_ns ] d(mn|ls)/dA          */
/* over canonical quartets with weight f = 1/|stabiliser|; summing the bracket */
/* over the 8 permutations gives 4 D_mn D_ls - kx (D_ml D_ns + D_ms D_nl).     */
/* kx = 1 for Hartree-Fock; a hybrid functional's fraction of exact exchange  */
/* otherwise (0.20 for B3LYP). Each of the four centres is differentiated     */
/* explicitly.                                                                */
/* ------------------------------------------------------------------------- */
void oracle_grad_2e_kx(BASIS_ARGS, int natom, const double *D, double tau, double kx, double *grad)
{
    MAKE_BASIS;
    int ns = bs.nshell;
    int *off = malloc(sizeof(int) * (ns + 1));
    shell_offsets(&bs, off);
    int N = off[ns];
    double *Q = malloc(sizeof(double) * ns * ns);
    oracle_schwarz(nshell, l, nprim, poff, exps, coefs, cen, atom, spherical, Q);
    memset(grad, 0, sizeof(double) * natom * 3);
    int npair = ns * (ns + 1) / 2;
#pragma omp parallel
    {
        double *gt = calloc((size_t)natom * 3, sizeof(double));
        double *up = malloc(sizeof(double) * BLK), *dn = malloc(sizeof(double) * BLK);
        double *der = malloc(sizeof(double) * BLK), *tmp = malloc(sizeof(double) * BLK);
#pragma omp for schedule(dynamic)
        for (int pab = 0; pab < npair; pab++) {
            int a = (int)((sqrt(8.0 * pab + 1) - 1) / 2);
            while (a * (a + 1) / 2 > pab) a--;
            while ((a + 1) * (a + 2) / 2 <= pab) a++;
            int b = pab - a * (a + 1) / 2;
            for (int pcd = 0; pcd <= pab; pcd++) {
                int c = (int)((sqrt(8.0 * pcd + 1) - 1) / 2);
                while (c * (c + 1) / 2 > pcd) c--;
                while ((c + 1) * (c + 2) / 2 <= pcd) c++;
                int d = pcd - c * (c + 1) / 2;
                if (Q[a * ns + b] * Q[c * ns + d] < tau) continue;
                double f = 1.0;
                if (a == b) f *= 0.5;
                if (c == d) f *= 0.5;
                if (pab == pcd) f *= 0.5;
                int sh[4] = {a, b, c, d};
                int ls[4] = {bs.l[a], bs.l[b], bs.l[c], bs.l[d]};
                int nb_[4] = {shell_nbf(&bs, a), shell_nbf(&bs, b), shell_nbf(&bs, c), shell_nbf(&bs, d)};
                for (int k = 0; k < 4; k++) {          /* centre being moved */
                    int dl[4] = {0, 0, 0, 0}, w[4] = {0, 0, 0, 0};
                    dl[k] = 1; w[k] = 1;
                    eri_contracted_cart(&bs, sh, dl, w, up);   /* 2 alpha (l+1) */
                    int haslow = ls[k] > 0;
                    if (haslow) {
                        dl[k] = -1; w[k] = 0;
                        eri_contracted_cart(&bs, sh, dl, w, dn);   /* (l-1) */
                    }
                    int nc0[4] = {NCART(ls[0]), NCART(ls[1]), NCART(ls[2]), NCART(ls[3])};
                    int ncu[4], ncd[4];
                    for (int j = 0; j < 4; j++) { ncu[j] = nc0[j]; ncd[j] = nc0[j]; }
                    ncu[k] = NCART(ls[k] + 1);
                    ncd[k] = ls[k] > 0 ? NCART(ls[k] - 1) : 0;
                    int cu[MAXC][3], cdn[MAXC][3], c0[MAXC][3];
                    cart_list(ls[k] + 1, cu);
                    if (haslow) cart_list(ls[k] - 1, cdn);
                    cart_list(ls[k], c0);
                    for (int x = 0; x < 3; x++) {
                        /* derivative block in cartesian components of the original shells */
                        for (int i0 = 0; i0 < nc0[0]; i0++) for (int i1 = 0; i1 < nc0[1]; i1++)
                        for (int i2 = 0; i2 < nc0[2]; i2++) for (int i3 = 0; i3 < nc0[3]; i3++) {
                            int idx[4] = {i0, i1, i2, i3};
                            int ex[3] = {c0[idx[k]][0], c0[idx[k]][1], c0[idx[k]][2]};
                            /* component raised along x */
                            int e2[3] = {ex[0], ex[1], ex[2]};
                            e2[x]++;
                            int iu = -1;
                            for (int z = 0; z < ncu[k]; z++)
                                if (cu[z][0] == e2[0] && cu[z][1] == e2[1] && cu[z][2] == e2[2]) iu = z;
                            int ju[4] = {i0, i1, i2, i3};
                            ju[k] = iu;
                            double v = up[((ju[0] * ncu[1] + ju[1]) * ncu[2] + ju[2]) * ncu[3] + ju[3]];
                            if (ex[x] > 0) {
                                int e3[3] = {ex[0], ex[1], ex[2]};
                                e3[x]--;
                                int id_ = -1;
                                for (int z = 0; z < ncd[k]; z++)
                                    if (cdn[z][0] == e3[0] && cdn[z][1] == e3[1] && cdn[z][2] == e3[2]) id_ = z;
                                int jd[4] = {i0, i1, i2, i3};
                                jd[k] = id_;
                                v -= ex[x] * dn[((jd[0] * ncd[1] + jd[1]) * ncd[2] + jd[2]) * ncd[3] + jd[3]];
                            }
                            der[((i0 * nc0[1] + i1) * nc0[2] + i2) * nc0[3] + i3] = v;
                        }
                        block_to_basis(&bs, ls[0], ls[1], ls[2], ls[3], der, tmp);
                        double s = 0.0;
                        for (int i = 0; i < nb_[0]; i++) for (int j = 0; j < nb_[1]; j++)
                        for (int kk = 0; kk < nb_[2]; kk++) for (int m = 0; m < nb_[3]; m++) {
                            int p = off[a] + i, q = off[b] + j, r = off[c] + kk, s2 = off[d] + m;
                            double gam = 4.0 * D[p * N + q] * D[r * N + s2]
                                         - kx * (D[p * N + r] * D[q * N + s2] + D[p * N + s2] * D[q * N + r]);
                            s += gam * der[((i * nb_[1] + j) * nb_[2] + kk) * nb_[3] + m];
                        }
                        gt[bs.atom[sh[k]] * 3 + x] += f * s;
                    }
                }
            }
        }
#pragma omp critical
        {
            for (int x = 0; x < natom * 3; x++) grad[x] += gt[x];
        }
        free(gt); free(up); free(dn); free(der); free(tmp);
    }
    free(Q);
    free(off);
}

void oracle_grad_2e(BASIS_ARGS, int natom, const double *D, double tau, double *grad)
{
    oracle_grad_2e_kx(nshell, l, nprim, poff, exps, coefs, cen, atom, spherical, natom, D, tau, 1.0, grad);
}

/* ------------------------------------------------------------------------- */
/* one-electron integrals                                                     */
/* ------------------------------------------------------------------------- */

/* primitive cartesian blocks of S, T and V (V summed over the nuclei) for
 * shells of angular momentum la, lb; out[ia*nb + ib]. If dnuc >= 0, V is
 * replaced by the derivative of nucleus dnuc's attraction with respect to
 * that nucleus' coordinate dx (Hellmann-Feynman operator term). */
static void one_e_prim(int la, int lb, double a, double b, const double *A, const double *B,
                       int nnuc, const double *Zn, const double *Cn, int dnuc, int dx,
                       double *S, double *T, double *V)
{
    Etab E[3];
    static __thread Rtab R;
    int ca[MAXC][3], cb[MAXC][3];
    int na = cart_list(la, ca), nb = cart_list(lb, cb);
    double p = a + b, P[3];
    for (int x = 0; x < 3; x++) {
        P[x] = (a * A[x] + b * B[x]) / p;
        hermite_E(la, lb + 2, a, b, A[x] - B[x], E[x]);
    }
    double sp = sqrt(M_PI / p);
    for (int ia = 0; ia < na; ia++)
        for (int ib = 0; ib < nb; ib++) {
            double s1[3], k1[3];
            for (int x = 0; x < 3; x++) {
                int i = ca[ia][x], j = cb[ib][x];
                s1[x] = E[x][i][j][0] * sp;
                /* <i| d^2/dx^2 |j> = 4b^2 S_{i,j+2} - 2b(2j+1) S_{ij} + j(j-1) S_{i,j-2} */
                double d2 = 4 * b * b * E[x][i][j + 2][0] * sp - 2 * b * (2 * j + 1) * E[x][i][j][0] * sp;
                if (j >= 2) d2 += j * (j - 1) * E[x][i][j - 2][0] * sp;
                k1[x] = d2;
            }
            if (S) S[ia * nb + ib] = s1[0] * s1[1] * s1[2];
            if (T) T[ia * nb + ib] = -0.5 * (k1[0] * s1[1] * s1[2] + s1[0] * k1[1] * s1[2] + s1[0] * s1[1] * k1[2]);
        }
    if (!V) return;
    memset(V, 0, sizeof(double) * na * nb);
    int L = la + lb + 1;
    for (int c = 0; c < nnuc; c++) {
        if (dnuc >= 0 && c != dnuc) continue;
        const double *C = Cn + 3 * c;
        hermite_R(L, p, P[0] - C[0], P[1] - C[1], P[2] - C[2], R);
        double pre = -Zn[c] * 2.0 * M_PI / p;
        for (int ia = 0; ia < na; ia++)
            for (int ib = 0; ib < nb; ib++) {
                double s = 0.0;
                for (int t = 0; t <= ca[ia][0] + cb[ib][0]; t++)
                for (int u = 0; u <= ca[ia][1] + cb[ib][1]; u++)
                for (int v = 0; v <= ca[ia][2] + cb[ib][2]; v++) {
                    double r;
                    if (dnuc < 0) r = R[t][u][v];
                    else r = -(dx == 0 ? R[t + 1][u][v] : dx == 1 ? R[t][u + 1][v] : R[t][u][v + 1]);
                    s += E[0][ca[ia][0]][cb[ib][0]][t] * E[1][ca[ia][1]][cb[ib][1]][u] * E[2][ca[ia][2]][cb[ib][2]][v] * r;
                }
                V[ia * nb + ib] += pre * s;
            }
    }
}

/* contracted cartesian S, T, V blocks with bra raised/lowered by dla and bra
 * primitives weighted by 2a when wa != 0 */
static void one_e_contracted(const basis_t *bs, int sa, int sb, int dla, int wa,
                             int nnuc, const double *Zn, const double *Cn, int dnuc, int dx,
                             double *S, double *T, double *V)
{
    int la = bs->l[sa] + dla, lb = bs->l[sb];
    int n = NCART(la) * NCART(lb);
    double s[MAXC * MAXC], t[MAXC * MAXC], v[MAXC * MAXC];
    memset(S, 0, sizeof(double) * n);
    memset(T, 0, sizeof(double) * n);
    memset(V, 0, sizeof(double) * n);
    for (int i = 0; i < bs->nprim[sa]; i++)
        for (int j = 0; j < bs->nprim[sb]; j++) {
            int pi = bs->poff[sa] + i, pj = bs->poff[sb] + j;
            double a = bs->exps[pi], b = bs->exps[pj];
            double w = bs->coefs[pi] * bs->coefs[pj] * (wa ? 2 * a : 1.0);
            one_e_prim(la, lb, a, b, bs->cen + 3 * sa, bs->cen + 3 * sb, nnuc, Zn, Cn, dnuc, dx, s, t, v);
            for (int x = 0; x < n; x++) { S[x] += w * s[x]; T[x] += w * t[x]; V[x] += w * v[x]; }
        }
}

static void pair_to_basis(const basis_t *bs, int la, int lb, double *blk)
{
    double Ta[36], Tb[36], tmp[MAXC * MAXC];
    int na = NCART(la), nb = NCART(lb);
    int fa = cart_to_basis(bs, la, Ta), fb = cart_to_basis(bs, lb, Tb);
    for (int i = 0; i < fa; i++)
        for (int j = 0; j < nb; j++) {
            double s = 0;
            for (int c = 0; c < na; c++) s += Ta[i * na + c] * blk[c * nb + j];
            tmp[i * nb + j] = s;
        }
    for (int i = 0; i < fa; i++)
        for (int j = 0; j < fb; j++) {
            double s = 0;
            for (int c = 0; c < nb; c++) s += Tb[j * nb + c] * tmp[i * nb + c];
            blk[i * fb + j] = s;
        }
}

/* S, T, V matrices [N][N] for nuclei of charges Zn at Cn */
void oracle_one_electron(BASIS_ARGS, int nnuc, const double *Zn, const double *Cn,
                         double *S, double *T, double *V)
{
    MAKE_BASIS;
    int ns = bs.nshell;
    int *off = malloc(sizeof(int) * (ns + 1));
    shell_offsets(&bs, off);
    int N = off[ns];
#pragma omp parallel for schedule(dynamic)
    for (int a = 0; a < ns; a++)
        for (int b = 0; b < ns; b++) {
            double s[MAXC * MAXC], t[MAXC * MAXC], v[MAXC * MAXC];
            one_e_contracted(&bs, a, b, 0, 0, nnuc, Zn, Cn, -1, 0, s, t, v);
            pair_to_basis(&bs, bs.l[a], bs.l[b], s);
            pair_to_basis(&bs, bs.l[a], bs.l[b], t);
            pair_to_basis(&bs, bs.l[a], bs.l[b], v);
            int na = shell_nbf(&bs, a), nb = shell_nbf(&bs, b);
            for (int i = 0; i < na; i++)
                for (int j = 0; j < nb; j++) {
                    S[(off[a] + i) * N + off[b] + j] = s[i * nb + j];
                    T[(off[a] + i) * N + off[b] + j] = t[i * nb + j];
                    V[(off[a] + i) * N + off[b] + j] = v[i * nb + j];
                }
        }
    free(off);
}

/* one-electron gradient:
 *   g_A = sum_mn D_mn dh_mn/dA - sum_mn W_mn dS_mn/dA
 * with h = T + V. Basis-function derivatives act on the bra only and are
 * doubled (D, W, S, h symmetric); the operator term of V differentiates the
 * attraction of nucleus A itself. */
void oracle_grad_1e(BASIS_ARGS, int natom, const double *Zn, const double *Cn,
                    const double *D, const double *W, double *grad)
{
    MAKE_BASIS;
    int ns = bs.nshell;
    int *off = malloc(sizeof(int) * (ns + 1));
    shell_offsets(&bs, off);
    int N = off[ns];
    memset(grad, 0, sizeof(double) * natom * 3);
#pragma omp parallel
    {
        double *gt = calloc((size_t)natom * 3, sizeof(double));
        double su[MAXC * MAXC], tu[MAXC * MAXC], vu[MAXC * MAXC];
        double sd[MAXC * MAXC], td[MAXC * MAXC], vd[MAXC * MAXC];
        double ds[MAXC * MAXC], dh[MAXC * MAXC];
#pragma omp for schedule(dynamic)
        for (int a = 0; a < ns; a++)
            for (int b = 0; b < ns; b++) {
                int la = bs.l[a], lb = bs.l[b];
                int nca = NCART(la), ncb = NCART(lb);
                int ca[MAXC][3], cu[MAXC][3], cdn[MAXC][3];
                cart_list(la, ca);
                cart_list(la + 1, cu);
                if (la > 0) cart_list(la - 1, cdn);
                one_e_contracted(&bs, a, b, +1, 1, natom, Zn, Cn, -1, 0, su, tu, vu);
                if (la > 0) one_e_contracted(&bs, a, b, -1, 0, natom, Zn, Cn, -1, 0, sd, td, vd);
                int na = shell_nbf(&bs, a), nb = shell_nbf(&bs, b);
                for (int x = 0; x < 3; x++) {
                    for (int ia = 0; ia < nca; ia++)
                        for (int ib = 0; ib < ncb; ib++) {
                            int e2[3] = {ca[ia][0], ca[ia][1], ca[ia][2]};
                            e2[x]++;
                            int iu = -1;
                            for (int z = 0; z < NCART(la + 1); z++)
                                if (cu[z][0] == e2[0] && cu[z][1] == e2[1] && cu[z][2] == e2[2]) iu = z;
                            double vs = su[iu * ncb + ib], vh = tu[iu * ncb + ib] + vu[iu * ncb + ib];
                            if (ca[ia][x] > 0) {
                                int e3[3] = {ca[ia][0], ca[ia][1], ca[ia][2]};
                                e3[x]--;
                                int idn = -1;
                                for (int z = 0; z < NCART(la - 1); z++)
                                    if (cdn[z][0] == e3[0] && cdn[z][1] == e3[1] && cdn[z][2] == e3[2]) idn = z;
                                vs -= ca[ia][x] * sd[idn * ncb + ib];
                                vh -= ca[ia][x] * (td[idn * ncb + ib] + vd[idn * ncb + ib]);
                            }
                            ds[ia * ncb + ib] = vs;
                            dh[ia * ncb + ib] = vh;
                        }
                    pair_to_basis(&bs, la, lb, ds);
                    pair_to_basis(&bs, la, lb, dh);
                    double s = 0.0;
                    for (int i = 0; i < na; i++)
                        for (int j = 0; j < nb; j++) {
                            int p = off[a] + i, q = off[b] + j;
                            s += 2.0 * (D[p * N + q] * dh[i * nb + j] - W[p * N + q] * ds[i * nb + j]);
                        }
                    gt[bs.atom[a] * 3 + x] += s;
                }
                /* Hellmann-Feynman: derivative of each nucleus' own attraction */
                for (int c = 0; c < natom; c++)
                    for (int x = 0; x < 3; x++) {
                        double s0[MAXC * MAXC], t0[MAXC * MAXC], v0[MAXC * MAXC];
                        one_e_contracted(&bs, a, b, 0, 0, natom, Zn, Cn, c, x, s0, t0, v0);
                        pair_to_basis(&bs, la, lb, v0);
                        double s = 0.0;
                        for (int i = 0; i < na; i++)
                            for (int j = 0; j < nb; j++)
                                s += D[(off[a] + i) * N + off[b] + j] * v0[i * nb + j];
                        gt[c * 3 + x] += s;
                    }
            }
#pragma omp critical
        {
            for (int x = 0; x < natom * 3; x++) grad[x] += gt[x];
        }
        free(gt);
    }
    free(off);
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Timing samples for the CPU baseline: the same contracted blocks as above  */
/* for a caller-given list of shell quartets (4 ints each); returns the sum  */
/* of |values| so that the work cannot be skipped.                           */
/* ------------------------------------------------------------------------- */
double oracle_eri_list(BASIS_ARGS, int nq, const int *quartets)
{
    MAKE_BASIS;
    double total = 0.0;
#pragma omp parallel for schedule(dynamic) reduction(+ : total)
    for (int q = 0; q < nq; q++) {
        double blk[BLK];
        const int *s = quartets + 4 * q;
        eri_block(&bs, s[0], s[1], s[2], s[3], blk);
        int n = shell_nbf(&bs, s[0]) * shell_nbf(&bs, s[1]) * shell_nbf(&bs, s[2]) * shell_nbf(&bs, s[3]);
        for (int x = 0; x < n; x++) total += fabs(blk[x]);
    }
    return total;
}

/* derivative blocks (raised and lowered on each of the four centres, as in
 * oracle_grad_2e) for a list of quartets */
double oracle_deriv_list(BASIS_ARGS, int nq, const int *quartets)
{
    MAKE_BASIS;
    double total = 0.0;
#pragma omp parallel for schedule(dynamic) reduction(+ : total)
    for (int q = 0; q < nq; q++) {
        double *up = malloc(sizeof(double) * BLK), *dn = malloc(sizeof(double) * BLK);
        const int *sh = quartets + 4 * q;
        for (int k = 0; k < 4; k++) {
            int dl[4] = {0, 0, 0, 0}, w[4] = {0, 0, 0, 0};
            dl[k] = 1;
            w[k] = 1;
            eri_contracted_cart(&bs, sh, dl, w, up);
            total += fabs(up[0]);
            if (bs.l[sh[k]] > 0) {
                dl[k] = -1;
                w[k] = 0;
                eri_contracted_cart(&bs, sh, dl, w, dn);
                total += fabs(dn[0]);
            }
        }
        free(up);
        free(dn);
    }
    return total;
}

/* ------------------------------------------------------------------------- */
/* One block of G = J - K/2 straight from the definitions, for sampled checks  */
/* of large systems: for shells a, b                                          */
/*   J_mn = sum_{c,d} sum_{l in c, s in d} D_ls (mn|ls)                        */
/*   K_mn = sum_{c,d} sum_{l in c, s in d} D_ls (ml|ns)     (m in a, n in b)   */
/* over every ordered shell pair (c, d), no screening and no symmetry.        */
/* ------------------------------------------------------------------------- */
void oracle_g_block(BASIS_ARGS, const double *D, int a, int b, double *out)
{
    MAKE_BASIS;
    int ns = bs.nshell;
    int *off = malloc(sizeof(int) * (ns + 1));
    shell_offsets(&bs, off);
    int N = off[ns];
    int na = shell_nbf(&bs, a), nb = shell_nbf(&bs, b);
    double Jb[25] = {0}, Kb[25] = {0};
#pragma omp parallel
    {
        double Jt[25] = {0}, Kt[25] = {0};
        double blk[BLK];
#pragma omp for schedule(dynamic)
        for (int c = 0; c < ns; c++)
            for (int d = 0; d < ns; d++) {
                int nc = shell_nbf(&bs, c), nd = shell_nbf(&bs, d);
                eri_block(&bs, a, b, c, d, blk); /* (ab|cd) */
                for (int i = 0; i < na; i++)
                    for (int j = 0; j < nb; j++)
                        for (int k = 0; k < nc; k++)
                            for (int m = 0; m < nd; m++)
                                Jt[i * nb + j] += D[(off[c] + k) * N + off[d] + m] * blk[((i * nb + j) * nc + k) * nd + m];
                eri_block(&bs, a, c, b, d, blk); /* (ac|bd) */
                for (int i = 0; i < na; i++)
                    for (int k = 0; k < nc; k++)
                        for (int j = 0; j < nb; j++)
                            for (int m = 0; m < nd; m++)
                                Kt[i * nb + j] += D[(off[c] + k) * N + off[d] + m] * blk[((i * nc + k) * nb + j) * nd + m];
            }
#pragma omp critical
        {
            for (int x = 0; x < na * nb; x++) { Jb[x] += Jt[x]; Kb[x] += Kt[x]; }
        }
    }
    for (int x = 0; x < na * nb; x++) out[x] = Jb[x] - 0.5 * Kb[x];
    free(off);
}
