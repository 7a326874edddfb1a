// Cooperative ERI kernels for the quartet classes with the largest
// recursions ((dd|dd), (dd|dp), (dp|dp), (dd|pp), (dd|ds) and their
// gradients). The same Obara-Saika / Head-Gordon-Pople recursions as the
// straight-line kernels, read from generated op tapes that are sorted into
// dependency levels: the threads of a block (1 to 4 warps) work on one quartet
// at a time, keep every intermediate and accumulator in shared memory, and
// execute the (independent) ops of a level in parallel, with a block barrier
// between levels. The primitive quartets' geometric factors and Boys values
// are computed one per thread, a block's worth at a time. One workspace per
// block rather than per warp lets 2 to 3 times more warps share an SM's shared
// memory for the largest classes, which hides the latency of the tape loads.
// Templated on the arithmetic precision R: FP64, or FP32 for the small
// quartets of the mixed mode (pair data, Boys table and density in FP32; the
// Fock matrix and the gradient accumulate in FP64).
#pragma once
#include "grad_kernels.cuh"

namespace pimd {

struct CoopTape {
    const int* vrr;        // 4 ints per op (see coop_vrr), level-sorted, each level by chain length
    const int* vrr_lv;     // level offsets
    const int* acc;        // 1 int per op: dst | src << 14 | weight << 28 (see coop_accumulate)
    const int* hrr[6];     // HRR tapes, 2 ints per op (energy: [0] only; gradient: Ap Bp Cp Am Bm Cm)
    const int* hrr_lv[6];
    const int* out[6];     // slots of the Cartesian outputs of each HRR tape
    int nvlev, naccop, nhlev[6], nhrr;
    int hpos[6], hup[6];   // centre (0 A, 1 B, 2 C) and direction (1 raised, 0 lowered) of each HRR tape
    int L, NACC, F0, NWORK;
};

template <typename R>
__device__ __forceinline__ R warp_sum_r(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// per primitive quartet in shared memory: PA, WP, QC, WQ (12), o2p, o2pr, o2q,
// o2qr, o2pq (5), 2a, 2b, 2c (3), then F_m * theta (L + 1)
constexpr int COOP_NG0 = 20;
// coefficient table of the primitive quartet being recursed: PA, WP, QC, WQ
// (0..11), then k o2p, -k o2pr, k o2q, -k o2qr, k o2pq for k = 1..5 (12..36)
constexpr int COOP_CT = 37;
constexpr int COOP_KMAX = 5;

// coefficient table ct of one primitive from its geometry g (thread tid of n)
template <typename R>
__device__ __forceinline__ void coop_fill_ct(const R* g, R* ct, int tid, int n)
{
    for (int e = tid; e < COOP_CT; e += n) {
        if (e < 12) {
            ct[e] = g[e];
        } else {
            const int t = (e - 12) / COOP_KMAX, k = (e - 12) % COOP_KMAX + 1;
            const R v = R(k) * g[12 + t];
            ct[e] = (t == 1 || t == 3) ? -v : v;
        }
    }
}

// run the level-sorted VRR of one primitive quartet (coefficients ct) in sm:
// every op is sm[dst] = sum over its 2..5 terms of ct[c_t] sm[s_t], encoded
// as {dst | s1 << 16, s2 | s3 << 16, s4 | s5 << 16, c1 | c2 << 6 | c3 << 12 |
// c4 << 18 | c5 << 24 | (terms - 2) << 30}. The ops of a level are
// independent (they read earlier levels only and write distinct slots), so a
// thread takes two of them at a time and the loads of both overlap.
template <typename R>
__device__ __forceinline__ R coop_vrr_op(const int4 op, const R* sm, const R* ct)
{
    const unsigned w0 = (unsigned)op.x, w1 = (unsigned)op.y, w2 = (unsigned)op.z, w3 = (unsigned)op.w;
    const unsigned n = w3 >> 30;
    R v = ct[w3 & 63] * sm[w0 >> 16];
    v = fma(ct[(w3 >> 6) & 63], sm[w1 & 0xffff], v);
    if (n >= 1) v = fma(ct[(w3 >> 12) & 63], sm[w1 >> 16], v);
    if (n >= 2) v = fma(ct[(w3 >> 18) & 63], sm[w2 & 0xffff], v);
    if (n >= 3) v = fma(ct[(w3 >> 24) & 63], sm[w2 >> 16], v);
    return v;
}

template <typename R>
__device__ __forceinline__ void coop_vrr(const CoopTape& tp, R* sm, const R* ct, int tid, int n)
{
    for (int lv = 0; lv < tp.nvlev; lv++) {
        const int hi = __ldg(tp.vrr_lv + lv + 1);
        int o = __ldg(tp.vrr_lv + lv) + tid;
        for (; o + n < hi; o += 2 * n) {
            const int4 a = __ldg((const int4*)(tp.vrr + 4 * o));
            const int4 b = __ldg((const int4*)(tp.vrr + 4 * (o + n)));
            const R va = coop_vrr_op<R>(a, sm, ct);
            const R vb = coop_vrr_op<R>(b, sm, ct);
            sm[(unsigned)a.x & 0xffff] = va;
            sm[(unsigned)b.x & 0xffff] = vb;
        }
        if (o < hi) {
            const int4 a = __ldg((const int4*)(tp.vrr + 4 * o));
            sm[(unsigned)a.x & 0xffff] = coop_vrr_op<R>(a, sm, ct);
        }
        __syncthreads();
    }
}

// accumulation of one primitive quartet's VRR results into the contracted
// sets: op {dst | src << 14 | weight << 28}, sm[dst] += w[weight] sm[src]
// (w = 1, 2a, 2b, 2c); every accumulator has one op, so the ops are
// independent and a thread takes two at a time
template <typename R>
__device__ __forceinline__ void coop_accumulate(const CoopTape& tp, R* sm, const R w[4], int tid, int n)
{
    auto wsel = [&](unsigned k) { return k == 0 ? w[0] : (k == 1 ? w[1] : (k == 2 ? w[2] : w[3])); };
    int o = tid;
    for (; o + n < tp.naccop; o += 2 * n) {
        const unsigned a = (unsigned)__ldg(tp.acc + o), b = (unsigned)__ldg(tp.acc + o + n);
        const R va = fma(wsel(a >> 28), sm[(a >> 14) & 0x3fff], sm[a & 0x3fff]);
        const R vb = fma(wsel(b >> 28), sm[(b >> 14) & 0x3fff], sm[b & 0x3fff]);
        sm[a & 0x3fff] = va;
        sm[b & 0x3fff] = vb;
    }
    if (o < tp.naccop) {
        const unsigned a = (unsigned)__ldg(tp.acc + o);
        sm[a & 0x3fff] = fma(wsel(a >> 28), sm[(a >> 14) & 0x3fff], sm[a & 0x3fff]);
    }
}

// HRR op {dst | s1 << 16, s2 | c << 16}: sm[dst] = sm[s1] + hc[c] sm[s2],
// hc = (AB_x, AB_y, AB_z, CD_x, CD_y, CD_z)
template <typename R>
__device__ __forceinline__ void coop_hrr(const CoopTape& tp, int h, R* sm, const R hc[6], int tid, int n)
{
    const int* ops = tp.hrr[h];
    const int* lvo = tp.hrr_lv[h];
    auto coef = [&](unsigned c) {
        return c == 0 ? hc[0] : c == 1 ? hc[1] : c == 2 ? hc[2] : c == 3 ? hc[3] : c == 4 ? hc[4] : hc[5];
    };
    for (int lv = 0; lv < tp.nhlev[h]; lv++) {
        const int hi = __ldg(lvo + lv + 1);
        int o = __ldg(lvo + lv) + tid;
        // a level's ops are independent: two per thread at a time
        for (; o + n < hi; o += 2 * n) {
            const int2 p = __ldg((const int2*)(ops + 2 * o)), q = __ldg((const int2*)(ops + 2 * (o + n)));
            const unsigned pa = (unsigned)p.x, pb = (unsigned)p.y, qa = (unsigned)q.x, qb = (unsigned)q.y;
            const R vp = fma(coef(pb >> 16), sm[pb & 0xffff], sm[pa >> 16]);
            const R vq = fma(coef(qb >> 16), sm[qb & 0xffff], sm[qa >> 16]);
            sm[pa & 0xffff] = vp;
            sm[qa & 0xffff] = vq;
        }
        if (o < hi) {
            const int2 p = __ldg((const int2*)(ops + 2 * o));
            const unsigned pa = (unsigned)p.x, pb = (unsigned)p.y;
            sm[pa & 0xffff] = fma(coef(pb >> 16), sm[pb & 0xffff], sm[pa >> 16]);
        }
        __syncthreads();
    }
}

// geometry + Boys of primitive quartet k of (ab|cd) into g (lane-private slot)
template <typename R>
__device__ __forceinline__ void coop_prim(const Pairs& P, int ab, int cd, int k, int npp_ab, int L,
                                          const R* __restrict__ boys, R* g)
{
    const int i = k % npp_ab, j = k / npp_ab;
    R bra[PP_NF], ket[PP_NF];
    load_ppn(P, ab, i, bra, PP_NF);
    load_ppn(P, cd, j, ket, PP_NF);
    PrimQ<R> q;
    prim_quartet<R>(bra, ket, q);
    for (int x = 0; x < 3; x++) {
        g[x] = q.PA[x];
        g[3 + x] = q.WP[x];
        g[6 + x] = q.QC[x];
        g[9 + x] = q.WQ[x];
    }
    g[12] = q.o2p;
    g[13] = q.o2pr;
    g[14] = q.o2q;
    g[15] = q.o2qr;
    g[16] = q.o2pq;
    g[17] = R(2) * bra[PP_EA];
    g[18] = R(2) * bra[PP_EB];
    g[19] = R(2) * ket[PP_EA];
    R F[BOYS_MMAX + 1];
    boys_eval_n(L, q.T, boys, q.theta, F);
    for (int m = 0; m <= L; m++) g[COOP_NG0 + m] = F[m];
}

// contracted accumulators of one quartet: zero, then every primitive quartet
// through the VRR and the accumulation ops. Primitive quartets (i|j) whose
// bound is below qthr are skipped (qthr <= 0: none): qp_i qp_j for the Fock
// build, qg_i qp_j + qp_i qg_j for the gradient (grad); returns the number
// evaluated. All n threads of the block call it (block barriers inside);
// s_cnt: shared scratch of one int per warp.
template <typename R>
__device__ __forceinline__ int coop_primitive_loop(const CoopTape& tp, const Pairs& P, int ab, int cd,
                                                   const R* __restrict__ boys, R* sm, R* geom, R* ct, int tid,
                                                   int n, int* s_cnt, float qthr = 0.0f, bool grad = false)
{
    const int NG = COOP_NG0 + tp.L + 1;
    const int w = tid >> 5, lane = tid & 31, nw = n >> 5;
    for (int i = tid; i < tp.NACC; i += n) sm[i] = R(0);
    const int nab = P.npp[ab], npq = nab * P.npp[cd];
    int done = 0;
    for (int base = 0; base < npq; base += n) {
        const int k = base + tid;
        bool keep = k < npq;
        if (keep && qthr > 0.0f) {
            const size_t i = (size_t)(k % nab) * P.n + ab, j = (size_t)(k / nab) * P.n + cd;
            keep = grad ? __ldg(P.qg + i) * __ldg(P.qp + j) + __ldg(P.qp + i) * __ldg(P.qg + j) >= qthr
                        : __ldg(P.qp + i) * __ldg(P.qp + j) >= qthr;
        }
        // compaction of the surviving primitive quartets over the block: a
        // warp's count, then its offset from the counts of the warps before it
        const unsigned mask = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) s_cnt[w] = __popc(mask);
        __syncthreads();
        int off = 0, nb = 0;
        for (int v = 0; v < nw; v++) {
            const int c = s_cnt[v];
            off += v < w ? c : 0;
            nb += c;
        }
        if (keep) coop_prim<R>(P, ab, cd, k, nab, tp.L, boys, geom + (off + __popc(mask & ((1u << lane) - 1u))) * NG);
        __syncthreads();
        done += nb;
        for (int p = 0; p < nb; p++) {
            const R* g = geom + p * NG;
            if (tid <= tp.L) sm[tp.F0 + tid] = g[COOP_NG0 + tid];
            coop_fill_ct<R>(g, ct, tid, n);
            __syncthreads();
            coop_vrr<R>(tp, sm, ct, tid, n);
            const R wt[4] = {R(1), g[17], g[18], g[19]};
            coop_accumulate<R>(tp, sm, wt, tid, n);
            __syncthreads();
        }
    }
    return done;
}

// one index of a block between Cartesian (nc) and spherical (ns) d components,
// thread-parallel: fwd: in[n0][6][n2] -> out[n0][5][n2]; else the transpose
template <typename R>
__device__ __forceinline__ void coop_sph_pass(const R* in, R* out, int n0, int l, int n2, bool fwd, int tid,
                                              int n)
{
    const R s3 = R(kSqrt3), h = R(0.5), hs3 = R(0.5 * kSqrt3);
    const int nin = l < 2 ? ncart(l) : (fwd ? 6 : 5), nout = l < 2 ? ncart(l) : (fwd ? 5 : 6);
    for (int e = tid; e < n0 * nout * n2; e += n) {
        const int i0 = e / (nout * n2), f = (e / n2) % nout, i2 = e % n2;
        const R* s = in + (size_t)i0 * nin * n2 + i2;
        R v;
        if (l < 2) {
            v = s[f * n2];
        } else if (fwd) {
            const R xx = s[0], xy = s[n2], xz = s[2 * n2], yy = s[3 * n2], yz = s[4 * n2], zz = s[5 * n2];
            v = f == 0 ? s3 * xy
              : f == 1 ? s3 * yz
              : f == 2 ? zz - h * (xx + yy)
              : f == 3 ? s3 * xz
                       : hs3 * (xx - yy);
        } else {
            const R m2 = s[0], m1 = s[n2], m0 = s[2 * n2], p1 = s[3 * n2], p2 = s[4 * n2];
            v = f == 0 ? -h * m0 + hs3 * p2
              : f == 1 ? s3 * m2
              : f == 2 ? s3 * p1
              : f == 3 ? -h * m0 - hs3 * p2
              : f == 4 ? s3 * m1
                       : m0;
        }
        out[e] = v;
    }
    __syncthreads();
}

template <int LA, int LB, int LC, int LD, typename R>
__device__ __forceinline__ void coop_cart_to_sph(R* buf, R* tmp, int tid, int n)
{
    constexpr int cb = ncart(LB), cc = ncart(LC), cd = ncart(LD);
    constexpr int sa = nsph(LA), sb = nsph(LB), sc = nsph(LC);
    coop_sph_pass(buf, tmp, 1, LA, cb * cc * cd, true, tid, n);
    coop_sph_pass(tmp, buf, sa, LB, cc * cd, true, tid, n);
    coop_sph_pass(buf, tmp, sa * sb, LC, cd, true, tid, n);
    coop_sph_pass(tmp, buf, sa * sb * sc, LD, 1, true, tid, n);
}

template <int LA, int LB, int LC, int LD, typename R>
__device__ __forceinline__ void coop_sph_to_cart_t(R* buf, R* tmp, int tid, int n)
{
    constexpr int ca = ncart(LA), cb = ncart(LB), cc = ncart(LC);
    constexpr int sb = nsph(LB), sc = nsph(LC), sd = nsph(LD);
    coop_sph_pass(buf, tmp, 1, LA, sb * sc * sd, false, tid, n);
    coop_sph_pass(tmp, buf, ca, LB, sc * sd, false, tid, n);
    coop_sph_pass(buf, tmp, ca * cb, LC, sd, false, tid, n);
    coop_sph_pass(tmp, buf, ca * cb * cc, LD, 1, false, tid, n);
}

// thread-parallel J/K scatter of a spherical block I (see scatter_jk): the
// contraction in R, the accumulation into G' in FP64
template <int LA, int LB, int LC, int LD, typename R>
__device__ __forceinline__ void coop_scatter_jk(const R* I, double f, int fa, int fb, int fc, int fd, int N,
                                                const R* __restrict__ D, double* G, int tid, int n, double fxs)
{
    constexpr int na = nsph(LA), nb = nsph(LB), nc = nsph(LC), nd = nsph(LD);
#define IDX(a, b, c, d) ((((a) * nb + (b)) * nc + (c)) * nd + (d))
#define DM(i, j) __ldg(D + (size_t)(i) * N + (j))
    for (int e = tid; e < na * nb; e += n) {
        const int a = e / nb, b = e % nb;
        R s = R(0);
        for (int c = 0; c < nc; c++)
            for (int d = 0; d < nd; d++) s += DM(fc + c, fd + d) * I[IDX(a, b, c, d)];
        det_add(G + (size_t)(fa + a) * N + fb + b, 2.0 * f * (double)s, fxs);
    }
    for (int e = tid; e < nc * nd; e += n) {
        const int c = e / nd, d = e % nd;
        R s = R(0);
        for (int a = 0; a < na; a++)
            for (int b = 0; b < nb; b++) s += DM(fa + a, fb + b) * I[IDX(a, b, c, d)];
        det_add(G + (size_t)(fc + c) * N + fd + d, 2.0 * f * (double)s, fxs);
    }
    for (int e = tid; e < na * nc; e += n) {
        const int a = e / nc, c = e % nc;
        R s = R(0);
        for (int b = 0; b < nb; b++)
            for (int d = 0; d < nd; d++) s += DM(fb + b, fd + d) * I[IDX(a, b, c, d)];
        det_add(G + (size_t)(fa + a) * N + fc + c, -0.5 * f * (double)s, fxs);
    }
    for (int e = tid; e < nb * nc; e += n) {
        const int b = e / nc, c = e % nc;
        R s = R(0);
        for (int a = 0; a < na; a++)
            for (int d = 0; d < nd; d++) s += DM(fa + a, fd + d) * I[IDX(a, b, c, d)];
        det_add(G + (size_t)(fb + b) * N + fc + c, -0.5 * f * (double)s, fxs);
    }
    for (int e = tid; e < na * nd; e += n) {
        const int a = e / nd, d = e % nd;
        R s = R(0);
        for (int b = 0; b < nb; b++)
            for (int c = 0; c < nc; c++) s += DM(fb + b, fc + c) * I[IDX(a, b, c, d)];
        det_add(G + (size_t)(fa + a) * N + fd + d, -0.5 * f * (double)s, fxs);
    }
    for (int e = tid; e < nb * nd; e += n) {
        const int b = e / nd, d = e % nd;
        R s = R(0);
        for (int a = 0; a < na; a++)
            for (int c = 0; c < nc; c++) s += DM(fa + a, fc + c) * I[IDX(a, b, c, d)];
        det_add(G + (size_t)(fb + b) * N + fd + d, -0.5 * f * (double)s, fxs);
    }
#undef IDX
#undef DM
}

// shared memory (elements) of one warp
// elements of a block's workspace for nthr threads: accumulators and work
// slots, one geometry record per thread, two Cartesian blocks, the
// coefficient table
__host__ __device__ constexpr int coop_block_elems(int NACC, int NWORK, int L, int ncart4, int nthr)
{
    return NACC + NWORK + nthr * (COOP_NG0 + L + 1) + 2 * ncart4 + COOP_CT;
}

// warps per block: the W in 1..4 (the kernels' launch bound) that maximises W
// x (blocks resident per SM), the SM holding 228 KB of shared memory with 1 KB
// reserved per block and a block at most 227 KB; ties go to the larger block
inline int coop_best_warps(int NACC, int NWORK, int L, int ncart4, size_t elem)
{
    const size_t sm_bytes = 228 * 1024, blk_max = 227 * 1024, reserve = 1024;
    int best = 1;
    size_t best_warps = 0;
    for (int W = 1; W <= 4; W++) {
        const size_t blk = (size_t)coop_block_elems(NACC, NWORK, L, ncart4, 32 * W) * elem;
        if (blk > blk_max) break;
        const size_t warps = (size_t)W * (sm_bytes / (blk + reserve));
        if (warps >= best_warps) {
            best_warps = warps;
            best = W;
        }
    }
    return best;
}

// Fock build of the quartets whose density-weighted bound lies in [tau_lo, tau_hi)
template <int LA, int LB, int LC, int LD, typename Rt>
__global__ void __launch_bounds__(128) jk_coop_kernel(Pairs P, Shells S, Reps R, const Tile* __restrict__ tiles,
                                                      const Rt* __restrict__ Dall, double* __restrict__ Gall,
                                                      const Rt* __restrict__ boys, double tau_lo, double tau_hi,
                                                      const double* __restrict__ Dsh,
                                                      unsigned long long* __restrict__ cnt, CoopTape tp,
                                                      double tau_prim, double fxs)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_cnt[4];
    constexpr int NC4 = ncart(LA) * ncart(LB) * ncart(LC) * ncart(LD);
    const int tid = threadIdx.x, n = blockDim.x;
    Rt* sm = (Rt*)smem_raw;
    Rt* geom = sm + tp.NACC + tp.NWORK;
    Rt* cart = geom + n * (COOP_NG0 + tp.L + 1);
    Rt* tmp = cart + NC4;
    Rt* ct = tmp + NC4;
    const Tile t = tiles[blockIdx.x];
    if (!R.active[t.rep]) return;
    const int ab = t.ab, r = t.rep;
    const int sa = P.sa[ab], sb = P.sb[ab];
    double A[3], B[3];
    for (int x = 0; x < 3; x++) {
        A[x] = S.xyz[3 * sa + x];
        B[x] = S.xyz[3 * sb + x];
    }
    // the block's threads take the tile's quartets one at a time (the bound
    // and hence every branch below is the same for all of them)
    for (int cd = t.c0; cd < t.c1; cd++) {
        const int sc = P.sa[cd], sd = P.sb[cd];
        const double dq = fmax(fmax(fmax(shell_bound(R, Dsh, r, sa, sb), shell_bound(R, Dsh, r, sc, sd)),
                                    fmax(shell_bound(R, Dsh, r, sa, sc), shell_bound(R, Dsh, r, sa, sd))),
                               fmax(shell_bound(R, Dsh, r, sb, sc), shell_bound(R, Dsh, r, sb, sd)));
        const double bound = P.Q[ab] * P.Q[cd] * dq;
        if (bound < tau_lo || bound >= tau_hi) continue;
        double Cc[3], Dd[3];
        for (int x = 0; x < 3; x++) {
            Cc[x] = S.xyz[3 * sc + x];
            Dd[x] = S.xyz[3 * sd + x];
        }
        const int nprim = coop_primitive_loop<Rt>(tp, P, ab, cd, boys, sm, geom, ct, tid, n, s_cnt,
                                                  (float)(tau_prim / dq));
        if (tid == 0) {
            atomicAdd(cnt, 1ull);
            atomicAdd(cnt + 1, (unsigned long long)nprim);
            atomicAdd(R.qrep + 2 * r + (sizeof(Rt) == 4 ? 1 : 0), 1ull);
        }
        const Rt hc[6] = {Rt(A[0] - B[0]), Rt(A[1] - B[1]), Rt(A[2] - B[2]),
                          Rt(Cc[0] - Dd[0]), Rt(Cc[1] - Dd[1]), Rt(Cc[2] - Dd[2])};
        coop_hrr<Rt>(tp, 0, sm, hc, tid, n);
        for (int e = tid; e < NC4; e += n) cart[e] = sm[__ldg(tp.out[0] + e)];
        __syncthreads();
        coop_cart_to_sph<LA, LB, LC, LD, Rt>(cart, tmp, tid, n);
        double f = 1.0;
        if (sa == sb) f *= 0.5;
        if (sc == sd) f *= 0.5;
        if (ab == cd) f *= 0.5;
        const int N = R.nbf[r];
        const size_t off = R.moff[r];
        coop_scatter_jk<LA, LB, LC, LD, Rt>(cart, f, S.bf[sa], S.bf[sb], S.bf[sc], S.bf[sd], N, Dall + off,
                                            Gall + off, tid, n, fxs);
        __syncthreads();
    }
}

// gradient: derivative blocks of the six shifted classes contracted with
// Gamma, for the quartets whose bound Q_ab Q_cd |Gamma| lies in [tau_lo, tau_hi)
template <int LA, int LB, int LC, int LD, typename Rt>
__global__ void __launch_bounds__(128) grad2e_coop_kernel(Pairs P, Shells S, Reps R, const Tile* __restrict__ tiles,
                                                          const double* __restrict__ Dall, double* __restrict__ grad,
                                                          const Rt* __restrict__ boys, double tau_lo, double tau_hi,
                                                          const double* __restrict__ Dsh,
                                                          unsigned long long* __restrict__ cnt, CoopTape tp,
                                                          double tau_prim, double fxs)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_cnt[4];
    __shared__ double s_red[4][9];
    constexpr int NC4 = ncart(LA) * ncart(LB) * ncart(LC) * ncart(LD);
    constexpr int Ls[4] = {LA, LB, LC, LD};
    const int tid = threadIdx.x, n = blockDim.x, w = tid >> 5, lane = tid & 31;
    Rt* sm = (Rt*)smem_raw;
    Rt* geom = sm + tp.NACC + tp.NWORK;
    Rt* gc = geom + n * (COOP_NG0 + tp.L + 1);
    Rt* tmp = gc + NC4;
    Rt* ct = tmp + NC4;
    const Tile t = tiles[blockIdx.x];
    const int ab = t.ab, r = t.rep;
    const int sa = P.sa[ab], sb = P.sb[ab];
    double A[3], B[3];
    for (int x = 0; x < 3; x++) {
        A[x] = S.xyz[3 * sa + x];
        B[x] = S.xyz[3 * sb + x];
    }
    const int N = R.nbf[r];
    const double* D = Dall + R.moff[r];
    // one quartet at a time over the block (uniform branches)
    for (int cd = t.c0; cd < t.c1; cd++) {
        const int sc = P.sa[cd], sd = P.sb[cd];
        const double gam = gamma_bound(R, Dsh, r, sa, sb, sc, sd);
        const double bound = P.Q[ab] * P.Q[cd] * gam;
        if (bound < tau_lo || bound >= tau_hi) continue;
        double Cc[3], Dd[3];
        for (int x = 0; x < 3; x++) {
            Cc[x] = S.xyz[3 * sc + x];
            Dd[x] = S.xyz[3 * sd + x];
        }
        const int nprim = coop_primitive_loop<Rt>(tp, P, ab, cd, boys, sm, geom, ct, tid, n, s_cnt,
                                                  (float)(tau_prim / gam), true);
        if (tid == 0) {
            atomicAdd(cnt, 1ull);
            atomicAdd(cnt + 1, (unsigned long long)nprim);
        }
        // Gamma: spherical, then the transpose transform to Cartesian components
        double f = 1.0;
        if (sa == sb) f *= 0.5;
        if (sc == sd) f *= 0.5;
        if (ab == cd) f *= 0.5;
        {
            constexpr int na = nsph(LA), nb = nsph(LB), nc = nsph(LC), nd = nsph(LD);
            const int fa = S.bf[sa], fb = S.bf[sb], fc = S.bf[sc], fd = S.bf[sd];
            for (int e = tid; e < na * nb * nc * nd; e += n) {
                const int a = e / (nb * nc * nd), b = (e / (nc * nd)) % nb, c = (e / nd) % nc, d = e % nd;
                const double dab = D[(size_t)(fa + a) * N + fb + b], dcd = D[(size_t)(fc + c) * N + fd + d];
                const double dac = D[(size_t)(fa + a) * N + fc + c], dbd = D[(size_t)(fb + b) * N + fd + d];
                const double dad = D[(size_t)(fa + a) * N + fd + d], dbc = D[(size_t)(fb + b) * N + fc + c];
                gc[e] = Rt(f * (4.0 * dab * dcd - dac * dbd - dad * dbc));
            }
            __syncthreads();
            coop_sph_to_cart_t<LA, LB, LC, LD, Rt>(gc, tmp, tid, n);
        }
        const Rt hc[6] = {Rt(A[0] - B[0]), Rt(A[1] - B[1]), Rt(A[2] - B[2]),
                          Rt(Cc[0] - Dd[0]), Rt(Cc[1] - Dd[1]), Rt(Cc[2] - Dd[2])};
        Rt gX[3][3] = {{Rt(0), Rt(0), Rt(0)}, {Rt(0), Rt(0), Rt(0)}, {Rt(0), Rt(0), Rt(0)}};
        // tapes in the order Ap, Bp, Cp, then the lowered ones that exist
        for (int h = 0; h < tp.nhrr; h++) {
            coop_hrr<Rt>(tp, h, sm, hc, tid, n);
            const int pos = tp.hpos[h];
            const bool up = tp.hup[h] != 0;
            const int lp = Ls[pos] + (up ? 1 : -1);
            int nsh4[4] = {ncart(LA), ncart(LB), ncart(LC), ncart(LD)};
            nsh4[pos] = ncart(lp);
            const int* out = tp.out[h];
            for (int e = tid; e < NC4; e += n) {
                int idx[4];
                idx[0] = e / (ncart(LB) * ncart(LC) * ncart(LD));
                idx[1] = (e / (ncart(LC) * ncart(LD))) % ncart(LB);
                idx[2] = (e / ncart(LD)) % ncart(LC);
                idx[3] = e % ncart(LD);
                int ex[3];
                cart_of(Ls[pos], idx[pos], ex[0], ex[1], ex[2]);
                const Rt gm = gc[e];
                for (int x = 0; x < 3; x++) {
                    int eq[3] = {ex[0], ex[1], ex[2]};
                    Rt coef = Rt(1);
                    if (up) {
                        eq[x]++;
                    } else {
                        if (ex[x] == 0) continue;
                        coef = Rt(-ex[x]);
                        eq[x]--;
                    }
                    int j[4] = {idx[0], idx[1], idx[2], idx[3]};
                    j[pos] = cidx(eq[0], eq[1], eq[2]);
                    const int o = ((j[0] * nsh4[1] + j[1]) * nsh4[2] + j[2]) * nsh4[3] + j[3];
                    gX[pos][x] += coef * gm * sm[__ldg(out + o)];
                }
            }
            __syncthreads();
        }
        // sum over the block: the warps' shuffle sums, then thread 0 over the warps
        for (int p = 0; p < 3; p++)
            for (int x = 0; x < 3; x++) {
                const double v = (double)warp_sum_r<Rt>(gX[p][x]);
                if (lane == 0) s_red[w][3 * p + x] = v;
            }
        __syncthreads();
        if (tid == 0) {
            double gd[3][3];
            for (int p = 0; p < 3; p++)
                for (int x = 0; x < 3; x++) {
                    double v = 0.0;
                    for (int v2 = 0; v2 < (n >> 5); v2++) v += s_red[v2][3 * p + x];
                    gd[p][x] = v;
                }
            scatter_grad<double>(grad, S, sa, sb, sc, sd, gd[0], gd[1], gd[2], fxs);
        }
        __syncthreads();
    }
}

}  // namespace pimd
