// Host-side driver and C ABI of the batched RHF library.
//
// One call evaluates every replica of a step (the paper's n replicas, Sec. 2)
// with the same sequence of batched launches:
//   shells/pairs bookkeeping -> primitive-pair data -> Schwarz factors ->
//   sorted pair lists and quartet tiles (cutoff 1e-12, Sec. 3.1) ->
//   S, T, V, h, V_nn -> X = S^{-1/2} -> guess (core Hamiltonian, or the
//   replica's MOs from the previous call, Sec. 2) -> SCF iterations
//   (Fock build, energy, DIIS error, DIIS, diagonalisation, density) with a
//   per-replica convergence mask -> W, one- and two-electron gradient, V_nn.
// Replicas that converge leave the batch while the others keep iterating, so
// the launch never waits on a finished replica (the load imbalance of
// Sec. 3.2 is absorbed inside the batch).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "../../include/pimdgb.h"
#include "boys.cuh"
#include "internal.h"

using namespace pimd;

// ---------------------------------------------------------------------------
// basis
// ---------------------------------------------------------------------------
struct ShellDef {
    int l, nprim;
    double exps[PIMD_MAXPRIM];
    double coefs[PIMD_MAXPRIM];  // normalised (x^l component)
};

struct pimd_basis {
    std::map<int, int> elem;               // Z -> element index
    std::vector<std::vector<ShellDef>> shells;
    std::vector<int> nbf_elem;
    // flattened primitives (element-major, shell order) for the device
    std::vector<double> exps, coefs;
    std::vector<std::vector<int>> prim_off;  // per element, per shell
    long long uid = 0;                       // distinct per basis created in the process
};

static std::atomic<long long> g_basis_uid{1};

static double dfact(int n)
{
    double r = 1.0;
    for (int k = n; k > 1; k -= 2) r *= k;
    return r;
}

// normalised contraction: primitive norm (2a/pi)^{3/4} (4a)^{l/2} / sqrt((2l-1)!!),
// then the contraction scaled so that <phi|phi> = 1 for the x^l component,
// <g_a|g_b> = (pi/(a+b))^{3/2} (2l-1)!! / (2(a+b))^l
static void normalise(ShellDef& s)
{
    const double pi = 3.14159265358979323846;
    double c[PIMD_MAXPRIM];
    for (int i = 0; i < s.nprim; i++) {
        const double a = s.exps[i];
        c[i] = s.coefs[i] * pow(2 * a / pi, 0.75) * pow(4 * a, 0.5 * s.l) / sqrt(dfact(2 * s.l - 1));
    }
    double ov = 0.0;
    for (int i = 0; i < s.nprim; i++)
        for (int j = 0; j < s.nprim; j++) {
            const double p = s.exps[i] + s.exps[j];
            ov += c[i] * c[j] * pow(pi / p, 1.5) * dfact(2 * s.l - 1) / pow(2 * p, s.l);
        }
    for (int i = 0; i < s.nprim; i++) s.coefs[i] = c[i] / sqrt(ov);
}

// ---------------------------------------------------------------------------
// device buffers
// ---------------------------------------------------------------------------
struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

struct pimd_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    double* boys = nullptr;
    float* boysf = nullptr;
    std::map<std::string, DevBuf> bufs;
    std::string last_error;
    pimd_stats stats{};
    // MO cache keyed by replica index
    struct MO {
        std::vector<int> Z;
        int N = 0;
        DevBuf C;   // MO coefficients of the replica's last call
        DevBuf F;   // its final Fock matrix (AO basis)
    };
    std::vector<MO> mo;
    cudaEvent_t ev[8];
    // the class-pair launches of a Fock build (and of the gradient) are
    // spread over the context stream and these side streams (fork/join by
    // events, also inside a captured graph), so that one launch's last wave
    // overlaps the next launches instead of leaving SMs idle
    static constexpr int kSide = 3;
    cudaStream_t side[kSide] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[kSide] = {};
    int nsm = 152;
    pimd_guess* guess_model = nullptr;   // not owned (guess = 2, 3)
    // per class pair: ket width of the quartet tiles (the straight-line
    // Fock kernel's block size), 0 = the cooperative Fock kernel; and the
    // gradient variant (0 cooperative, 1 straight-line). Defaults until
    // pimd_autotune times the alternatives: 128 / straight where generated.
    int tile_w[64];
    int grad_var[64];
    // SAD guess: atomic densities per (basis uid, Z), row-major nbf x nbf
    std::map<std::pair<long long, int>, std::vector<double>> sad;
    // SCF record of the last call: per replica, per iteration (E, error, full build)
    struct TraceRow {
        double E, err;
        int full;
    };
    std::vector<std::vector<TraceRow>> trace;
    // per SCF iteration of the last call: device time of its Fock build (ms,
    // all replicas) and the shell quartets it executed
    std::vector<double> fock_ms_it;
    std::vector<long long> fock_q_it;
};

static int set_err(pimd_ctx* ctx, int code, const std::string& msg)
{
    if (ctx) ctx->last_error = msg;
    return code;
}

#define CK(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return set_err(ctx, PIMD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
static int dev_ensure(pimd_ctx* ctx, const char* name, size_t count, T** out)
{
    DevBuf& b = ctx->bufs[name];
    const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    if (b.cap < bytes) {
        if (b.p) cudaFree(b.p);
        b.p = nullptr;
        b.cap = 0;
        if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return set_err(ctx, PIMD_ENOMEM, std::string("cudaMalloc failed for ") + name);
        }
        b.cap = bytes;
    }
    *out = (T*)b.p;
    return PIMD_OK;
}

#define ENSURE(name, count, ptr)                                   \
    do {                                                           \
        int rc_ = dev_ensure(ctx, name, (size_t)(count), &(ptr)); \
        if (rc_) return rc_;                                       \
    } while (0)

template <typename T>
static int upload(pimd_ctx* ctx, const char* name, const std::vector<T>& v, T** out)
{
    int rc = dev_ensure(ctx, name, v.size(), out);
    if (rc) return rc;
    if (!v.empty()) CK(cudaMemcpyAsync(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    return PIMD_OK;
}

#define UPLOAD(name, vec, ptr)                      \
    do {                                            \
        int rc_ = upload(ctx, name, vec, &(ptr));   \
        if (rc_) return rc_;                        \
    } while (0)

// ---------------------------------------------------------------------------
// C ABI: options, context, basis
// ---------------------------------------------------------------------------
extern "C" void pimd_scf_opts_default(pimd_scf_opts* o)
{
    memset(o, 0, sizeof(*o));
    o->struct_size = sizeof(*o);
    o->conv_energy = 1e-10;
    o->conv_error = 1e-8;
    o->max_iter = 64;
    o->diis_size = 8;
    o->schwarz_tau = 1e-12;
    o->fp32_tau = 0.0;
    o->guess = 0;
    o->deterministic = 0;
    o->want_gradient = 1;
    o->use_graphs = 1;
    o->full_every = 8;
    o->prim_screen = 1.0 / 81.0;
    o->reuse_mode = 0;
    o->split_size = 1;
    o->split_rank = 0;
    o->reduce_fn = nullptr;
    o->reduce_user = nullptr;
}

extern "C" int pimd_ctx_create(pimd_ctx** out, int device)
{
    if (!out) return PIMD_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return PIMD_ECUDA;
    }
    pimd_ctx* ctx = new pimd_ctx();
    ctx->device = device;
    for (int i = 0; i < 64; i++) {
        const bool ok = i < n_class_pairs();
        ctx->tile_w[i] = ok && !class_pair_straight(i) ? 0 : 128;
        ctx->grad_var[i] = ok && !grad_pair_straight(i) ? 0 : 1;
    }
    if (cudaSetDevice(device) != cudaSuccess || cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete ctx;
        return PIMD_ECUDA;
    }
    boys_table_upload(&ctx->boys, &ctx->boysf);
    grad2e_tapes_upload();
    for (int i = 0; i < 8; i++) cudaEventCreate(&ctx->ev[i]);
    cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming);
    for (int i = 0; i < pimd_ctx::kSide; i++) {
        cudaStreamCreateWithFlags(&ctx->side[i], cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&ctx->join_ev[i], cudaEventDisableTiming);
    }
    cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, device);
    if (cudaGetLastError() != cudaSuccess) {
        delete ctx;
        return PIMD_ECUDA;
    }
    *out = ctx;
    return PIMD_OK;
}

extern "C" void pimd_ctx_destroy(pimd_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto& kv : ctx->bufs)
        if (kv.second.p) cudaFree(kv.second.p);
    for (auto& m : ctx->mo) {
        if (m.C.p) cudaFree(m.C.p);
        if (m.F.p) cudaFree(m.F.p);
    }
    if (ctx->boys) cudaFree(ctx->boys);
    if (ctx->boysf) cudaFree(ctx->boysf);
    for (int i = 0; i < 8; i++) cudaEventDestroy(ctx->ev[i]);
    for (int i = 0; i < pimd_ctx::kSide; i++) {
        if (ctx->side[i]) {
            cudaStreamSynchronize(ctx->side[i]);
            cudaStreamDestroy(ctx->side[i]);
        }
        if (ctx->join_ev[i]) cudaEventDestroy(ctx->join_ev[i]);
    }
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    cudaStreamDestroy(ctx->stream);
    delete ctx;
}

extern "C" void pimd_ctx_clear_guess(pimd_ctx* ctx)
{
    if (!ctx) return;
    for (auto& m : ctx->mo) {
        m.Z.clear();
        m.N = 0;
    }
}

extern "C" int pimd_ctx_set_guess_model(pimd_ctx* ctx, pimd_guess* g)
{
    if (!ctx) return PIMD_EINVAL;
    if (g && guess_device(g) != ctx->device) return set_err(ctx, PIMD_EINVAL, "guess model on another device");
    ctx->guess_model = g;
    return PIMD_OK;
}

namespace pimd {
int basis_elem_shells(const pimd_basis* b, int Z, int* l_out, int maxsh)
{
    auto it = b->elem.find(Z);
    if (it == b->elem.end()) return -1;
    const auto& sh = b->shells[it->second];
    for (size_t k = 0; k < sh.size() && (int)k < maxsh; k++) l_out[k] = sh[k].l;
    return (int)sh.size();
}
}  // namespace pimd

extern "C" int pimd_basis_create(pimd_basis** out, int nelem, const int* Z_of_elem, const int* nshell_of_elem,
                                 const int* shell_l, const int* shell_nprim, const double* exps,
                                 const double* coefs, int spherical)
{
    if (!out || nelem <= 0 || !Z_of_elem || !nshell_of_elem || !shell_l || !shell_nprim || !exps || !coefs)
        return PIMD_EINVAL;
    if (spherical != 1) return PIMD_EINVAL;
    pimd_basis* b = new pimd_basis();
    b->uid = g_basis_uid++;
    int s = 0, p = 0;
    for (int e = 0; e < nelem; e++) {
        const int Z = Z_of_elem[e];
        if (Z < 1 || Z > 118 || b->elem.count(Z) || nshell_of_elem[e] <= 0) {
            delete b;
            return PIMD_EINVAL;
        }
        b->elem[Z] = e;
        std::vector<ShellDef> sh;
        std::vector<int> offs;
        int nbf = 0;
        for (int k = 0; k < nshell_of_elem[e]; k++, s++) {
            ShellDef d;
            d.l = shell_l[s];
            d.nprim = shell_nprim[s];
            if (d.l < 0 || d.l > PIMD_LMAX || d.nprim < 1 || d.nprim > PIMD_MAXPRIM) {
                delete b;
                return PIMD_EINVAL;
            }
            for (int i = 0; i < d.nprim; i++, p++) {
                d.exps[i] = exps[p];
                d.coefs[i] = coefs[p];
                if (!(exps[p] > 0.0) || !isfinite(exps[p]) || !isfinite(coefs[p])) {
                    delete b;
                    return PIMD_EINVAL;
                }
            }
            normalise(d);
            offs.push_back((int)b->exps.size());
            for (int i = 0; i < d.nprim; i++) {
                b->exps.push_back(d.exps[i]);
                b->coefs.push_back(d.coefs[i]);
            }
            nbf += nsph(d.l);
            sh.push_back(d);
        }
        b->shells.push_back(sh);
        b->prim_off.push_back(offs);
        b->nbf_elem.push_back(nbf);
    }
    *out = b;
    return PIMD_OK;
}

extern "C" void pimd_basis_destroy(pimd_basis* b) { delete b; }

extern "C" int pimd_basis_nbf(const pimd_basis* b, int natom, const int* Z)
{
    if (!b || natom < 0 || (natom > 0 && !Z)) return PIMD_EINVAL;
    int n = 0;
    for (int i = 0; i < natom; i++) {
        auto it = b->elem.find(Z[i]);
        if (it == b->elem.end()) return PIMD_EINVAL;
        n += b->nbf_elem[it->second];
    }
    return n;
}

extern "C" const char* pimd_strerror(int code)
{
    switch (code) {
        case PIMD_OK: return "ok";
        case PIMD_EINVAL: return "invalid argument";
        case PIMD_ENOMEM: return "device allocation failed";
        case PIMD_ECUDA: return "CUDA runtime error";
        case PIMD_ENOTCONV: return "SCF did not converge for some replica";
        case PIMD_ETIMEOUT: return "bounded device wait expired";
        case PIMD_EBASIS: return "overlap matrix numerically singular";
        default: return "unknown error";
    }
}

extern "C" const char* pimd_last_error(const pimd_ctx* ctx)
{
    if (!ctx) return "";
    return ctx->last_error.c_str();
}

extern "C" int pimd_last_trace(const pimd_ctx* ctx, int rep, int maxit, double* energy, double* error,
                               int* full_build)
{
    if (!ctx || rep < 0 || maxit < 0) return PIMD_EINVAL;
    if (rep >= (int)ctx->trace.size()) return PIMD_EINVAL;
    const auto& t = ctx->trace[rep];
    for (int k = 0; k < (int)t.size() && k < maxit; k++) {
        if (energy) energy[k] = t[k].E;
        if (error) error[k] = t[k].err;
        if (full_build) full_build[k] = t[k].full;
    }
    return (int)t.size();
}

extern "C" int pimd_last_fock_times(const pimd_ctx* ctx, int maxit, double* ms, long long* quartets)
{
    if (!ctx || maxit < 0) return PIMD_EINVAL;
    const int n = (int)ctx->fock_ms_it.size();
    for (int k = 0; k < n && k < maxit; k++) {
        if (ms) ms[k] = ctx->fock_ms_it[k];
        if (quartets) quartets[k] = ctx->fock_q_it[k];
    }
    return n;
}

extern "C" int pimd_last_stats(const pimd_ctx* ctx, pimd_stats* out)
{
    if (!ctx || !out) return PIMD_EINVAL;
    *out = ctx->stats;
    return PIMD_OK;
}

// ---------------------------------------------------------------------------
// batch setup
// ---------------------------------------------------------------------------
struct Batch {
    int nrep = 0;
    bool allow_odd = false;     // isolated atoms of the SAD guess (occupations set by the caller)
    std::vector<int> natom, atom0, nbf, nocc;
    std::vector<int> atom_f0;   // first function of each atom within its replica
    int* d_Zi = nullptr;        // nuclear charges (int) on the device
    std::vector<long long> moff;
    long long mtot = 0;
    int maxN = 0;
    // shells
    std::vector<int> sh_l, sh_bf, sh_atom, sh_rep, sh_prim, sh_nprim;
    std::vector<int> rep_sh0;
    std::vector<int> nsh_rep;
    std::vector<long long> dsoff;
    int maxsh = 0;
    double* Dsh = nullptr;
    std::vector<int> npp;
    unsigned long long* cnt = nullptr;   // [4 * 64] per class pair: executed FP64 quartets and primitive
                                         // quartets, then the same for FP32, of the Fock builds; the
                                         // next [4 * 64] the same for the two-electron gradient
    // pairs grouped by (rep, class)
    std::vector<int> pa, pb;
    std::vector<int> grp0;   // [nrep * 6 + 1] start of group (rep, X)
    // tiles per class pair
    std::vector<std::vector<Tile>> tiles;
    std::vector<long long> nq_cp;
    long long nquart = 0;
    std::vector<long long> nquart_rep;
    double vrr_flops = 0.0;
    double eris = 0.0;
    // device views
    Pairs P{};
    Shells S{};
    Reps R{};
    AtomsDev At{};
    BasisPrimDev B{};
    std::vector<Tile*> d_tiles;
};

static int pair_class(int la, int lb)
{
    // order ss, ps, pp, ds, dp, dd
    static const int t[3][3] = {{0, -1, -1}, {1, 2, -1}, {3, 4, 5}};
    return t[la][lb];
}

static int class_pair_index(int X, int Y)
{
    return X * (X + 1) / 2 + Y;  // X >= Y, same order as the generator
}

// validate and lay out replicas; coordinates already on the device (d_xyz)
static int setup_batch(pimd_ctx* ctx, Batch& bt, int nrep, const int* natom_of, const int* Zc, const double* d_xyz,
                       const pimd_basis* basis, double tau, int split_size = 1, int split_rank = 0)
{
    bt.nrep = nrep;
    bt.natom.assign(natom_of, natom_of + nrep);
    bt.atom0.resize(nrep + 1);
    bt.nbf.resize(nrep);
    bt.nocc.resize(nrep);
    bt.moff.resize(nrep + 1);
    bt.rep_sh0.resize(nrep + 1);
    int a0 = 0;
    long long moff = 0;
    std::vector<double> Zd;
    std::vector<int> atom_rep;
    for (int r = 0; r < nrep; r++) {
        bt.atom0[r] = a0;
        bt.rep_sh0[r] = (int)bt.sh_l.size();
        int nel = 0, nbf = 0;
        for (int i = 0; i < natom_of[r]; i++) {
            const int Z = Zc[a0 + i];
            auto it = basis->elem.find(Z);
            if (it == basis->elem.end()) return set_err(ctx, PIMD_EINVAL, "element missing from basis");
            nel += Z;
            bt.atom_f0.push_back(nbf);
            const int e = it->second;
            for (size_t k = 0; k < basis->shells[e].size(); k++) {
                const ShellDef& d = basis->shells[e][k];
                bt.sh_l.push_back(d.l);
                bt.sh_bf.push_back(nbf);
                bt.sh_atom.push_back(a0 + i);
                bt.sh_rep.push_back(r);
                bt.sh_prim.push_back(basis->prim_off[e][k]);
                bt.sh_nprim.push_back(d.nprim);
                nbf += nsph(d.l);
            }
            Zd.push_back((double)Z);
            atom_rep.push_back(r);
        }
        if (nel % 2 && !bt.allow_odd) return set_err(ctx, PIMD_EINVAL, "odd electron count (RHF needs a closed shell)");
        if (nbf > 768) return set_err(ctx, PIMD_EINVAL, "more than 768 basis functions in one replica");
        bt.nbf[r] = nbf;
        bt.nocc[r] = nel / 2;
        if (bt.nocc[r] > nbf) return set_err(ctx, PIMD_EINVAL, "more occupied orbitals than basis functions");
        bt.moff[r] = moff;
        moff += (long long)nbf * nbf;
        bt.maxN = std::max(bt.maxN, nbf);
        a0 += natom_of[r];
    }
    bt.atom0[nrep] = a0;
    bt.rep_sh0[nrep] = (int)bt.sh_l.size();
    bt.moff[nrep] = moff;
    bt.mtot = moff;
    const int nsh = (int)bt.sh_l.size();

    // pairs grouped by (rep, class)
    std::vector<std::vector<std::pair<int, int>>> groups((size_t)nrep * 6);
    for (int r = 0; r < nrep; r++)
        for (int a = bt.rep_sh0[r]; a < bt.rep_sh0[r + 1]; a++)
            for (int b = bt.rep_sh0[r]; b <= a; b++) {
                int x = a, y = b;
                if (bt.sh_l[y] > bt.sh_l[x]) std::swap(x, y);
                groups[(size_t)r * 6 + pair_class(bt.sh_l[x], bt.sh_l[y])].push_back({x, y});
            }
    bt.grp0.assign((size_t)nrep * 6 + 1, 0);
    bt.pa.clear();
    bt.pb.clear();
    for (size_t g = 0; g < groups.size(); g++) {
        bt.grp0[g] = (int)bt.pa.size();
        for (auto& pr : groups[g]) {
            bt.pa.push_back(pr.first);
            bt.pb.push_back(pr.second);
        }
    }
    bt.grp0[groups.size()] = (int)bt.pa.size();
    const int npair = (int)bt.pa.size();

    // device: atoms, shells
    double* d_Z;
    int *d_atom0, *d_atom_rep;
    UPLOAD("Z", Zd, d_Z);
    {
        std::vector<int> Zi(Zc, Zc + a0);
        UPLOAD("Zi", Zi, bt.d_Zi);
    }
    UPLOAD("atom0", bt.atom0, d_atom0);
    UPLOAD("atom_rep", atom_rep, d_atom_rep);
    bt.At.xyz = d_xyz;
    bt.At.Z = d_Z;
    bt.At.rep_atom0 = d_atom0;
    int *d_l, *d_bf, *d_satom, *d_srep, *d_sprim, *d_snprim;
    UPLOAD("sh_l", bt.sh_l, d_l);
    UPLOAD("sh_bf", bt.sh_bf, d_bf);
    UPLOAD("sh_atom", bt.sh_atom, d_satom);
    UPLOAD("sh_rep", bt.sh_rep, d_srep);
    UPLOAD("sh_prim", bt.sh_prim, d_sprim);
    UPLOAD("sh_nprim", bt.sh_nprim, d_snprim);
    double* d_exps;
    double* d_coefs;
    UPLOAD("b_exps", basis->exps, d_exps);
    UPLOAD("b_coefs", basis->coefs, d_coefs);
    bt.B = BasisPrimDev{d_exps, d_coefs, d_sprim, d_snprim};
    // shell centres gathered from the atom coordinates on the device
    double* d_shxyz;
    ENSURE("sh_xyz", (size_t)nsh * 3, d_shxyz);
    {
        std::vector<int> src(bt.sh_atom);
        int* d_src;
        UPLOAD("sh_src", src, d_src);
        gather_xyz(d_xyz, d_src, nsh, d_shxyz, ctx->stream);
    }
    bt.S = Shells{d_shxyz, d_l, d_bf, d_satom, d_srep};

    // replicas
    int* d_nbf;
    long long* d_moff;
    UPLOAD("nbf", bt.nbf, d_nbf);
    UPLOAD("moff", bt.moff, d_moff);
    int* d_active;
    ENSURE("active", nrep, d_active);
    bt.nsh_rep.resize(nrep);
    bt.dsoff.resize(nrep + 1);
    long long dso = 0;
    for (int r = 0; r < nrep; r++) {
        bt.nsh_rep[r] = bt.rep_sh0[r + 1] - bt.rep_sh0[r];
        bt.maxsh = std::max(bt.maxsh, bt.nsh_rep[r]);
        bt.dsoff[r] = dso;
        dso += (long long)bt.nsh_rep[r] * bt.nsh_rep[r];
    }
    bt.dsoff[nrep] = dso;
    int *d_sh0, *d_nshr;
    long long* d_dsoff;
    UPLOAD("rep_sh0", bt.rep_sh0, d_sh0);
    UPLOAD("nsh_rep", bt.nsh_rep, d_nshr);
    UPLOAD("dsoff", bt.dsoff, d_dsoff);
    ENSURE("Dsh", dso, bt.Dsh);
    ENSURE("cnt", 8 * 64, bt.cnt);
    CK(cudaMemsetAsync(bt.cnt, 0, sizeof(unsigned long long) * 8 * 64, ctx->stream));
    unsigned long long* d_qrep;
    ENSURE("qrep", 2 * nrep, d_qrep);
    CK(cudaMemsetAsync(d_qrep, 0, sizeof(unsigned long long) * 2 * nrep, ctx->stream));
    bt.R = Reps{d_nbf, d_moff, d_active, d_sh0, d_nshr, d_dsoff, d_qrep};

    // pair data, Schwarz factors (unsorted), then sort each group by Q
    int *d_pa, *d_pb, *d_npp;
    double *d_pp, *d_Q;
    UPLOAD("pa", bt.pa, d_pa);
    UPLOAD("pb", bt.pb, d_pb);
    ENSURE("npp", npair, d_npp);
    ENSURE("pp", (size_t)PP_NF * PIMD_MAXPP * npair, d_pp);
    ENSURE("Q", npair, d_Q);
    bt.P = Pairs{npair, d_pa, d_pb, d_npp, d_pp, d_Q, nullptr, nullptr, nullptr};
    launch_pair_data(bt.P, d_npp, d_pp, bt.S, bt.B, ctx->stream);
    ctx->stats.kernel_launches += 2;
    for (int X = 0; X < 6; X++) {
        std::vector<int> list;
        for (int r = 0; r < nrep; r++)
            for (int g = bt.grp0[r * 6 + X]; g < bt.grp0[r * 6 + X + 1]; g++) list.push_back(g);
        if (list.empty()) continue;
        int* d_list;
        std::string nm = "sw_list" + std::to_string(X);
        UPLOAD(nm.c_str(), list, d_list);
        launch_schwarz(X, bt.P, bt.S, d_list, (int)list.size(), ctx->boys, d_Q, ctx->stream);
        ctx->stats.kernel_launches++;
    }
    CK(cudaGetLastError());
    std::vector<double> Q(npair);
    std::vector<int> npp(npair);
    if (npair) {
        CK(cudaMemcpyAsync(Q.data(), d_Q, sizeof(double) * npair, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(npp.data(), d_npp, sizeof(int) * npair, cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    for (int q = 0; q < npair; q++)
        if (!isfinite(Q[q])) return set_err(ctx, PIMD_EINVAL, "non-finite integrals (check coordinates)");
    {
        // each (replica, class) group ordered by primitive-pair count, then by
        // Schwarz factor (descending): ket pairs of a warp then run the same
        // number of primitive iterations, and each equal-count run is sorted by Q
        std::vector<int> perm(npair);
        for (int i = 0; i < npair; i++) perm[i] = i;
        for (size_t g = 0; g + 1 < bt.grp0.size(); g++)
            std::stable_sort(perm.begin() + bt.grp0[g], perm.begin() + bt.grp0[g + 1], [&](int x, int y) {
                return npp[x] != npp[y] ? npp[x] > npp[y] : Q[x] > Q[y];
            });
        std::vector<int> pa2(npair), pb2(npair), npp2(npair);
        std::vector<double> Q2(npair);
        for (int i = 0; i < npair; i++) {
            pa2[i] = bt.pa[perm[i]];
            pb2[i] = bt.pb[perm[i]];
            Q2[i] = Q[perm[i]];
            npp2[i] = npp[perm[i]];
        }
        bt.pa.swap(pa2);
        bt.pb.swap(pb2);
        Q.swap(Q2);
        bt.npp.swap(npp2);
        UPLOAD("pa", bt.pa, d_pa);
        UPLOAD("pb", bt.pb, d_pb);
        UPLOAD("Q", Q, d_Q);
        float* d_ppf;
        ENSURE("ppf", (size_t)PP_NF * PIMD_MAXPP * npair, d_ppf);
        float *d_qp, *d_qg;
        ENSURE("qp", (size_t)PIMD_MAXPP * npair, d_qp);
        ENSURE("qg", (size_t)PIMD_MAXPP * npair, d_qg);
        bt.P = Pairs{npair, d_pa, d_pb, d_npp, d_pp, d_Q, d_ppf, d_qp, d_qg};
        launch_pair_data(bt.P, d_npp, d_pp, bt.S, bt.B, ctx->stream);
        // primitive-pair bounds, and each pair's primitives in descending order of them
        for (int X = 0; X < 6; X++) {
            std::vector<int> list;
            for (int r = 0; r < nrep; r++)
                for (int g = bt.grp0[r * 6 + X]; g < bt.grp0[r * 6 + X + 1]; g++) list.push_back(g);
            if (list.empty()) continue;
            int* d_list;
            std::string nm = "psw_list" + std::to_string(X);
            UPLOAD(nm.c_str(), list, d_list);
            launch_prim_schwarz(X, bt.P, bt.S, d_list, (int)list.size(), ctx->boys, d_pp, d_qp, d_qg, ctx->stream);
            ctx->stats.kernel_launches++;
        }
        launch_to_float(d_pp, d_ppf, (long long)PP_NF * PIMD_MAXPP * npair, ctx->stream);
    }
    // quartet tiles: for bra pair i of class X and each run of ket pairs of
    // class Y <= X with equal primitive count, the ket pairs with
    // Q_j >= tau / Q_i form a prefix of the run; for X == Y only kets at or
    // before i are canonical (ab >= cd).
    const int ncp = n_class_pairs();
    bt.tiles.assign(ncp, {});
    bt.nq_cp.assign(ncp, 0);
    bt.nquart = 0;
    bt.nquart_rep.assign(nrep, 0);
    bt.vrr_flops = 0.0;
    bt.eris = 0.0;
    for (int X = 0; X < 6; X++)
        for (int Y = 0; Y <= X; Y++) {
            const int cp = class_pair_index(X, Y);
            const int tw = ctx->tile_w[cp] > 0 ? ctx->tile_w[cp] : 128;
            auto& tl = bt.tiles[cp];
            for (int r = 0; r < nrep; r++) {
                const int b0 = bt.grp0[r * 6 + X], b1 = bt.grp0[r * 6 + X + 1];
                const int k0 = bt.grp0[r * 6 + Y], k1 = bt.grp0[r * 6 + Y + 1];
                for (int i = b0; i < b1; i++) {
                    if (Q[i] <= 0.0) continue;
                    const double thr = tau / Q[i];
                    for (int s0 = k0; s0 < k1;) {
                        int s1 = s0;
                        while (s1 < k1 && bt.npp[s1] == bt.npp[s0]) s1++;
                        // first index in [s0, s1) with Q < thr (Q descending within the run)
                        int lo = s0, hi = s1;
                        while (lo < hi) {
                            const int mid = (lo + hi) / 2;
                            if (Q[mid] >= thr) lo = mid + 1;
                            else hi = mid;
                        }
                        int kend = lo;
                        if (X == Y) kend = std::min(kend, i + 1);
                        if (kend > s0) {
                            const long long nqi = kend - s0;
                            bt.nq_cp[cp] += nqi;
                            bt.nquart_rep[r] += nqi;
                            for (int c = s0; c < kend; c += tw) tl.push_back(Tile{i, c, std::min(c + tw, kend), r});
                        }
                        s0 = s1;
                    }
                }
            }
            bt.nquart += bt.nq_cp[cp];
        }
    if (split_size > 1) {
        // force-parallel split of every replica over split_size processes: this
        // process keeps every split_size-th tile of each class pair (the counts
        // above stay those of the whole batch)
        for (int cp = 0; cp < ncp; cp++) {
            std::vector<Tile> mine;
            for (size_t i = split_rank; i < bt.tiles[cp].size(); i += split_size) mine.push_back(bt.tiles[cp][i]);
            bt.tiles[cp].swap(mine);
        }
    }
    bt.d_tiles.assign(ncp, nullptr);
    for (int cp = 0; cp < ncp; cp++) {
        if (bt.tiles[cp].empty()) continue;
        std::string nm = "tiles" + std::to_string(cp);
        UPLOAD(nm.c_str(), bt.tiles[cp], bt.d_tiles[cp]);
    }
    CK(cudaGetLastError());
    return PIMD_OK;
}

// ---------------------------------------------------------------------------
// SCF
// ---------------------------------------------------------------------------
struct Mats {
    double *S, *H, *T, *V, *X, *F, *G, *D, *Fb, *M1, *M2, *Er, *C, *Cp, *W, *Ev, *work, *Cs, *Cq;
    double *Fh, *Eh, *Bd, *coef;
    double *E, *emax, *enn;
    double *Dp, *dD;
    int *slot, *count, *diis_on, *active, *fin, *mode;
    int* jnc;   // per replica: the eigensolver hit its sweep limit in this call
    long long stride = 0;   // elements between one replica's DIIS history matrices
    RepMat* rm;
    int ldE;
};

static int alloc_mats(pimd_ctx* ctx, Batch& bt, Mats& m, int hist)
{
    const long long mt = bt.mtot;
    ENSURE("S", mt, m.S);
    ENSURE("H", mt, m.H);
    ENSURE("T", mt, m.T);
    ENSURE("V", mt, m.V);
    ENSURE("X", mt, m.X);
    ENSURE("F", mt, m.F);
    ENSURE("G", mt, m.G);
    ENSURE("D", mt, m.D);
    ENSURE("Fb", mt, m.Fb);
    ENSURE("M1", mt, m.M1);
    ENSURE("M2", mt, m.M2);
    ENSURE("Er", mt, m.Er);
    ENSURE("C", mt, m.C);
    ENSURE("Cp", mt, m.Cp);
    ENSURE("Cq", mt, m.Cq);
    ENSURE("W", mt, m.W);
    ENSURE("work", mt, m.work);
    ENSURE("Cs", mt, m.Cs);
    ENSURE("Dp", mt, m.Dp);
    ENSURE("dD", mt, m.dD);
    ENSURE("mode", bt.nrep, m.mode);
    m.ldE = bt.maxN;
    ENSURE("Ev", (size_t)bt.nrep * m.ldE, m.Ev);
    const long long stride = (long long)bt.maxN * bt.maxN;
    ENSURE("Fh", (size_t)bt.nrep * hist * stride, m.Fh);
    ENSURE("Eh", (size_t)bt.nrep * hist * stride, m.Eh);
    ENSURE("Bd", (size_t)bt.nrep * hist * hist, m.Bd);
    ENSURE("coef", (size_t)bt.nrep * hist, m.coef);
    ENSURE("E", bt.nrep, m.E);
    ENSURE("emax", bt.nrep, m.emax);
    ENSURE("enn", bt.nrep, m.enn);
    ENSURE("slot", bt.nrep, m.slot);
    ENSURE("count", bt.nrep, m.count);
    ENSURE("diis_on", bt.nrep, m.diis_on);
    ENSURE("fin", bt.nrep, m.fin);
    ENSURE("jac_nc", bt.nrep, m.jnc);
    CK(cudaMemsetAsync(m.jnc, 0, sizeof(int) * bt.nrep, ctx->stream));
    m.active = (int*)bt.R.active;
    std::vector<RepMat> rm(bt.nrep);
    for (int r = 0; r < bt.nrep; r++) rm[r] = RepMat{bt.nbf[r], bt.nocc[r], bt.moff[r]};
    UPLOAD("rm", rm, m.rm);
    m.stride = stride;
    return PIMD_OK;
}

struct GemmSet {
    GemmDesc* d = nullptr;
    int n = 0, maxM = 0, maxN = 0;
};

// per-replica GEMM descriptors: C = alpha op(A) op(B) + beta C, square N x N
// unless K is the occupied count
static int make_gemm(pimd_ctx* ctx, const char* name, const Batch& bt, const double* A, int ta, const double* B,
                     int tb, double* C, double alpha, bool kocc, GemmSet& gs, double beta = 0.0)
{
    std::vector<GemmDesc> v(bt.nrep);
    for (int r = 0; r < bt.nrep; r++) {
        const int N = bt.nbf[r];
        const long long o = bt.moff[r];
        v[r] = GemmDesc{N, N, kocc ? bt.nocc[r] : N, A + o, N, ta, B + o, N, tb, C + o, N, alpha, beta, r};
    }
    UPLOAD(name, v, gs.d);
    gs.n = bt.nrep;
    gs.maxM = gs.maxN = bt.maxN;
    return PIMD_OK;
}

struct ScfPlan {
    GemmSet FD, FDS, XtE, XtEX, XtF, XtFX, QtF, FQ, QU, XC, Dn, Wn;
    GemmSet DS, DSD, DSDS, Pur;   // McWeeny step of a reused density in the new overlap metric
};

static int make_plan(pimd_ctx* ctx, const Batch& bt, Mats& m, ScfPlan& p)
{
    int rc;
    if ((rc = make_gemm(ctx, "g_FD", bt, m.F, 0, m.D, 0, m.M1, 1.0, false, p.FD))) return rc;
    if ((rc = make_gemm(ctx, "g_FDS", bt, m.M1, 0, m.S, 0, m.M2, 1.0, false, p.FDS))) return rc;
    if ((rc = make_gemm(ctx, "g_XtE", bt, m.X, 1, m.Er, 0, m.M1, 1.0, false, p.XtE))) return rc;
    if ((rc = make_gemm(ctx, "g_XtEX", bt, m.M1, 0, m.X, 0, m.M2, 1.0, false, p.XtEX))) return rc;
    if ((rc = make_gemm(ctx, "g_XtF", bt, m.X, 1, m.Fb, 0, m.M1, 1.0, false, p.XtF))) return rc;
    if ((rc = make_gemm(ctx, "g_XtFX", bt, m.M1, 0, m.X, 0, m.Cs, 1.0, false, p.XtFX))) return rc;
    if ((rc = make_gemm(ctx, "g_QtF", bt, m.Cq, 1, m.Cs, 0, m.M1, 1.0, false, p.QtF))) return rc;
    if ((rc = make_gemm(ctx, "g_FQ", bt, m.M1, 0, m.Cq, 0, m.M2, 1.0, false, p.FQ))) return rc;
    if ((rc = make_gemm(ctx, "g_QU", bt, m.Cq, 0, m.Cp, 0, m.M1, 1.0, false, p.QU))) return rc;
    if ((rc = make_gemm(ctx, "g_XC", bt, m.X, 0, m.Cq, 0, m.C, 1.0, false, p.XC))) return rc;

    if ((rc = make_gemm(ctx, "g_Dn", bt, m.C, 0, m.C, 1, m.D, 2.0, true, p.Dn))) return rc;
    if ((rc = make_gemm(ctx, "g_Wn", bt, m.Cs, 0, m.C, 1, m.W, 2.0, true, p.Wn))) return rc;
    // D <- 3/4 D S D - 1/4 D S D S D (P = D/2: P <- 3 PSP - 2 PSPSP), result in M2
    if ((rc = make_gemm(ctx, "g_DS", bt, m.D, 0, m.S, 0, m.M1, 1.0, false, p.DS))) return rc;
    if ((rc = make_gemm(ctx, "g_DSD", bt, m.M1, 0, m.D, 0, m.M2, 0.75, false, p.DSD))) return rc;
    if ((rc = make_gemm(ctx, "g_DSDS", bt, m.M2, 0, m.S, 0, m.Er, 4.0 / 3.0, false, p.DSDS))) return rc;
    // (the last product accumulates onto 3/4 DSD already in M2)
    if ((rc = make_gemm(ctx, "g_Pur", bt, m.Er, 0, m.D, 0, m.M2, -0.25, false, p.Pur, 1.0))) return rc;
    return PIMD_OK;
}

static void gemm(pimd_ctx* ctx, const GemmSet& g, const int* mask)
{
    launch_gemm(g.d, g.n, g.maxM, g.maxN, mask, ctx->stream);
    ctx->stats.kernel_launches++;
}

// Fbar -> F' = X^T Fbar X, diagonalised in the basis of the previous
// eigenvectors Q (F'' = Q^T F' Q is nearly diagonal, so the Jacobi sweeps start
// close to convergence) -> Q <- Q U, C = X Q, D = 2 C_occ C_occ^T (replicas in mask)
static void diag_density(pimd_ctx* ctx, const Batch& bt, Mats& m, ScfPlan& p, const int* mask)
{
    gemm(ctx, p.XtF, mask);
    gemm(ctx, p.XtFX, mask);   // F' -> Cs
    gemm(ctx, p.QtF, mask);
    gemm(ctx, p.FQ, mask);     // F'' -> M2
    launch_jacobi(m.rm, bt.nrep, m.M2, m.Cp, m.Ev, m.ldE, m.work, mask, 1, ctx->stream, m.jnc);
    gemm(ctx, p.QU, mask);     // Q U -> M1
    launch_copy_mats(m.rm, bt.nrep, m.M1, m.Cq, mask, ctx->stream);
    gemm(ctx, p.XC, mask);
    gemm(ctx, p.Dn, mask);
    ctx->stats.kernel_launches += 2;
}

// Launch fn(cp, stream) for every class pair with tiles, the k-th on stream
// k mod (side streams + 1) (0: the context stream), after everything already
// queued on the context stream; the context stream then waits for all of them.
template <class Fn>
static int fan_out_class_pairs(pimd_ctx* ctx, const Batch& bt, Fn&& fn)
{
    constexpr int ns = pimd_ctx::kSide + 1;
    CK(cudaEventRecord(ctx->fork_ev, ctx->stream));
    bool used[pimd_ctx::kSide] = {};
    int k = 0;
    for (int cp = 0; cp < n_class_pairs(); cp++) {
        if (bt.tiles[cp].empty()) continue;
        const int j = k++ % ns;
        cudaStream_t st = ctx->stream;
        if (j > 0) {
            st = ctx->side[j - 1];
            if (!used[j - 1]) {
                CK(cudaStreamWaitEvent(st, ctx->fork_ev, 0));
                used[j - 1] = true;
            }
        }
        fn(cp, st);
    }
    for (int i = 0; i < pimd_ctx::kSide; i++)
        if (used[i]) {
            CK(cudaEventRecord(ctx->join_ev[i], ctx->side[i]));
            CK(cudaStreamWaitEvent(ctx->stream, ctx->join_ev[i], 0));
        }
    return PIMD_OK;
}

// G' += G'(M) over all class pairs for the replicas in the active mask, with
// the quartets screened by Q_ab Q_cd max|M block| >= tau; those below fp32_tau
// (if > 0) are evaluated in FP32 from Mf, an FP32 copy of M made here
static int fock_build(pimd_ctx* ctx, Batch& bt, Mats& m, double tau, double fp32_tau, const double* M,
                      double tau_prim, double fxs)
{
    // deterministic mode: the build accumulates into G' as fixed-point integers
    if (fxs > 0) launch_double_to_fixed(m.G, bt.mtot, fxs, ctx->stream);
    launch_shell_bounds(bt.S, bt.R, bt.nrep, bt.maxsh, M, bt.Dsh, bt.R.active, ctx->stream);
    ctx->stats.kernel_launches++;
    float* Mf = nullptr;
    if (fp32_tau > tau) {
        ENSURE("Mf", bt.mtot, Mf);
        launch_to_float(M, Mf, bt.mtot, ctx->stream);
        ctx->stats.kernel_launches++;
    }
    const int rc = fan_out_class_pairs(ctx, bt, [&](int cp, cudaStream_t st) {
        launch_jk(cp, bt.P, bt.S, bt.R, bt.d_tiles[cp], (int)bt.tiles[cp].size(), M, Mf, m.G, ctx->boys, ctx->boysf,
                  tau, fp32_tau, bt.Dsh, bt.cnt + 4 * cp, ctx->tile_w[cp], tau_prim, fxs, st);
        ctx->stats.kernel_launches += fp32_tau > tau ? 2 : 1;
    });
    if (rc) return rc;
    if (fxs > 0) {
        launch_fixed_to_double(m.G, bt.mtot, fxs, ctx->stream);
        ctx->stats.kernel_launches += 2;
    }
    return PIMD_OK;
}

// ---------------------------------------------------------------------------
// SAD guess: superposition of spherically averaged atomic densities
// ---------------------------------------------------------------------------
// Each element's density comes from an SCF of the isolated neutral atom in
// the same basis, with the configuration 1s^2 2s^2 2p^n (Z <= 10) and the
// partly filled p shell spread evenly over its three orbitals, so that the
// density stays spherical. Orbitals are occupied by angular momentum (the
// lowest s orbitals, then the lowest p triplet), not by energy order: in a
// fractional-occupation atomic SCF the 2s can rise above the 2p. The atom's
// Fock matrix has no s-p-d mixing, so every eigenvector has one l.
// Integrals, Fock builds, diagonalisations and densities run in the kernels
// of the molecular SCF; the host picks the occupied orbitals from the
// eigenvectors' l and stops when no density element changes by 1e-9 or more.
static int sad_atomic(pimd_ctx* ctx, const pimd_basis* basis, const std::vector<int>& Zs)
{
    const int n = (int)Zs.size();
    std::vector<int> natom(n, 1);
    std::vector<double> xyz(3 * (size_t)n, 0.0);
    double* d_xyz;
    UPLOAD("sad_xyz", xyz, d_xyz);
    Batch bt;
    bt.allow_odd = true;
    int rc = setup_batch(ctx, bt, n, natom.data(), Zs.data(), d_xyz, basis, 1e-12);
    if (rc) return rc;
    // per replica (atom): angular momentum of every function
    std::vector<std::vector<int>> lfun(n);
    for (int r = 0; r < n; r++) {
        for (int sh = bt.rep_sh0[r]; sh < bt.rep_sh0[r + 1]; sh++)
            for (int k = 0; k < nsph(bt.sh_l[sh]); k++) lfun[r].push_back(bt.sh_l[sh]);
        bt.nocc[r] = bt.nbf[r];   // densities over all columns, unoccupied ones weighted 0
    }
    Mats m;
    if ((rc = alloc_mats(ctx, bt, m, 2))) return rc;
    ScfPlan plan;
    if ((rc = make_plan(ctx, bt, m, plan))) return rc;
    std::vector<int> active(n, 1), mode(n, 2);
    UPLOAD("active", active, m.active);
    bt.R.active = m.active;
    int* d_mode;
    UPLOAD("sad_mode", mode, d_mode);
    cudaStream_t st = ctx->stream;
    launch_one_electron(bt.P, bt.S, bt.B, bt.At, bt.R, m.S, m.T, m.V, ctx->boys, st);
    add_mats(m.rm, n, m.T, m.V, m.H, st);
    CK(cudaMemsetAsync(m.enn, 0, sizeof(double) * n, st));
    launch_jacobi(m.rm, n, m.S, m.Cp, m.Ev, m.ldE, m.work, nullptr, 0, st);
    launch_orth_from_eig(m.rm, n, m.Cp, m.Ev, m.ldE, m.X, st);
    launch_copy_mats(m.rm, n, m.H, m.Fb, nullptr, st);
    std::vector<double> C(bt.mtot), ev((size_t)n * m.ldE), half((size_t)n * m.ldE);
    // Fb -> orbitals -> D = sum_k occ_k C_k C_k^T (W = 2 Cs C^T with Cs = C occ/2)
    auto density = [&]() -> int {
        launch_identity(m.rm, n, m.Cq, nullptr, st);
        diag_density(ctx, bt, m, plan, nullptr);
        CK(cudaMemcpyAsync(C.data(), m.C, sizeof(double) * bt.mtot, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(ev.data(), m.Ev, sizeof(double) * ev.size(), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        std::fill(half.begin(), half.end(), 0.0);
        for (int r = 0; r < n; r++) {
            const int N = bt.nbf[r];
            const double* Cr = C.data() + bt.moff[r];
            std::vector<int> ls(N);
            for (int k = 0; k < N; k++) {
                double w[3] = {0.0, 0.0, 0.0};
                for (int i = 0; i < N; i++) w[lfun[r][i]] += Cr[(size_t)i * N + k] * Cr[(size_t)i * N + k];
                ls[k] = (int)(std::max_element(w, w + 3) - w);
            }
            int left = Zs[r], ns = 0, np = 0;
            std::vector<int> pk;
            for (int k = 0; k < N; k++) {   // eigenvalues ascending
                if (ls[k] == 0 && ns < 2 && left > 0) {
                    const int x = std::min(left, 2);
                    half[(size_t)r * m.ldE + k] = 0.5 * x;
                    left -= x;
                    ns++;
                } else if (ls[k] == 1 && np < 3) {
                    pk.push_back(k);
                    np++;
                }
            }
            if (left > 0) {
                if ((int)pk.size() < 3 || left > 6) return PIMD_EINVAL;
                for (int k : pk) half[(size_t)r * m.ldE + k] = 0.5 * left / 3.0;
            }
        }
        double* d_half;
        UPLOAD("sad_half", half, d_half);
        launch_scale_cols(m.rm, n, m.C, d_half, m.ldE, m.Cs, nullptr, st);
        gemm(ctx, plan.Wn, nullptr);
        launch_copy_mats(m.rm, n, m.W, m.D, nullptr, st);
        return PIMD_OK;
    };
    std::vector<double> D(bt.mtot), Dn(bt.mtot);
    auto fetch = [&](std::vector<double>& out) -> int {
        CK(cudaMemcpyAsync(out.data(), m.D, sizeof(double) * bt.mtot, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        return PIMD_OK;
    };
    if ((rc = density())) return set_err(ctx, rc, "SAD: atom without a 2p shell in the basis");
    if ((rc = fetch(D))) return rc;
    bool conv = false;
    for (int it = 1; it <= 200 && !conv; it++) {
        launch_delta_density(m.rm, n, m.D, m.Dp, m.dD, m.G, d_mode, st);
        // fixed-point accumulation: the cached atomic densities do not depend on
        // the order of the additions
        if ((rc = fock_build(ctx, bt, m, 1e-12, 0.0, m.dD, 0.0, kFixG))) return rc;
        launch_fock_assemble(m.rm, n, m.H, m.G, m.F, m.active, st);
        launch_copy_mats(m.rm, n, m.F, m.Fb, nullptr, st);
        if ((rc = density())) return set_err(ctx, rc, "SAD: atom without a 2p shell in the basis");
        if ((rc = fetch(Dn))) return rc;
        double diff = 0.0;
        for (long long e = 0; e < bt.mtot; e++) {
            if (!std::isfinite(Dn[e])) return set_err(ctx, PIMD_ECUDA, "SAD: non-finite atomic density");
            diff = std::max(diff, fabs(Dn[e] - D[e]));
        }
        D.swap(Dn);
        conv = diff < 1e-9;
    }
    // an atomic SCF still short of the 1e-9 bound after 200 cycles keeps its last
    // density: the molecular SCF converges from any starting density
    CK(cudaGetLastError());
    for (int r = 0; r < n; r++)
        ctx->sad[{basis->uid, Zs[r]}] =
            std::vector<double>(D.begin() + bt.moff[r], D.begin() + bt.moff[r] + (size_t)bt.nbf[r] * bt.nbf[r]);
    return PIMD_OK;
}

// atomic densities of every element in Zc[0..natot) present in the cache
static int sad_ensure(pimd_ctx* ctx, const pimd_basis* basis, const int* Zc, int natot)
{
    std::vector<int> need;
    for (int a = 0; a < natot; a++) {
        const int Z = Zc[a];
        if (Z < 1 || Z > 10) return set_err(ctx, PIMD_EINVAL, "SAD guess: elements up to Z = 10 only");
        if (!basis->elem.count(Z)) return set_err(ctx, PIMD_EINVAL, "element missing from basis");
        if (!ctx->sad.count({basis->uid, Z}) && std::find(need.begin(), need.end(), Z) == need.end())
            need.push_back(Z);
    }
    if (need.empty()) return PIMD_OK;
    return sad_atomic(ctx, basis, need);
}

extern "C" int pimd_sad_atomic_density(pimd_ctx* ctx, const pimd_basis* basis, int Z, double* D, int n)
{
    if (!ctx || !basis || !D) return PIMD_EINVAL;
    auto it = basis->elem.find(Z);
    if (it == basis->elem.end() || basis->nbf_elem[it->second] != n) return PIMD_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return PIMD_ECUDA;
    int rc = sad_ensure(ctx, basis, &Z, 1);
    if (rc) return rc;
    const auto& Da = ctx->sad.at({basis->uid, Z});
    std::copy(Da.begin(), Da.end(), D);
    return PIMD_OK;
}

// One segment of an SCF iteration's kernel sequence. The first use runs the
// launches directly (one-time set-up such as tape uploads happens there); the
// second captures them on the context stream into a CUDA graph, which that
// and every later use replays. Every argument of the captured launches is a
// device pointer or a scalar fixed for the whole call (per-iteration values
// such as build modes, DIIS slots and active masks live in device buffers
// that the host refreshes between graph launches), so a replay performs
// exactly the launches of a direct run.
struct GraphSeg {
    cudaGraphExec_t exec = nullptr;
    int uses = 0;
    long long launches = 0;   // kernel launches of one run, counted on the direct run
    ~GraphSeg()
    {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

template <class Body>
static int run_seg(pimd_ctx* ctx, GraphSeg& sg, bool use_graph, Body&& body)
{
    const int use = sg.uses++;
    if (!use_graph || use == 0) {
        const long long k0 = ctx->stats.kernel_launches;
        const int rc = body();
        sg.launches = ctx->stats.kernel_launches - k0;
        return rc;
    }
    if (!sg.exec) {
        cudaGraph_t gr = nullptr;
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        const long long k0 = ctx->stats.kernel_launches;
        const int rc = body();
        ctx->stats.kernel_launches = k0;
        const cudaError_t e = cudaStreamEndCapture(ctx->stream, &gr);
        if (rc || e != cudaSuccess || !gr) {
            if (gr) cudaGraphDestroy(gr);
            cudaGetLastError();
            return rc ? rc : set_err(ctx, PIMD_ECUDA, "CUDA graph capture of an SCF iteration failed");
        }
        const cudaError_t ei = cudaGraphInstantiate(&sg.exec, gr, 0);
        cudaGraphDestroy(gr);
        if (ei != cudaSuccess) {
            sg.exec = nullptr;
            cudaGetLastError();
            return set_err(ctx, PIMD_ECUDA, "CUDA graph instantiation failed");
        }
    }
    CK(cudaGraphLaunch(sg.exec, ctx->stream));
    ctx->stats.kernel_launches += sg.launches;
    return PIMD_OK;
}

// block-diagonal D of the cached atomic densities for the replicas in mask
// (tr(D S) = electrons exactly), into dst; m.dD serves as scratch
static int sad_place(pimd_ctx* ctx, const pimd_basis* basis, const Batch& bt, Mats& m, const int* Zc,
                     const std::vector<int>& mask, double* dst)
{
    std::vector<double> tab;
    std::map<int, int> toff;
    std::vector<int> desc;
    for (int r = 0; r < bt.nrep; r++) {
        if (!mask[r]) continue;
        for (int a = bt.atom0[r]; a < bt.atom0[r + 1]; a++) {
            const auto& Da = ctx->sad.at({basis->uid, Zc[a]});
            if (!toff.count(Zc[a])) {
                toff[Zc[a]] = (int)tab.size();
                tab.insert(tab.end(), Da.begin(), Da.end());
            }
            const int na = (int)lround(sqrt((double)Da.size()));
            desc.insert(desc.end(), {r, bt.atom_f0[a], na, toff[Zc[a]]});
        }
    }
    double* d_tab;
    int *d_desc, *d_ms;
    UPLOAD("sad_tab", tab, d_tab);
    UPLOAD("sad_desc", desc, d_desc);
    UPLOAD("mask_sad", mask, d_ms);
    CK(cudaMemsetAsync(m.dD, 0, sizeof(double) * bt.mtot, ctx->stream));
    launch_place_blocks(m.rm, d_desc, (int)desc.size() / 4, d_tab, m.dD, ctx->stream);
    launch_copy_mats(m.rm, bt.nrep, m.dD, dst, d_ms, ctx->stream);
    return PIMD_OK;
}

static int run_batch(pimd_ctx* ctx, int nrep, const int* natom_of, const int* Zc, const double* d_xyz,
                     const pimd_basis* basis, const pimd_scf_opts* o, double* d_E, double* d_grad, pimd_info* info)
{
    Batch bt;
    ctx->stats = pimd_stats{};
    CK(cudaEventRecord(ctx->ev[0], ctx->stream));
    const bool want_sad = o->guess == 4 || o->guess == 5;
    int rc = PIMD_OK;
    if (want_sad) {
        int natot = 0;
        for (int r = 0; r < nrep; r++) natot += natom_of[r];
        if ((rc = sad_ensure(ctx, basis, Zc, natot))) return rc;
    }
    const bool split = o->split_size > 1;
    rc = setup_batch(ctx, bt, nrep, natom_of, Zc, d_xyz, basis, o->schwarz_tau, split ? o->split_size : 1,
                     split ? o->split_rank : 0);
    if (rc) return rc;
    const int hist = std::max(2, std::min(16, o->diis_size));
    Mats m;
    if ((rc = alloc_mats(ctx, bt, m, hist))) return rc;
    ScfPlan plan;
    if ((rc = make_plan(ctx, bt, m, plan))) return rc;
    std::vector<int> active(nrep, 1), fin(nrep, 0), slot(nrep, hist - 1), count(nrep, 0), diis_on(nrep, 0);
    UPLOAD("active", active, m.active);
    bt.R.active = m.active;
    // one-electron part
    launch_one_electron(bt.P, bt.S, bt.B, bt.At, bt.R, m.S, m.T, m.V, ctx->boys, ctx->stream);
    {
        add_mats(m.rm, nrep, m.T, m.V, m.H, ctx->stream);
    }
    CK(cudaMemsetAsync(m.enn, 0, sizeof(double) * nrep, ctx->stream));
    // deterministic mode: fixed-point accumulation of G', V_nn and the gradient
    const double fx_g = o->deterministic ? kFixG : 0.0, fx_grad = o->deterministic ? kFixGrad : 0.0;
    {
        std::vector<int> atom_rep;
        for (int r = 0; r < nrep; r++)
            for (int i = 0; i < bt.natom[r]; i++) atom_rep.push_back(r);
        int* d_ar;
        UPLOAD("atom_rep2", atom_rep, d_ar);
        launch_vnn(bt.At, bt.atom0[nrep], d_ar, m.enn, nullptr, ctx->stream, fx_grad);
        if (fx_grad > 0) launch_fixed_to_double(m.enn, nrep, fx_grad, ctx->stream);
    }
    // X = S^{-1/2}
    launch_jacobi(m.rm, nrep, m.S, m.Cp, m.Ev, m.ldE, m.work, nullptr, 0, ctx->stream, m.jnc);
    ctx->stats.kernel_launches += 5;
    {
        std::vector<double> ev((size_t)nrep * m.ldE);
        CK(cudaMemcpyAsync(ev.data(), m.Ev, sizeof(double) * ev.size(), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        for (int r = 0; r < nrep; r++)
            if (bt.nbf[r] > 0 && ev[(size_t)r * m.ldE] < 1e-8)
                return set_err(ctx, PIMD_EBASIS, "overlap matrix numerically singular");
    }
    launch_orth_from_eig(m.rm, nrep, m.Cp, m.Ev, m.ldE, m.X, ctx->stream);
    // guess per replica: cached MOs of the same replica index (guess 1, 3),
    // else the learned density (guess 2, 3), else the core Hamiltonian
    const bool want_cache = o->guess == 1 || o->guess == 3 || o->guess == 5;
    const bool want_learned = o->guess == 2 || o->guess == 3;
    if (want_learned && !ctx->guess_model) return set_err(ctx, PIMD_EINVAL, "learned guess without a model");
    if ((int)ctx->mo.size() < nrep) ctx->mo.resize(nrep);
    std::vector<int> use_cache(nrep, 0), core(nrep, 0), learned(nrep, 0), sadm(nrep, 0);
    int nlearned = 0, nsad = 0;
    for (int r = 0; r < nrep; r++) {
        auto& mo = ctx->mo[r];
        std::vector<int> z(Zc + bt.atom0[r], Zc + bt.atom0[r + 1]);
        use_cache[r] = (want_cache && mo.N == bt.nbf[r] && mo.Z == z);
        learned[r] = !use_cache[r] && want_learned;
        sadm[r] = !use_cache[r] && want_sad;
        core[r] = !use_cache[r] && !learned[r] && !sadm[r];
        nlearned += learned[r];
        nsad += sadm[r];
        if (use_cache[r]) {
            // the cached MOs, or for reuse_mode 2 the cached Fock matrix (stored with them)
            const DevBuf& src = o->reuse_mode == 2 ? mo.F : mo.C;
            CK(cudaMemcpyAsync((o->reuse_mode == 2 ? m.Fb : m.C) + bt.moff[r], src.p,
                               sizeof(double) * bt.nbf[r] * bt.nbf[r], cudaMemcpyDeviceToDevice, ctx->stream));
        }
    }
    int* d_mask;
    UPLOAD("mask_core", core, d_mask);
    int* d_mc;
    UPLOAD("mask_cache", use_cache, d_mc);
    // starting eigenvector basis Q of the warm-started diagonalisation: the
    // identity (the cached MOs are orthonormal for the previous geometry only,
    // so they seed the density, not Q; Q stays orthogonal because it is only
    // ever multiplied by Jacobi rotations)
    launch_identity(m.rm, nrep, m.Cq, nullptr, ctx->stream);
    launch_copy_mats(m.rm, nrep, m.H, m.Fb, d_mask, ctx->stream);
    if (o->reuse_mode == 2) {
        // core-Hamiltonian replicas and reused Fock matrices: one diagonalisation
        std::vector<int> both(nrep);
        for (int r = 0; r < nrep; r++) both[r] = core[r] || use_cache[r];
        int* d_both;
        UPLOAD("mask_diag0", both, d_both);
        diag_density(ctx, bt, m, plan, d_both);
    } else {
        diag_density(ctx, bt, m, plan, d_mask);
        gemm(ctx, plan.Dn, d_mc);
        if (o->reuse_mode == 1)
            for (int step = 0; step < 2; step++) {
                gemm(ctx, plan.DS, d_mc);
                gemm(ctx, plan.DSD, d_mc);
                gemm(ctx, plan.DSDS, d_mc);
                gemm(ctx, plan.Pur, d_mc);
                launch_copy_mats(m.rm, nrep, m.M2, m.D, d_mc, ctx->stream);
                ctx->stats.kernel_launches++;
            }
    }
    if (nlearned > 0) {
        pimd_guess* gm = ctx->guess_model;
        if (guess_device(gm) != ctx->device) return set_err(ctx, PIMD_EINVAL, "guess model on another device");
        for (int a = 0; a < bt.atom0[nrep]; a++) {
            const int e = basis->elem.at(Zc[a]);
            if (guess_elem_nbf(gm, Zc[a]) != basis->nbf_elem[e])
                return set_err(ctx, PIMD_EINVAL, "guess model built for another basis or element set");
        }
        int* d_ml;
        UPLOAD("mask_learned", learned, d_ml);
        // m.dD is scratch until the first incremental-build step overwrites it
        rc = guess_predict_device(gm, nrep, natom_of, Zc, bt.atom_f0, learned, d_xyz, bt.d_Zi, bt.At.rep_atom0,
                                  m.rm, d_ml, m.S, m.dD, bt.mtot, m.D, ctx->stream);
        if (rc) return set_err(ctx, rc, "learned guess failed");
        ctx->stats.kernel_launches += 19;
    }
    if (nsad > 0) {
        if ((rc = sad_place(ctx, basis, bt, m, Zc, sadm, m.D))) return rc;
        ctx->stats.kernel_launches += 2;
    }
    // SCF iterations
    std::vector<double> E(nrep), emax(nrep), Eprev(nrep, 0.0);
    std::vector<int> iters(nrep, 0), conv(nrep, 0);
    std::vector<double> fdE(nrep, 0.0), ferr(nrep, 0.0);
    // build mode per replica: 2 full Fock build, 1 incremental (G' += G'(D - D_prev))
    std::vector<int> mode(nrep, 2), since_full(nrep, 0);
    const int full_every = o->full_every > 0 ? o->full_every : 8;
    ctx->trace.assign(nrep, {});
    ctx->fock_ms_it.clear();
    ctx->fock_q_it.clear();
    // executed quartets of the Fock builds so far (counters [4 * 64]: quartets, primitive quartets, FP64 then FP32)
    std::vector<unsigned long long> cnt_it(4 * 64);
    long long fock_q_tot = 0;
    int nactive = nrep;
    const bool graphs = o->use_graphs != 0;
    GraphSeg seg_fock, seg_err, seg_diag;
    if (o->fp32_tau > o->schwarz_tau) {
        float* Mf;
        ENSURE("Mf", bt.mtot, Mf);   // allocated before any capture
    }
    double* Gsum = nullptr;   // force-split mode: G' summed over the processes
    if (split) ENSURE("Gsum", bt.mtot, Gsum);
    int *d_mode, *d_slot, *d_count, *d_on;
    ENSURE("mode", nrep, d_mode);
    ENSURE("slot", nrep, d_slot);
    ENSURE("count", nrep, d_count);
    ENSURE("diis_on", nrep, d_on);
    for (int it = 1; it <= o->max_iter && nactive > 0; it++) {
        for (int r = 0; r < nrep; r++) mode[r] = active[r] ? mode[r] : 0;
        UPLOAD("mode", mode, d_mode);
        CK(cudaEventRecord(ctx->ev[2], ctx->stream));
        rc = run_seg(ctx, seg_fock, graphs, [&]() -> int {
            launch_delta_density(m.rm, nrep, m.D, m.Dp, m.dD, m.G, d_mode, ctx->stream);
            ctx->stats.kernel_launches++;
            return fock_build(ctx, bt, m, o->schwarz_tau, o->fp32_tau, m.dD, o->schwarz_tau * o->prim_screen,
                              fx_g);
        });
        if (rc) return rc;
        CK(cudaEventRecord(ctx->ev[3], ctx->stream));
        ctx->stats.fock_builds++;
        if (split) {
            // this process's share of G' plus the others': the caller's sum
            // over the split_size processes (host callback between launches)
            CK(cudaMemcpyAsync(Gsum, m.G, sizeof(double) * bt.mtot, cudaMemcpyDeviceToDevice, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            if (o->reduce_fn(Gsum, bt.mtot, o->reduce_user) != 0)
                return set_err(ctx, PIMD_ECUDA, "force-split reduction of the Fock matrix failed");
        }
        rc = run_seg(ctx, seg_err, graphs, [&]() -> int {
            launch_fock_assemble(m.rm, nrep, m.H, split ? Gsum : m.G, m.F, m.active, ctx->stream);
            launch_energy(m.rm, nrep, m.D, m.H, m.F, m.enn, m.E, m.active, ctx->stream);
            gemm(ctx, plan.FD, m.active);
            gemm(ctx, plan.FDS, m.active);
            launch_antisym(m.rm, nrep, m.M2, m.Er, m.active, ctx->stream);
            gemm(ctx, plan.XtE, m.active);
            gemm(ctx, plan.XtEX, m.active);   // error -> M2
            launch_maxabs(m.rm, nrep, m.M2, m.emax, m.active, ctx->stream);
            ctx->stats.kernel_launches += 4;
            return PIMD_OK;
        });
        if (rc) return rc;
        CK(cudaMemcpyAsync(E.data(), m.E, sizeof(double) * nrep, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(emax.data(), m.emax, sizeof(double) * nrep, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(cnt_it.data(), bt.cnt, sizeof(unsigned long long) * cnt_it.size(), cudaMemcpyDeviceToHost,
                           ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        CK(cudaGetLastError());
        {
            long long tot = 0;
            for (size_t k = 0; k < cnt_it.size(); k += 2) tot += (long long)cnt_it[k];
            ctx->fock_q_it.push_back(tot - fock_q_tot);
            fock_q_tot = tot;
        }
        {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]);
            ctx->stats.ms_fock += ms;
            ctx->fock_ms_it.push_back(ms);
        }
        bool anyfin = false;
        for (int r = 0; r < nrep; r++) {
            fin[r] = 0;
            if (!active[r]) continue;
            if (!isfinite(E[r])) return set_err(ctx, PIMD_ECUDA, "non-finite SCF energy");
            iters[r] = it;
            fdE[r] = it > 1 ? fabs(E[r] - Eprev[r]) : INFINITY;
            ferr[r] = emax[r];
            ctx->trace[r].push_back({E[r], emax[r], mode[r] == 2 ? 1 : 0});
            const bool met = it > 1 && fdE[r] < o->conv_energy && emax[r] < o->conv_error;
            // convergence is only accepted on a full (non-incremental) build
            if (met && mode[r] == 2) {
                fin[r] = 1;
                conv[r] = 1;
                anyfin = true;
            } else if (it == o->max_iter) {
                fin[r] = 1;
                anyfin = true;
            }
            since_full[r] = mode[r] == 2 ? 1 : since_full[r] + 1;
            // once the commutator error is below its bar every build is a full
            // one: the energies of incremental builds carry the screening error
            // accumulated since the last full build (for 768 functions and 7e8
            // quartets a few 1e-9 hartree), which would hide |dE| < 1e-10; two
            // consecutive full builds compare exact energies
            mode[r] = (met || emax[r] < o->conv_error || since_full[r] >= full_every) ? 2 : 1;
            Eprev[r] = E[r];
        }
        if (anyfin) {
            // finishing replicas: orbitals, D and W from F(D) itself
            UPLOAD("fin", fin, m.fin);
            launch_copy_mats(m.rm, nrep, m.F, m.Fb, m.fin, ctx->stream);
            diag_density(ctx, bt, m, plan, m.fin);
            launch_scale_cols(m.rm, nrep, m.C, m.Ev, m.ldE, m.Cs, m.fin, ctx->stream);
            gemm(ctx, plan.Wn, m.fin);
            ctx->stats.kernel_launches += 2;
            for (int r = 0; r < nrep; r++)
                if (fin[r]) {
                    active[r] = 0;
                    nactive--;
                }
            UPLOAD("active", active, m.active);
        }
        if (nactive == 0) break;
        // DIIS on the continuing replicas
        for (int r = 0; r < nrep; r++)
            if (active[r]) {
                slot[r] = (slot[r] + 1) % hist;
                count[r] = std::min(count[r] + 1, hist);
                diis_on[r] = count[r] >= 2;
            }
        UPLOAD("slot", slot, d_slot);
        UPLOAD("count", count, d_count);
        UPLOAD("diis_on", diis_on, d_on);
        rc = run_seg(ctx, seg_diag, graphs, [&]() -> int {
            launch_diis_store(m.rm, nrep, m.F, m.M2, m.Fh, m.Eh, d_slot, hist, m.stride, m.active, ctx->stream);
            launch_diis_dots(m.rm, nrep, m.Eh, d_slot, d_count, hist, m.stride, m.Bd, m.active, ctx->stream);
            launch_diis_solve(nrep, m.Bd, d_slot, d_count, hist, m.coef, m.active, ctx->stream);
            launch_diis_combine(m.rm, nrep, m.Fh, m.coef, hist, m.stride, m.F, m.Fb, d_on, m.active, ctx->stream);
            ctx->stats.kernel_launches += 4;
            diag_density(ctx, bt, m, plan, m.active);
            return PIMD_OK;
        });
        if (rc) return rc;
    }
    CK(cudaGetLastError());
    // energies
    CK(cudaMemcpyAsync(d_E, E.data(), sizeof(double) * nrep, cudaMemcpyHostToDevice, ctx->stream));
    // gradient
    if (o->want_gradient && d_grad) {
        const int natot = bt.atom0[nrep];
        CK(cudaMemsetAsync(d_grad, 0, sizeof(double) * natot * 3, ctx->stream));
        // force-split mode: the one-electron and nuclear parts on process 0 only
        // (the sum over the processes adds every part once)
        if (!split || o->split_rank == 0) {
            launch_grad_1e(bt.P, bt.S, bt.B, bt.At, bt.R, m.D, m.W, d_grad, ctx->boys, fx_grad, ctx->stream);
            int* d_ar = (int*)ctx->bufs["atom_rep2"].p;
            double* d_dummy;
            ENSURE("enn_dummy", nrep, d_dummy);
            launch_vnn(bt.At, natot, d_ar, d_dummy, d_grad, ctx->stream, fx_grad);
        }
        CK(cudaEventRecord(ctx->ev[4], ctx->stream));
        launch_shell_bounds(bt.S, bt.R, nrep, bt.maxsh, m.D, bt.Dsh, nullptr, ctx->stream);
        const int rcg = fan_out_class_pairs(ctx, bt, [&](int cp, cudaStream_t st) {
            launch_grad2e(cp, bt.P, bt.S, bt.R, bt.d_tiles[cp], (int)bt.tiles[cp].size(), m.D, d_grad, ctx->boys,
                          ctx->boysf, o->schwarz_tau * 1e-2, o->fp32_tau, bt.Dsh, bt.cnt + 4 * 64 + 4 * cp,
                          ctx->grad_var[cp],
                          ctx->tile_w[cp] > 0 ? ctx->tile_w[cp] : 128, o->schwarz_tau * o->prim_screen,
                          fx_grad, st);
            ctx->stats.kernel_launches += o->fp32_tau > 0 ? 2 : 1;
        });
        if (rcg) return rcg;
        CK(cudaEventRecord(ctx->ev[5], ctx->stream));
        if (fx_grad > 0) launch_fixed_to_double(d_grad, natot * 3, fx_grad, ctx->stream);
        ctx->stats.kernel_launches += fx_grad > 0 ? 4 : 3;
        if (split) {
            CK(cudaStreamSynchronize(ctx->stream));
            if (o->reduce_fn(d_grad, (long long)natot * 3, o->reduce_user) != 0)
                return set_err(ctx, PIMD_ECUDA, "force-split reduction of the gradient failed");
        }
    }
    // MO cache (and the final Fock matrix)
    for (int r = 0; r < nrep; r++) {
        auto& mo = ctx->mo[r];
        const size_t bytes = sizeof(double) * bt.nbf[r] * bt.nbf[r];
        for (DevBuf* b : {&mo.C, &mo.F}) {
            if (b->cap >= bytes) continue;
            if (b->p) cudaFree(b->p);
            b->p = nullptr;
            b->cap = 0;
            if (cudaMalloc(&b->p, bytes) != cudaSuccess) {
                cudaGetLastError();
                mo.N = 0;
                return set_err(ctx, PIMD_ENOMEM, "MO cache allocation failed");
            }
            b->cap = bytes;
        }
        CK(cudaMemcpyAsync(mo.C.p, m.C + bt.moff[r], bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaMemcpyAsync(mo.F.p, m.F + bt.moff[r], bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        mo.Z.assign(Zc + bt.atom0[r], Zc + bt.atom0[r + 1]);
        mo.N = bt.nbf[r];
    }
    CK(cudaEventRecord(ctx->ev[1], ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaGetLastError());
    {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
        ctx->stats.ms_total = ms;
        if (o->want_gradient && d_grad) {
            cudaEventElapsedTime(&ms, ctx->ev[4], ctx->ev[5]);
            ctx->stats.ms_grad2e = ms;
        }
    }
    ctx->stats.nquartets_total = bt.nquart;
    {
        // executed work of all Fock builds of the call, from the device counters
        std::vector<unsigned long long> cnt(8 * 64);
        CK(cudaMemcpy(cnt.data(), bt.cnt, sizeof(unsigned long long) * cnt.size(), cudaMemcpyDeviceToHost));
        double fl = 0.0, er = 0.0, fl32 = 0.0, er32 = 0.0, gfl = 0.0, gfl32 = 0.0;
        long long q64 = 0, q32 = 0, gq = 0;
        for (int cp = 0; cp < n_class_pairs(); cp++) {
            int la, lb, lc, ld;
            class_pair_ls(cp, &la, &lb, &lc, &ld);
            const double nfun = (double)nsph(la) * nsph(lb) * nsph(lc) * nsph(ld);
            fl += (double)cnt[4 * cp + 1] * class_vrr_flops(cp);
            fl32 += (double)cnt[4 * cp + 3] * class_vrr_flops(cp);
            er += (double)(cnt[4 * cp] + cnt[4 * cp + 2]) * nfun;
            er32 += (double)cnt[4 * cp + 2] * nfun;
            q64 += (long long)cnt[4 * cp];
            q32 += (long long)cnt[4 * cp + 2];
            const unsigned long long* gc = cnt.data() + 4 * 64 + 4 * cp;
            gfl += (double)gc[1] * class_grad_flops(cp);
            gfl32 += (double)gc[3] * class_grad_flops(cp);
            gq += (long long)(gc[0] + gc[2]);
        }
        ctx->stats.grad_flops = gfl;
        ctx->stats.grad_flops32 = gfl32;
        ctx->stats.grad_quartets = gq;
        const int nb = std::max(1, ctx->stats.fock_builds);
        ctx->stats.eri_flops_per_build = fl / nb;
        ctx->stats.eri_flops32_per_build = fl32 / nb;
        ctx->stats.eris_per_build = er / nb;
        ctx->stats.eris32_per_build = er32 / nb;
        ctx->stats.quartets_fp64 = q64;
        ctx->stats.quartets_fp32 = q32;
    }
    std::vector<int> jnc(nrep);
    CK(cudaMemcpy(jnc.data(), m.jnc, sizeof(int) * nrep, cudaMemcpyDeviceToHost));
    std::vector<unsigned long long> qrep(2 * (size_t)nrep);
    CK(cudaMemcpy(qrep.data(), bt.R.qrep, sizeof(unsigned long long) * qrep.size(), cudaMemcpyDeviceToHost));
    bool allconv = true;
    for (int r = 0; r < nrep; r++) {
        if (jnc[r]) conv[r] = 0;   // a diagonalisation of the replica did not converge
        if (info) {
            info[r].iterations = iters[r];
            info[r].converged = conv[r];
            info[r].final_dE = fdE[r];
            info[r].final_error = ferr[r];
            info[r].nquartets = bt.nquart_rep[r];
            info[r].nq_fp64 = (long long)qrep[2 * r];
            info[r].nq_fp32 = (long long)qrep[2 * r + 1];
        }
        allconv = allconv && conv[r];
    }
    return allconv ? PIMD_OK : PIMD_ENOTCONV;
}

static int check_common(pimd_ctx* ctx, const pimd_basis* basis, const pimd_scf_opts* opts, pimd_scf_opts& o)
{
    if (!ctx || !basis) return PIMD_EINVAL;
    pimd_scf_opts_default(&o);
    if (opts) {
        if (opts->struct_size < sizeof(size_t) || opts->struct_size > sizeof(pimd_scf_opts)) return PIMD_EINVAL;
        memcpy(&o, opts, opts->struct_size);
    }
    if (!(o.conv_energy > 0) || !(o.conv_error > 0) || o.max_iter < 1 || o.max_iter > 10000 ||
        !(o.schwarz_tau >= 0) || o.guess < 0 || o.guess > 5 || o.full_every < 0 || !(o.prim_screen >= 0) ||
        o.prim_screen > 1.0 || o.reuse_mode < 0 || o.reuse_mode > 2 || o.diis_size > 16 || o.split_size < 0 ||
        (o.split_size > 1 && (o.split_rank < 0 || o.split_rank >= o.split_size || !o.reduce_fn)))
        return set_err(ctx, PIMD_EINVAL, "bad SCF options");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return PIMD_ECUDA;
    return PIMD_OK;
}

static int forces_impl(pimd_ctx* ctx, int nrep, const int* natom_of, const int* Zc, const double* coords,
                       bool coords_dev, const pimd_basis* basis, const pimd_scf_opts* opts, double* E,
                       double* grad, bool out_dev, pimd_info* info, cudaStream_t user_stream)
{
    pimd_scf_opts o;
    int rc = check_common(ctx, basis, opts, o);
    if (rc) return rc;
    if (nrep <= 0 || !natom_of || !Zc || !coords || !E) return set_err(ctx, PIMD_EINVAL, "bad sizes or pointers");
    if (o.want_gradient && !grad) return set_err(ctx, PIMD_EINVAL, "gradients == NULL with want_gradient");
    long long natot = 0;
    for (int r = 0; r < nrep; r++) {
        if (natom_of[r] <= 0 || natom_of[r] > 100000) return set_err(ctx, PIMD_EINVAL, "bad atom count");
        natot += natom_of[r];
    }
    if (user_stream) CK(cudaStreamSynchronize(user_stream));
    double* d_xyz;
    ENSURE("xyz", natot * 3, d_xyz);
    if (coords_dev) {
        CK(cudaMemcpyAsync(d_xyz, coords, sizeof(double) * natot * 3, cudaMemcpyDeviceToDevice, ctx->stream));
    } else {
        for (long long i = 0; i < natot * 3; i++)
            if (!isfinite(coords[i])) return set_err(ctx, PIMD_EINVAL, "non-finite coordinates");
        CK(cudaMemcpyAsync(d_xyz, coords, sizeof(double) * natot * 3, cudaMemcpyHostToDevice, ctx->stream));
    }
    double *d_E, *d_g = nullptr;
    ENSURE("out_E", nrep, d_E);
    if (o.want_gradient) ENSURE("out_g", natot * 3, d_g);
    rc = run_batch(ctx, nrep, natom_of, Zc, d_xyz, basis, &o, d_E, d_g, info);
    if (rc && rc != PIMD_ENOTCONV) return rc;
    const cudaMemcpyKind k = out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(E, d_E, sizeof(double) * nrep, k, ctx->stream));
    if (o.want_gradient) CK(cudaMemcpyAsync(grad, d_g, sizeof(double) * natot * 3, k, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return rc;
}

extern "C" int pimd_guess_add_data(pimd_guess* g, pimd_ctx* ctx, int nrep, int natom, const int* Z,
                                   const double* coords, const pimd_basis* basis, const pimd_scf_opts* opts,
                                   pimd_info* info)
{
    if (!g || !ctx || !basis || nrep <= 0 || natom <= 0 || !Z || !coords) return PIMD_EINVAL;
    if (guess_device(g) != ctx->device) return set_err(ctx, PIMD_EINVAL, "guess model on another device");
    std::vector<int> atom_f0;
    for (int r = 0; r < nrep; r++) {
        int f = 0;
        for (int i = 0; i < natom; i++) {
            auto it = basis->elem.find(Z[i]);
            if (it == basis->elem.end()) return set_err(ctx, PIMD_EINVAL, "element missing from basis");
            if (guess_elem_nbf(g, Z[i]) != basis->nbf_elem[it->second])
                return set_err(ctx, PIMD_EINVAL, "guess model built for another basis or element set");
            atom_f0.push_back(f);
            f += basis->nbf_elem[it->second];
        }
    }
    pimd_scf_opts o;
    pimd_scf_opts_default(&o);
    if (opts) {
        if (opts->struct_size < sizeof(size_t) || opts->struct_size > sizeof(pimd_scf_opts)) return PIMD_EINVAL;
        memcpy(&o, opts, opts->struct_size);
        o.struct_size = sizeof(pimd_scf_opts);
    }
    o.want_gradient = 0;
    std::vector<int> natom_of(nrep, natom), Zc;
    for (int r = 0; r < nrep; r++) Zc.insert(Zc.end(), Z, Z + natom);
    std::vector<double> E(nrep);
    int rc = forces_impl(ctx, nrep, natom_of.data(), Zc.data(), coords, false, basis, &o, E.data(), nullptr, false,
                         info, nullptr);
    if (rc) return rc;   // unconverged densities are not training data
    // the call's device state: coordinates, charges, replica layout, converged D
    return guess_collect_device(g, nrep, natom_of.data(), Zc.data(), atom_f0, (const double*)ctx->bufs["xyz"].p,
                                (const int*)ctx->bufs["Zi"].p, (const int*)ctx->bufs["atom0"].p,
                                (const RepMat*)ctx->bufs["rm"].p, (double*)ctx->bufs["D"].p, ctx->stream);
}

extern "C" int pimd_bo_forces(pimd_ctx* ctx, int nrep, int natom, const int* Z, const double* coords,
                              const pimd_basis* basis, const pimd_scf_opts* opts, double* energies,
                              double* gradients, pimd_info* info)
{
    if (nrep <= 0 || natom <= 0 || !Z) return PIMD_EINVAL;
    std::vector<int> nat(nrep, natom), Zc((size_t)nrep * natom);
    for (int r = 0; r < nrep; r++) std::copy(Z, Z + natom, Zc.begin() + (size_t)r * natom);
    return forces_impl(ctx, nrep, nat.data(), Zc.data(), coords, false, basis, opts, energies, gradients, false, info,
                       nullptr);
}

extern "C" int string_images_forces(pimd_ctx* ctx, int nimg, const int* natom_of_img, const int* Z_concat,
                                    const double* coords_concat, const pimd_basis* basis, const pimd_scf_opts* opts,
                                    double* energies, double* gradients_concat, pimd_info* info)
{
    return forces_impl(ctx, nimg, natom_of_img, Z_concat, coords_concat, false, basis, opts, energies,
                       gradients_concat, false, info, nullptr);
}

extern "C" int pimd_screened_quartets(pimd_ctx* ctx, int nrep, const int* natom_of, const int* Zc,
                                      const double* coords, const pimd_basis* basis, double schwarz_tau,
                                      long long* counts)
{
    if (!ctx || !basis || nrep <= 0 || !natom_of || !Zc || !coords || !counts || !(schwarz_tau >= 0))
        return PIMD_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return PIMD_ECUDA;
    long long natot = 0;
    for (int r = 0; r < nrep; r++) {
        if (natom_of[r] <= 0 || natom_of[r] > 100000) return set_err(ctx, PIMD_EINVAL, "bad atom count");
        natot += natom_of[r];
    }
    for (long long i = 0; i < natot * 3; i++)
        if (!isfinite(coords[i])) return set_err(ctx, PIMD_EINVAL, "non-finite coordinates");
    double* d_xyz;
    ENSURE("xyz", natot * 3, d_xyz);
    CK(cudaMemcpyAsync(d_xyz, coords, sizeof(double) * natot * 3, cudaMemcpyHostToDevice, ctx->stream));
    Batch bt;
    bt.allow_odd = true;
    const int rc = setup_batch(ctx, bt, nrep, natom_of, Zc, d_xyz, basis, schwarz_tau);
    if (rc) return rc;
    for (int r = 0; r < nrep; r++) counts[r] = bt.nquart_rep[r];
    return PIMD_OK;
}

extern "C" int pimd_bo_forces_dev(pimd_ctx* ctx, int nrep, int natom, const int* Z, const double* coords_dev,
                                  const pimd_basis* basis, const pimd_scf_opts* opts, double* energies_dev,
                                  double* gradients_dev, pimd_info* info, void* stream)
{
    if (nrep <= 0 || natom <= 0 || !Z) return PIMD_EINVAL;
    std::vector<int> nat(nrep, natom), Zc((size_t)nrep * natom);
    for (int r = 0; r < nrep; r++) std::copy(Z, Z + natom, Zc.begin() + (size_t)r * natom);
    return forces_impl(ctx, nrep, nat.data(), Zc.data(), coords_dev, true, basis, opts, energies_dev, gradients_dev,
                       true, info, (cudaStream_t)stream);
}

extern "C" int string_images_forces_dev(pimd_ctx* ctx, int nimg, const int* natom_of_img, const int* Z_concat,
                                        const double* coords_concat_dev, const pimd_basis* basis,
                                        const pimd_scf_opts* opts, double* energies_dev, double* gradients_concat_dev,
                                        pimd_info* info, void* stream)
{
    return forces_impl(ctx, nimg, natom_of_img, Z_concat, coords_concat_dev, true, basis, opts, energies_dev,
                       gradients_concat_dev, true, info, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// testing hooks
// ---------------------------------------------------------------------------
// Autotuner: per class pair, the Fock-build kernel (straight-line with ket
// tiles of 32, 64 or 128 quartets per block, or the cooperative tape
// kernel, where generated) and then the gradient kernel (straight-line or
// cooperative, where both exist) that run this workload fastest. Each
// candidate is timed with CUDA events around the class pair's launches, the
// second of two passes, on the SAD density of the given replicas with the
// options' thresholds.
extern "C" int pimd_autotune(pimd_ctx* ctx, int nrep, int natom, const int* Z, const double* coords,
                             const pimd_basis* basis, const pimd_scf_opts* opts, int* widths, double* ms_best)
{
    pimd_scf_opts o;
    int rc = check_common(ctx, basis, opts, o);
    if (rc) return rc;
    if (nrep <= 0 || natom <= 0 || !Z || !coords) return set_err(ctx, PIMD_EINVAL, "bad sizes or pointers");
    std::vector<int> nat(nrep, natom), Zc((size_t)nrep * natom);
    for (int r = 0; r < nrep; r++) std::copy(Z, Z + natom, Zc.begin() + (size_t)r * natom);
    for (long long i = 0; i < (long long)nrep * natom * 3; i++)
        if (!std::isfinite(coords[i])) return set_err(ctx, PIMD_EINVAL, "non-finite coordinates");
    if ((rc = sad_ensure(ctx, basis, Zc.data(), nrep * natom))) return rc;
    double* d_xyz;
    ENSURE("xyz", (size_t)nrep * natom * 3, d_xyz);
    CK(cudaMemcpyAsync(d_xyz, coords, sizeof(double) * nrep * natom * 3, cudaMemcpyHostToDevice, ctx->stream));
    const int ncp = n_class_pairs();
    const int cand[4] = {32, 64, 128, 0};
    const double inf = 1e300;
    std::vector<double> ms((size_t)ncp * 4, inf), gms((size_t)ncp * 2, inf);
    std::vector<cudaEvent_t> ev(2 * (size_t)ncp);
    for (auto& e : ev) CK(cudaEventCreate(&e));
    int rc2 = PIMD_OK;
    // one batch with the current widths; the density, bounds and (for the
    // gradient) the SAD density itself serve every candidate
    auto prepare = [&](Batch& bt, Mats& m, float** Mf) -> int {
        int r2 = setup_batch(ctx, bt, nrep, nat.data(), Zc.data(), d_xyz, basis, o.schwarz_tau);
        if (r2) return r2;
        if ((r2 = alloc_mats(ctx, bt, m, 2))) return r2;
        std::vector<int> active(nrep, 1);
        if ((r2 = upload(ctx, "active", active, &m.active))) return r2;
        bt.R.active = m.active;
        if ((r2 = sad_place(ctx, basis, bt, m, Zc.data(), active, m.D))) return r2;
        *Mf = nullptr;
        if (o.fp32_tau > o.schwarz_tau && (r2 = dev_ensure(ctx, "Mf", (size_t)bt.mtot, Mf))) return r2;
        return PIMD_OK;
    };
    auto timed = [&](std::vector<double>& out, int stride, int col, const std::vector<int>& use,
                     auto&& launch) -> int {
        for (int pass = 0; pass < 2; pass++) {
            for (int cp = 0; cp < ncp; cp++) {
                cudaEventRecord(ev[2 * cp], ctx->stream);
                if (use[cp]) launch(cp);
                cudaEventRecord(ev[2 * cp + 1], ctx->stream);
            }
            if (cudaStreamSynchronize(ctx->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
                return set_err(ctx, PIMD_ECUDA, "autotune: kernel failed");
            if (pass == 1)
                for (int cp = 0; cp < ncp; cp++)
                    if (use[cp]) {
                        float t = 0.f;
                        cudaEventElapsedTime(&t, ev[2 * cp], ev[2 * cp + 1]);
                        out[(size_t)cp * stride + col] = t;
                    }
        }
        return PIMD_OK;
    };
    // Fock build: every candidate width (or the cooperative kernel)
    for (int ci = 0; ci < 4 && !rc2; ci++) {
        std::vector<int> use(ncp, 0);
        for (int cp = 0; cp < ncp; cp++) {
            const bool ok = cand[ci] > 0 ? class_pair_straight(cp) : class_pair_coop(cp);
            use[cp] = ok;
            ctx->tile_w[cp] = ok ? cand[ci] : (class_pair_straight(cp) ? 128 : 0);
        }
        Batch bt;
        Mats m;
        float* Mf;
        if ((rc2 = prepare(bt, m, &Mf))) break;
        cudaMemsetAsync(m.G, 0, sizeof(double) * bt.mtot, ctx->stream);
        launch_shell_bounds(bt.S, bt.R, bt.nrep, bt.maxsh, m.D, bt.Dsh, bt.R.active, ctx->stream);
        if (Mf) launch_to_float(m.D, Mf, bt.mtot, ctx->stream);
        rc2 = timed(ms, 4, ci, use, [&](int cp) {
            if (!bt.tiles[cp].empty())
                launch_jk(cp, bt.P, bt.S, bt.R, bt.d_tiles[cp], (int)bt.tiles[cp].size(), m.D, Mf, m.G, ctx->boys,
                          ctx->boysf, o.schwarz_tau, o.fp32_tau, bt.Dsh, bt.cnt + 4 * cp, cand[ci],
                          o.schwarz_tau * o.prim_screen, 0.0, ctx->stream);
        });
    }
    double best = 0.0;
    for (int cp = 0; cp < ncp; cp++) {
        int bi = class_pair_straight(cp) ? 2 : 3;
        if (!rc2)
            for (int ci = 0; ci < 4; ci++)
                if (ms[(size_t)cp * 4 + ci] < ms[(size_t)cp * 4 + bi]) bi = ci;
        ctx->tile_w[cp] = cand[bi];
        if (ms[(size_t)cp * 4 + bi] < inf) best += ms[(size_t)cp * 4 + bi];
        if (widths) widths[cp] = cand[bi];
    }
    // gradient: both variants where both exist, on tiles of the chosen widths
    if (!rc2) {
        Batch bt;
        Mats m;
        float* Mf;
        rc2 = prepare(bt, m, &Mf);
        double* d_g = nullptr;
        if (!rc2) rc2 = dev_ensure(ctx, "tune_grad", (size_t)nrep * natom * 3, &d_g);
        if (!rc2) {
            launch_shell_bounds(bt.S, bt.R, nrep, bt.maxsh, m.D, bt.Dsh, nullptr, ctx->stream);
            for (int v = 0; v < 2 && !rc2; v++) {
                std::vector<int> use(ncp, 0);
                for (int cp = 0; cp < ncp; cp++)
                    use[cp] = (v == 0 ? grad_pair_coop(cp) : grad_pair_straight(cp)) && !bt.tiles[cp].empty();
                rc2 = timed(gms, 2, v, use, [&](int cp) {
                    launch_grad2e(cp, bt.P, bt.S, bt.R, bt.d_tiles[cp], (int)bt.tiles[cp].size(), m.D, d_g,
                                  ctx->boys, ctx->boysf, o.schwarz_tau * 1e-2, o.fp32_tau, bt.Dsh,
                                  bt.cnt + 4 * 64 + 4 * cp, v,
                                  ctx->tile_w[cp] > 0 ? ctx->tile_w[cp] : 128,
                                  o.schwarz_tau * o.prim_screen, 0.0, ctx->stream);
                });
            }
        }
        if (!rc2)
            for (int cp = 0; cp < ncp; cp++) {
                const double t0 = gms[(size_t)cp * 2], t1 = gms[(size_t)cp * 2 + 1];
                if (t0 < inf || t1 < inf) ctx->grad_var[cp] = t0 < t1 ? 0 : 1;
                if (widths) widths[32 + cp] = ctx->grad_var[cp];
            }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (ms_best) *ms_best = best;
    return rc2;
}

extern "C" int pimd_fock_dev(pimd_ctx* ctx, int nrep, int natom, const int* Z, const double* coords,
                             const pimd_basis* basis, double schwarz_tau, double fp32_tau, const double* D_dev,
                             double* G_dev)
{
    if (!ctx || !basis || nrep <= 0 || natom <= 0 || !Z || !coords || !D_dev || !G_dev) return PIMD_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return PIMD_ECUDA;
    std::vector<int> nat(nrep, natom), Zc((size_t)nrep * natom);
    for (int r = 0; r < nrep; r++) std::copy(Z, Z + natom, Zc.begin() + (size_t)r * natom);
    double* d_xyz;
    ENSURE("xyz", (size_t)nrep * natom * 3, d_xyz);
    CK(cudaMemcpyAsync(d_xyz, coords, sizeof(double) * nrep * natom * 3, cudaMemcpyHostToDevice, ctx->stream));
    Batch bt;
    int rc = setup_batch(ctx, bt, nrep, nat.data(), Zc.data(), d_xyz, basis, schwarz_tau);
    if (rc) return rc;
    Mats m;
    if ((rc = alloc_mats(ctx, bt, m, 2))) return rc;
    std::vector<int> active(nrep, 1);
    UPLOAD("active", active, m.active);
    bt.R.active = m.active;
    CK(cudaMemcpyAsync(m.D, D_dev, sizeof(double) * bt.mtot, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemsetAsync(m.G, 0, sizeof(double) * bt.mtot, ctx->stream));
    {
        pimd_scf_opts d;
        pimd_scf_opts_default(&d);
        if ((rc = fock_build(ctx, bt, m, schwarz_tau, fp32_tau, m.D, schwarz_tau * d.prim_screen, 0.0))) return rc;
    }
    // G_out = G' + G'^T
    CK(cudaMemsetAsync(m.H, 0, sizeof(double) * bt.mtot, ctx->stream));
    launch_fock_assemble(m.rm, nrep, m.H, m.G, m.F, nullptr, ctx->stream);
    CK(cudaMemcpyAsync(G_dev, m.F, sizeof(double) * bt.mtot, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaGetLastError());
    ctx->stats.nquartets_total = bt.nquart;
    ctx->stats.eri_flops_per_build = bt.vrr_flops;
    return PIMD_OK;
}

extern "C" int pimd_one_electron(pimd_ctx* ctx, int natom, const int* Z, const double* coords,
                                 const pimd_basis* basis, double* S, double* T, double* V)
{
    if (!ctx || !basis || natom <= 0 || !Z || !coords || !S || !T || !V) return PIMD_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return PIMD_ECUDA;
    double* d_xyz;
    ENSURE("xyz", (size_t)natom * 3, d_xyz);
    CK(cudaMemcpyAsync(d_xyz, coords, sizeof(double) * natom * 3, cudaMemcpyHostToDevice, ctx->stream));
    Batch bt;
    int nat = natom;
    int rc = setup_batch(ctx, bt, 1, &nat, Z, d_xyz, basis, 1e-12);
    if (rc) return rc;
    Mats m;
    if ((rc = alloc_mats(ctx, bt, m, 2))) return rc;
    launch_one_electron(bt.P, bt.S, bt.B, bt.At, bt.R, m.S, m.T, m.V, ctx->boys, ctx->stream);
    const size_t n = (size_t)bt.nbf[0] * bt.nbf[0];
    CK(cudaMemcpyAsync(S, m.S, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(T, m.T, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(V, m.V, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaGetLastError());
    return PIMD_OK;
}

extern "C" int pimd_boys_dev(pimd_ctx* ctx, int n, int mord, const double* T_dev, double* F_dev)
{
    if (!ctx || n < 0 || mord < 0 || mord > BOYS_MMAX || (n > 0 && (!T_dev || !F_dev))) return PIMD_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return PIMD_ECUDA;
    launch_boys_eval(n, mord, T_dev, F_dev, ctx->boys, ctx->stream);
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaGetLastError());
    return PIMD_OK;
}

extern "C" int pimd_boys_f32_dev(pimd_ctx* ctx, int n, int mord, const float* T_dev, float* F_dev, int variant)
{
    if (!ctx || n < 0 || mord < 0 || mord > BOYS_MMAX || (variant != 0 && variant != 1) ||
        (n > 0 && (!T_dev || !F_dev)))
        return PIMD_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return PIMD_ECUDA;
    launch_boys_eval_f32(n, mord, T_dev, F_dev, ctx->boysf, variant, ctx->stream);
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaGetLastError());
    return PIMD_OK;
}

extern "C" int pimd_eigh_dev(pimd_ctx* ctx, int nmat, int n, const double* A_dev, double* V_dev, double* evals_dev,
                             void* stream)
{
    if (!ctx || nmat <= 0 || n <= 0 || n > 768 || !A_dev || !V_dev || !evals_dev) return PIMD_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return PIMD_ECUDA;
    if (stream) CK(cudaStreamSynchronize((cudaStream_t)stream));
    std::vector<RepMat> rm(nmat);
    for (int r = 0; r < nmat; r++) rm[r] = RepMat{n, 0, (long long)r * n * n};
    RepMat* d_rm;
    double* work;
    int* nc;
    UPLOAD("eigh_rm", rm, d_rm);
    ENSURE("eigh_work", (size_t)nmat * n * n, work);
    ENSURE("eigh_nc", nmat, nc);
    CK(cudaMemsetAsync(nc, 0, sizeof(int) * nmat, ctx->stream));
    launch_jacobi(d_rm, nmat, A_dev, V_dev, evals_dev, n, work, nullptr, 1, ctx->stream, nc);
    CK(cudaGetLastError());
    std::vector<int> hnc(nmat);
    CK(cudaMemcpyAsync(hnc.data(), nc, sizeof(int) * nmat, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int r = 0; r < nmat; r++)
        if (hnc[r]) return set_err(ctx, PIMD_ENOTCONV, "eigensolver sweep limit reached");
    return PIMD_OK;
}
