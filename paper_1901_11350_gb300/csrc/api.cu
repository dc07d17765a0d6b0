// api.cu -- the C ABI declared in include/spirit_gb.h: contexts, the host-side
// neighbour-stencil builder and the dispatch of every call to its kernels.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "ctx.h"

namespace {

int fail(sp_ctx *c, int code, const char *fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

int cuda_fail(sp_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, SP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int ensure(sp_ctx *c, DevBuf &b, size_t bytes)
{
    if (b.bytes >= bytes && b.p) return SP_OK;
    if (b.p) {
        cudaError_t e = cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaFree");
    }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc of context scratch");
    b.bytes = bytes;
    return SP_OK;
}

size_t rec_bytes(const sp_ctx *c) { return c->prec == SP_F64 ? sizeof(dq4) : sizeof(float4); }

void bond(const sp_ctx *c, int b, int jb, const int d[3], double r[3])
{
    double x[3];
    for (int k = 0; k < 3; ++k) x[k] = d[k] + c->basis[jb][k] - c->basis[b][k];
    for (int l = 0; l < 3; ++l) r[l] = c->a * (x[0] * c->A[0][l] + x[1] * c->A[1][l] + x[2] * c->A[2][l]);
}

// Directed neighbour stencil: shells are the distinct bond lengths found in a
// box of cells around every basis atom; each unique pair appears once from
// each side (D_ji = -D_ij); zero entries are dropped.
int build_stencil(sp_ctx *c)
{
    const sp_hamiltonian &h = c->h;
    int n_sh = h.n_shells;
    int n_dm = h.dmi_kind == SP_DMI_NONE ? 0 : h.n_dmi_shells;
    int n_need = std::max(n_sh, n_dm);
    c->nbr.clear();
    if (n_need > 0) {
        int R[3];
        for (int k = 0; k < 3; ++k) R[k] = c->nc[k] > 1 ? n_need + 2 : 0;
        struct Cand {
            double len;
            int b, jb, d[3];
        };
        std::vector<Cand> cand;
        for (int b = 0; b < c->nb; ++b)
            for (int jb = 0; jb < c->nb; ++jb)
                for (int d0 = -R[0]; d0 <= R[0]; ++d0)
                    for (int d1 = -R[1]; d1 <= R[1]; ++d1)
                        for (int d2 = -R[2]; d2 <= R[2]; ++d2) {
                            int d[3] = {d0, d1, d2};
                            double r[3];
                            bond(c, b, jb, d, r);
                            double len = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
                            if (len < 1e-8 * c->a) continue;
                            cand.push_back({len, b, jb, {d0, d1, d2}});
                        }
        std::vector<double> lens;
        for (auto &x : cand) lens.push_back(x.len);
        std::sort(lens.begin(), lens.end());
        std::vector<double> shells;
        for (double l : lens)
            if ((int)shells.size() < n_need && (shells.empty() || l - shells.back() > 1e-8 * c->a)) shells.push_back(l);
        for (auto &x : cand) {
            int s = -1;
            for (int q = 0; q < (int)shells.size(); ++q)
                if (std::fabs(shells[q] - x.len) <= 1e-8 * c->a) s = q;
            if (s < 0) continue;
            HostNbr e{};
            e.b = x.b;
            e.jb = x.jb;
            for (int k = 0; k < 3; ++k) e.d[k] = x.d[k];
            e.J = s < n_sh ? h.J[s] : 0.0;
            if (s < n_dm) {
                double r[3];
                bond(c, x.b, x.jb, x.d, r);
                double u[3] = {r[0] / x.len, r[1] / x.len, r[2] / x.len};
                if (h.dmi_kind == SP_DMI_BULK) {
                    for (int k = 0; k < 3; ++k) e.D[k] = h.D[s] * u[k];
                } else {  // z x rhat
                    e.D[0] = -h.D[s] * u[1];
                    e.D[1] = h.D[s] * u[0];
                    e.D[2] = 0.0;
                }
            }
            if (e.J == 0.0 && e.D[0] == 0.0 && e.D[1] == 0.0 && e.D[2] == 0.0) continue;
            c->nbr.push_back(e);
        }
    }
    for (const sp_pair &p : c->pairs) {
        HostNbr e{}, r{};
        e.b = p.i;
        e.jb = p.j;
        r.b = p.j;
        r.jb = p.i;
        for (int k = 0; k < 3; ++k) {
            e.d[k] = p.d[k];
            r.d[k] = -p.d[k];
            e.D[k] = p.D[k];
            r.D[k] = -p.D[k];
        }
        e.J = r.J = p.J;
        c->nbr.push_back(e);
        c->nbr.push_back(r);
    }
    if ((int)c->nbr.size() > SP_MAX_NBR)
        return fail(c, SP_ERR_ARG, "%d directed neighbour entries exceed SP_MAX_NBR=%d", (int)c->nbr.size(), SP_MAX_NBR);
    for (auto &e : c->nbr)
        for (int k = 0; k < 3; ++k)
            if (c->per[k] && std::abs(e.d[k]) > c->nc[k])
                return fail(c, SP_ERR_UNSUPPORTED, "bond offset %d exceeds the periodic extent %d", e.d[k], c->nc[k]);
    std::stable_sort(c->nbr.begin(), c->nbr.end(), [](const HostNbr &x, const HostNbr &y) { return x.b < y.b; });
    return SP_OK;
}

template <typename T> void fill_stencil(const sp_ctx *c, Stencil<T> &S)
{
    memset(&S, 0, sizeof S);
    S.nb = c->nb;
    S.n0 = c->nc[0];
    S.n1 = c->nc[1];
    S.n2 = c->nc[2];
    S.per0 = c->per[0];
    S.per1 = c->per[1];
    S.per2 = c->per[2];
    S.N = c->N;
    S.fnb = make_fastdiv(c->nb);
    S.fn0 = make_fastdiv(c->nc[0]);
    S.fn1 = make_fastdiv(c->nc[1]);
    for (int b = 0; b < c->nb; ++b) {
        double mu = c->mu_s[b] * kMuB;
        S.mu[b] = (T)mu;
        for (int k = 0; k < 3; ++k) S.Bz[b][k] = (T)(mu * c->h.B[k]);
        S.K[b] = (T)c->h.K[b];
        double kh[3] = {c->h.Khat[b][0], c->h.Khat[b][1], c->h.Khat[b][2]};
        double r = std::sqrt(kh[0] * kh[0] + kh[1] * kh[1] + kh[2] * kh[2]);
        for (int k = 0; k < 3; ++k) S.Kh[b][k] = (T)(r > 0 ? kh[k] / r : 0.0);
    }
    int q = 0;
    for (int b = 0; b <= c->nb; ++b) {
        S.off[b] = q;
        if (b == c->nb) break;
        for (auto &e : c->nbr)
            if (e.b == b) {
                NbrEntry<T> &E = S.e[q++];
                E.jb = e.jb;
                E.d0 = e.d[0];
                E.d1 = e.d[1];
                E.d2 = e.d[2];
                E.J = (T)e.J;
                E.Dx = (T)e.D[0];
                E.Dy = (T)e.D[1];
                E.Dz = (T)e.D[2];
                // i = b + nb (c0 + n0 (c1 + n1 c2)), j the same with jb, c + d
                E.lin = (e.jb - b) + c->nb * (e.d[0] + c->nc[0] * (e.d[1] + c->nc[1] * e.d[2]));
                S.r0 = std::max(S.r0, std::abs(e.d[0]));
                S.r1 = std::max(S.r1, std::abs(e.d[1]));
                S.r2 = std::max(S.r2, std::abs(e.d[2]));
            }
    }
}

// The 27-point fast path applies to a one-atom lattice whose bonds stay in
// the 3x3x3 cell neighbourhood with one exchange constant per offset class
// (faces, edges, corners) and DMI on the faces only.  Offsets along an open
// direction of extent 1 never connect two spins and are ignored.
template <typename T> void fill_cubic(const sp_ctx *c, const double J[27], const double D[27][3], const double Jc[4],
                                      CubicParams<T> &P)
{
    memset(&P, 0, sizeof P);
    P.nx = c->nc[0];
    P.ny = c->nc[1];
    P.nz = c->nc[2];
    P.per0 = c->per[0];
    P.per1 = c->per[1];
    P.per2 = c->per[2];
    P.J1 = (T)Jc[1];
    P.J2 = (T)Jc[2];
    P.J3 = (T)Jc[3];
    for (int k = 0; k < 3; ++k) {
        P.Dx[k] = (T)D[2 + 3 * 1 + 9 * 1][k];
        P.Dy[k] = (T)D[1 + 3 * 2 + 9 * 1][k];
        P.Dz[k] = (T)D[1 + 3 * 1 + 9 * 2][k];
    }
    double mu = c->mu_s[0] * kMuB;
    double kh[3] = {c->h.Khat[0][0], c->h.Khat[0][1], c->h.Khat[0][2]};
    double r = std::sqrt(kh[0] * kh[0] + kh[1] * kh[1] + kh[2] * kh[2]);
    for (int k = 0; k < 3; ++k) {
        P.Bz[k] = (T)(mu * c->h.B[k]);
        P.Kh[k] = (T)(r > 0 ? kh[k] / r : 0.0);
    }
    P.K = (T)c->h.K[0];
    // DMI kind: none, bulk-like (face vector along its bond, one magnitude) or general
    bool none = true, bulk = true;
    double Dm = D[2 + 3 * 1 + 9 * 1][0];
    const int faces[3] = {2 + 3 * 1 + 9 * 1, 1 + 3 * 2 + 9 * 1, 1 + 3 * 1 + 9 * 2};
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) {
            double v = D[faces[a]][k];
            if (v != 0) none = false;
            double want = (k == a) ? Dm : 0.0;
            bool irrelevant = c->nc[a] == 1 && !c->per[a];
            if (!irrelevant && v != want) bulk = false;
        }
    P.dmi_mode = none ? 0 : (bulk ? 1 : 2);
}

void detect_cubic(sp_ctx *c)
{
    c->cubic = false;
    if (c->nb != 1) return;
    double J[27] = {0}, D[27][3] = {{0}};
    for (auto &e : c->nbr) {
        if (std::abs(e.d[0]) > 1 || std::abs(e.d[1]) > 1 || std::abs(e.d[2]) > 1) return;
        int o = (e.d[0] + 1) + 3 * (e.d[1] + 1) + 9 * (e.d[2] + 1);
        J[o] += e.J;
        for (int k = 0; k < 3; ++k) D[o][k] += e.D[k];
    }
    double Jc[4] = {0, 0, 0, 0};
    bool seen[4] = {false, false, false, false};
    for (int o = 0; o < 27; ++o) {
        int d[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
        int cls = (d[0] != 0) + (d[1] != 0) + (d[2] != 0);
        bool relevant = true;
        for (int k = 0; k < 3; ++k)
            if (d[k] != 0 && c->nc[k] == 1 && !c->per[k]) relevant = false;
        if (!relevant) continue;
        if (cls == 0) {
            if (J[o] != 0 || D[o][0] != 0 || D[o][1] != 0 || D[o][2] != 0) return;
            continue;
        }
        if (seen[cls] && J[o] != Jc[cls]) return;
        seen[cls] = true;
        Jc[cls] = J[o];
        if (cls != 1 && (D[o][0] != 0 || D[o][1] != 0 || D[o][2] != 0)) return;
        if (cls == 1) {
            int m = 26 - o;  // opposite face
            for (int k = 0; k < 3; ++k)
                if (D[m][k] != -D[o][k]) return;
        }
    }
    // drop DMI of irrelevant faces
    for (int k = 0; k < 3; ++k) {
        int o = 1 + 3 * 1 + 9 * 1 + (k == 0 ? 1 : k == 1 ? 3 : 9);
        if (c->nc[k] == 1 && !c->per[k]) D[o][0] = D[o][1] = D[o][2] = 0;
    }
    fill_cubic(c, J, D, Jc, c->Cf);
    fill_cubic(c, J, D, Jc, c->Cd);
    c->zc_auto = 0;  // recomputed for the new lattice on first use
    c->zc_auto_corr = 0;
    c->cubic = true;
}

int ready(sp_ctx *c)
{
    if (!c) return SP_ERR_ARG;
    if (!c->have_geom || !c->have_ham) return fail(c, SP_ERR_STATE, "geometry and Hamiltonian must be set first");
    return SP_OK;
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

// A compute call on a configured context: surfaces a pending status first.
int enter(sp_ctx *c)
{
    int rc = ready(c);
    return rc ? rc : status_enter(c);
}

int check_spins(sp_ctx *c, const void *p, const char *what)
{
    if (!p) return fail(c, SP_ERR_ARG, "%s is NULL", what);
    if (!aligned(p, c->prec == SP_F64 ? 32 : 16))
        return fail(c, SP_ERR_ARG, "%s is not %d-byte aligned", what, c->prec == SP_F64 ? 32 : 16);
    return SP_OK;
}

// Dipole field of `n` into the context's bdd buffer (or null when the
// Hamiltonian has no dipole term).
int dipole(sp_ctx *c, const void *n, const void **out, cudaStream_t st)
{
    *out = nullptr;
    if (c->h.dipole != SP_DIPOLE_FFT) return SP_OK;
    int rc = ensure(c, c->bdd, rec_bytes(c) * (size_t)c->N);
    if (rc) return rc;
    int pr = c->prof.begin(SP_PROF_DIPOLE, st);
    cudaError_t e = dipole_field(c->dip, c->prec, n, c->bdd.p, st);
    c->prof.end(pr, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "dipole field");
    *out = c->bdd.p;
    return SP_OK;
}

template <typename T> LlgConst<T> llg_const(const sp_ctx *c, const sp_llg_params *p)
{
    LlgConst<T> k{};
    k.dt = (T)p->dt;
    k.alpha = (T)p->alpha;
    for (int b = 0; b < c->nb; ++b) {
        double mu = c->mu_s[b] * kMuB;
        k.cA[b] = (T)(-kGamma / ((1.0 + p->alpha * p->alpha) * mu));
        k.sig[b] = (T)std::sqrt(2.0 * p->alpha * kBoltzmann * p->T * mu / (kGamma * p->dt));
    }
    llg_set_seed(k, p->seed);
    k.replica = p->replica;
    k.thermal = (p->T > 0 && p->alpha > 0) ? 1 : 0;
    return k;
}

// Noise amplitudes of a batch of replicas at temperatures T[r] on the device
// (c->rsig), uploaded when they differ from the last batch's.
template <typename T> int replica_amplitudes(sp_ctx *c, const sp_llg_params *p, int n_rep, const double *temps,
                                             cudaStream_t st)
{
    std::vector<double> key{(double)n_rep, (double)c->nb, (double)sizeof(T), p->dt, p->alpha};
    key.insert(key.end(), temps, temps + n_rep);
    if (c->rsig.p && key == c->rsig_key) return SP_OK;
    std::vector<T> amp((size_t)n_rep * c->nb);
    for (int r = 0; r < n_rep; ++r)
        for (int b = 0; b < c->nb; ++b) {
            double mu = c->mu_s[b] * kMuB;
            amp[(size_t)r * c->nb + b] = (T)std::sqrt(2.0 * p->alpha * kBoltzmann * temps[r] * mu / (kGamma * p->dt));
        }
    int rc = ensure(c, c->rsig, sizeof(T) * amp.size());
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(c->rsig.p, amp.data(), sizeof(T) * amp.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // amp is freed on return
    if (e != cudaSuccess) return cuda_fail(c, e, "replica noise amplitudes");
    c->rsig_key.swap(key);
    return SP_OK;
}

template <typename T> int llg_run(sp_ctx *c, void *n, const sp_llg_params *p, int n_steps, cudaStream_t st)
{
    bool rk4 = p->solver == SP_RK4;
    size_t NR = (size_t)c->N;
    int rc = ensure(c, c->pred, (rk4 ? 3 : 2) * sizeof(rec_t<T>) * NR);
    if (rc) return rc;
    rec_t<T> *np = (rec_t<T> *)c->pred.p;
    rec_t<T> *q = np + NR;
    rec_t<T> *nn = (rec_t<T> *)n;
    const Stencil<T> &S = *(const Stencil<T> *)(c->prec == SP_F64 ? (const void *)&c->Sd : (const void *)&c->Sf);
    const CubicParams<T> &CP = *(const CubicParams<T> *)(c->prec == SP_F64 ? (const void *)&c->Cd : (const void *)&c->Cf);
    bool cub = c->cubic && c->use_cubic &&
               (p->solver == SP_HEUN || p->solver == SP_DEPONDT || p->solver == SP_SIB ||
                (p->solver == SP_RK4 && c->h.dipole == SP_DIPOLE_NONE));
    LlgConst<T> k = llg_const<T>(c, p);
    int per0 = cub ? cubic_per(c) : 0, per1 = cub ? cubic_per(c, 1) : 0;
    if (c->use_small && c->N <= kSmallMax && c->h.dipole == SP_DIPOLE_NONE && !rk4 && !c->prof.on) {
        if (std::is_same<T, float>::value) {
            // whole steps inside one CTA (the lattice fits in shared memory)
            k.step = p->step0;
            cudaError_t e = launch_llg_small(p->solver, *(const Stencil<float> *)&S, (float4 *)nn,
                                             *(const LlgConst<float> *)&k, n_steps, st);
            return e == cudaSuccess ? SP_OK : cuda_fail(c, e, "small-lattice LLG launch");
        }
        cub = false;  // FP64: per-spin kernels in small blocks over many SMs
    }
    for (int s = 0; s < n_steps; ++s) {
        k.step = p->step0 + (uint64_t)s;
        const void *bd;
        if (rk4) {
            // stage states ping-pong between np and q; acc follows them
            rec_t<T> *acc = q + NR;
            const rec_t<T> *src[4] = {nn, np, q, np};
            rec_t<T> *dst[4] = {np, q, np, nn};
            for (int stg = 0; stg < 4; ++stg) {
                if ((rc = dipole(c, src[stg], &bd, st))) return rc;
                int pr = c->prof.begin(stg == 0 ? SP_PROF_LLG_PREDICTOR : SP_PROF_LLG_CORRECTOR, st);
                cudaError_t e = cub ? launch_cubic<T>(stg, SP_RK4, CP, src[stg], dst[stg], acc, nn, nullptr, k, per0, st,
                                                      cubic_rows(c, 0))
                                    : launch_rk4_stage<T>(stg, S, nn, src[stg], dst[stg], acc, (const rec_t<T> *)bd, k,
                                                          st);
                c->prof.end(pr, st);
                if (e != cudaSuccess) return cuda_fail(c, e, "RK4 stage launch");
            }
            continue;
        }
        if ((rc = dipole(c, nn, &bd, st))) return rc;
        int pr = c->prof.begin(SP_PROF_LLG_PREDICTOR, st);
        cudaError_t e = cub ? launch_cubic<T>(0, p->solver, CP, nn, np, q, nn, (const rec_t<T> *)bd, k, per0, st,
                                              cubic_rows(c, 0), cubic_lean_taken(c, 0))
                            : launch_llg_pred<T>(p->solver, S, nn, (const rec_t<T> *)bd, np, q, k, st);
        c->prof.end(pr, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "LLG predictor launch");
        if ((rc = dipole(c, np, &bd, st))) return rc;
        pr = c->prof.begin(SP_PROF_LLG_CORRECTOR, st);
        e = cub ? launch_cubic<T>(1, p->solver, CP, np, nullptr, q, nn, (const rec_t<T> *)bd, k, per1, st,
                                  cubic_rows(c, 1), cubic_lean_taken(c, 1))
                : launch_llg_corr<T>(p->solver, S, nn, np, q, (const rec_t<T> *)bd, k, st);
        c->prof.end(pr, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "LLG corrector launch");
    }
    return SP_OK;
}

// ------------------------------------------------------------ replicas
constexpr int kLlgGraphSteps = 32;  // steps per replayed graph of a replica batch
constexpr int kCubicMinRun = 8;     // shortest balanced run (planes per CTA) worth the 27-point ring
constexpr size_t kLlgGraphs = 4;    // instantiated graphs kept per context

__global__ void k_set_u64(unsigned long long *p, unsigned long long v) { *p = v; }
__global__ void k_add_u64(unsigned long long *p, unsigned long long v) { *p += v; }

// The instantiated graph of G steps of a replica batch for this key, captured
// on first use: G steps whose kernels read the Philox step as *ctr + j, then
// ctr += G.
template <typename T, typename F>
int replica_graph(sp_ctx *c, const std::vector<char> &key, int G, const LlgConst<T> &k, unsigned long long *ctr,
                  F &&one_step, cudaGraphExec_t *out)
{
    for (auto &g : c->lg_graphs)
        if (g.key == key) {
            *out = g.exec;
            return SP_OK;
        }
    cudaError_t e = cudaSuccess;
    if (!c->lg_stream) e = cudaStreamCreateWithFlags(&c->lg_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(c->lg_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(c, e, "replica graph capture");
    for (int j = 0; j < G && e == cudaSuccess; ++j) {
        LlgConst<T> kk = k;
        kk.step = (uint64_t)j;
        kk.step_base = ctr;
        e = one_step(kk, c->lg_stream);
    }
    if (e == cudaSuccess) {
        k_add_u64<<<1, 1, 0, c->lg_stream>>>(ctr, (unsigned long long)G);
        e = cudaGetLastError();
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->lg_stream, &g);
    if (e == cudaSuccess) e = e2;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "replica graph");
    if (c->lg_graphs.size() >= kLlgGraphs) {
        cudaGraphExecDestroy(c->lg_graphs.front().exec);
        c->lg_graphs.erase(c->lg_graphs.begin());
    }
    c->lg_graphs.push_back(LlgGraph{key, exec});
    *out = exec;
    return SP_OK;
}

// n_steps steps of n_rep > 1 replicas stored one after another at
// temperatures temps[r] (sp_llg_step_replicas).  Runs of kLlgGraphSteps
// steps are replayed from a CUDA graph (the step counter on the device),
// the rest launched one step at a time.
template <typename T>
int replicas_run(sp_ctx *c, void *n, const sp_llg_params *p, int n_steps, cudaStream_t st, int n_rep,
                 const double *temps)
{
    bool rk4 = p->solver == SP_RK4;
    size_t NR = (size_t)c->N * n_rep;
    int rc = ensure(c, c->pred, (rk4 ? 3 : 2) * sizeof(rec_t<T>) * NR);
    if (rc) return rc;
    if ((rc = replica_amplitudes<T>(c, p, n_rep, temps, st))) return rc;
    if ((rc = ensure(c, c->step_ctr, sizeof(unsigned long long)))) return rc;
    rec_t<T> *np = (rec_t<T> *)c->pred.p, *q = np + NR, *acc = q + NR, *nn = (rec_t<T> *)n;
    const Stencil<T> &S = *(const Stencil<T> *)(c->prec == SP_F64 ? (const void *)&c->Sd : (const void *)&c->Sf);
    const CubicParams<T> &CP = *(const CubicParams<T> *)(c->prec == SP_F64 ? (const void *)&c->Cd : (const void *)&c->Cf);
    LlgConst<T> k = llg_const<T>(c, p);
    k.n_rep = n_rep;
    k.nb = c->nb;
    k.rsig = (const T *)c->rsig.p;
    bool hot = false;
    for (int r = 0; r < n_rep; ++r) hot = hot || temps[r] > 0;
    k.thermal = (hot && p->alpha > 0) ? 1 : 0;
    bool cub = c->cubic && c->use_cubic;  // all four solvers (a batch has no dipole term)
    int per0 = cub ? cubic_per_batch(c, 0, n_rep) : 0, per1 = cub ? cubic_per_batch(c, 1, n_rep) : 0;
    // runs of a few planes per CTA are mostly the ring's prologue: the
    // per-spin kernels are faster there (unless the user fixed the split)
    if (cub && c->zc == 0 && per0 < kCubicMinRun) cub = false;
    auto one_step = [&](const LlgConst<T> &kk, cudaStream_t s) -> cudaError_t {
        if (rk4) {
            const rec_t<T> *src[4] = {nn, np, q, np};
            rec_t<T> *dst[4] = {np, q, np, nn};
            for (int stg = 0; stg < 4; ++stg) {
                cudaError_t e = cub ? launch_cubic<T>(stg, SP_RK4, CP, src[stg], dst[stg], acc, nn, nullptr, kk, per0, s)
                                    : launch_rk4_stage<T>(stg, S, nn, src[stg], dst[stg], acc, nullptr, kk, s);
                if (e != cudaSuccess) return e;
            }
            return cudaSuccess;
        }
        cudaError_t e = cub ? launch_cubic<T>(0, p->solver, CP, nn, np, q, nn, nullptr, kk, per0, s)
                            : launch_llg_pred<T>(p->solver, S, nn, nullptr, np, q, kk, s);
        if (e != cudaSuccess) return e;
        return cub ? launch_cubic<T>(1, p->solver, CP, np, nullptr, q, nn, nullptr, kk, per1, s)
                   : launch_llg_corr<T>(p->solver, S, nn, np, q, nullptr, kk, s);
    };
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream query");
    int s = 0;
    if (n_steps >= 2 && cap == cudaStreamCaptureStatusNone) {
        int G = std::min(n_steps, kLlgGraphSteps);
        unsigned long long *ctr = (unsigned long long *)c->step_ctr.p;
        LlgConst<T> kk;
        std::memcpy(&kk, &k, sizeof kk);  // byte copy: the key compares padding too
        kk.step = 0;
        kk.step_base = ctr;
        struct Key {
            const void *n, *pred, *ctr;
            int n_rep, solver, cub, per0, per1, G;
        } key;
        std::memset(&key, 0, sizeof key);
        key.n = nn;
        key.pred = c->pred.p;
        key.ctr = ctr;
        key.n_rep = n_rep;
        key.solver = p->solver;
        key.cub = cub;
        key.per0 = per0;
        key.per1 = per1;
        key.G = G;
        std::vector<char> kb(sizeof key + sizeof kk + sizeof S + sizeof CP);
        std::memcpy(kb.data(), &key, sizeof key);
        std::memcpy(kb.data() + sizeof key, &kk, sizeof kk);
        std::memcpy(kb.data() + sizeof key + sizeof kk, &S, sizeof S);
        std::memcpy(kb.data() + sizeof key + sizeof kk + sizeof S, &CP, sizeof CP);
        cudaGraphExec_t exec = nullptr;
        if ((rc = replica_graph<T>(c, kb, G, k, ctr, one_step, &exec))) return rc;
        k_set_u64<<<1, 1, 0, st>>>(ctr, (unsigned long long)p->step0);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "step counter");
        for (; s + G <= n_steps; s += G)
            if ((e = cudaGraphLaunch(exec, st)) != cudaSuccess) return cuda_fail(c, e, "replica graph launch");
    }
    for (; s < n_steps; ++s) {
        k.step = p->step0 + (uint64_t)s;
        if ((e = one_step(k, st)) != cudaSuccess) return cuda_fail(c, e, "LLG replica launch");
    }
    return SP_OK;
}

// n_steps steps of n_sys systems of (possibly) different lattices, system k
// (context ctxs[k]) at records spin0[k] at temperature temps[k] on the
// thermal stream p->replica + k: one launch per pass for all of them.
template <typename T>
int llg_batch_run(sp_ctx *const *ctxs, int n_sys, void *spins, const long long *spin0, const double *temps,
                  const sp_llg_params *p, int n_steps, cudaStream_t st)
{
    sp_ctx *c0 = ctxs[0];
    std::vector<Stencil<T>> sten(n_sys);
    std::vector<LlgSys<T>> sys(n_sys);
    std::vector<int2> blk;
    long long total = 0;
    bool hot = false;
    for (int k = 0; k < n_sys; ++k) {
        sp_ctx *c = ctxs[k];
        sten[k] = *(const Stencil<T> *)(c->prec == SP_F64 ? (const void *)&c->Sd : (const void *)&c->Sf);
        LlgSys<T> s{};
        s.spin0 = spin0[k];
        s.N = c->N;
        s.replica = p->replica + (uint32_t)k;
        for (int b = 0; b < c->nb; ++b) {  // as llg_const does for one lattice
            double mu = c->mu_s[b] * kMuB;
            s.cA[b] = (T)(-kGamma / ((1.0 + p->alpha * p->alpha) * mu));
            s.sig[b] = (T)std::sqrt(2.0 * p->alpha * kBoltzmann * temps[k] * mu / (kGamma * p->dt));
        }
        sys[k] = s;
        for (int t = 0; t < blocks_for(c->N); ++t) blk.push_back(make_int2(k, t));
        total = std::max(total, spin0[k] + (long long)c->N);
        hot = hot || temps[k] > 0;
    }
    int rc = ensure(c0, c0->pred, 2 * sizeof(rec_t<T>) * (size_t)total);
    if (rc) return rc;
    size_t sb = sizeof(Stencil<T>) * n_sys, yb = sizeof(LlgSys<T>) * n_sys, bb = sizeof(int2) * blk.size();
    size_t o1 = (sb + 255) / 256 * 256, o2 = o1 + (yb + 255) / 256 * 256;
    std::vector<char> key(o2 + bb);
    std::memcpy(key.data(), sten.data(), sb);
    std::memcpy(key.data() + o1, sys.data(), yb);
    std::memcpy(key.data() + o2, blk.data(), bb);
    if (key != c0->lb_key) {
        if ((rc = ensure(c0, c0->lb_tab, key.size()))) return rc;
        cudaError_t e = cudaMemcpyAsync(c0->lb_tab.p, key.data(), key.size(), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host copy is freed on return
        if (e != cudaSuccess) return cuda_fail(c0, e, "batch tables");
        c0->lb_key.swap(key);
    }
    const char *tab = (const char *)c0->lb_tab.p;
    const Stencil<T> *Sv = (const Stencil<T> *)tab;
    const LlgSys<T> *Y = (const LlgSys<T> *)(tab + o1);
    const int2 *B = (const int2 *)(tab + o2);
    rec_t<T> *nn = (rec_t<T> *)spins, *np = (rec_t<T> *)c0->pred.p, *q = np + total;
    LlgConst<T> k = llg_const<T>(c0, p);  // dt, alpha, seed round keys; the rest per system
    k.thermal = (hot && p->alpha > 0) ? 1 : 0;
    const int nblk = (int)blk.size();
    auto one_step = [&](const LlgConst<T> &kk, cudaStream_t s) -> cudaError_t {
        cudaError_t e = launch_llg_batch<T>(0, p->solver, nblk, B, Sv, Y, nn, np, q, kk, s);
        return e == cudaSuccess ? launch_llg_batch<T>(1, p->solver, nblk, B, Sv, Y, nn, np, q, kk, s) : e;
    };
    // runs of kLlgGraphSteps steps replay a CUDA graph whose kernels read the
    // Philox step from a device counter (as the replica batches do)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return cuda_fail(c0, e, "stream query");
    int s = 0;
    if (n_steps >= 2 && cap == cudaStreamCaptureStatusNone) {
        if ((rc = ensure(c0, c0->step_ctr, sizeof(unsigned long long)))) return rc;
        int G = std::min(n_steps, kLlgGraphSteps);
        unsigned long long *ctr = (unsigned long long *)c0->step_ctr.p;
        LlgConst<T> kk;
        std::memcpy(&kk, &k, sizeof kk);  // byte copy: the key compares padding too
        kk.step = 0;
        kk.step_base = ctr;
        struct Key {
            const void *n, *pred, *ctr, *tab;
            int solver, G, nblk, tag;
        } gkey;
        std::memset(&gkey, 0, sizeof gkey);
        gkey.n = nn;
        gkey.pred = c0->pred.p;
        gkey.ctr = ctr;
        gkey.tab = tab;
        gkey.solver = p->solver;
        gkey.G = G;
        gkey.nblk = nblk;
        gkey.tag = 0x4c42;  // batches of lattices (the replica graphs carry other keys)
        std::vector<char> kb(sizeof gkey + sizeof kk);
        std::memcpy(kb.data(), &gkey, sizeof gkey);
        std::memcpy(kb.data() + sizeof gkey, &kk, sizeof kk);
        cudaGraphExec_t exec = nullptr;
        if ((rc = replica_graph<T>(c0, kb, G, k, ctr, one_step, &exec))) return rc;
        k_set_u64<<<1, 1, 0, st>>>(ctr, (unsigned long long)p->step0);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c0, e, "step counter");
        for (; s + G <= n_steps; s += G)
            if ((e = cudaGraphLaunch(exec, st)) != cudaSuccess) return cuda_fail(c0, e, "batch graph launch");
    }
    for (; s < n_steps; ++s) {
        k.step = p->step0 + (uint64_t)s;
        if ((e = one_step(k, st)) != cudaSuccess) return cuda_fail(c0, e, "batched LLG launch");
    }
    return SP_OK;
}

}  // namespace

namespace {

template <typename T> int autotune_run(sp_ctx *c, const void *n, int *chosen, cudaStream_t st)
{
    // np, q, and the corrector's output (the caller's spins are only read)
    int rc = ensure(c, c->pred, 3 * sizeof(rec_t<T>) * (size_t)c->N);
    if (rc) return rc;
    rec_t<T> *np = (rec_t<T> *)c->pred.p;
    rec_t<T> *q = np + c->N, *out = q + c->N;
    const CubicParams<T> &CP = *(const CubicParams<T> *)(c->prec == SP_F64 ? (const void *)&c->Cd : (const void *)&c->Cf);
    sp_llg_params p{SP_HEUN, 1e-3, 0.1, 10.0, 0, 0, 0};
    LlgConst<T> k = llg_const<T>(c, &p);
    k.step = 0;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return fail(c, SP_ERR_CUDA, "cudaEventCreate");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(c, SP_ERR_CUDA, "cudaEventCreate");
    }
    auto launch = [&](int pass, int per, int rows) {
        return pass == 0
                   ? launch_cubic<T>(0, SP_HEUN, CP, (const rec_t<T> *)n, np, q, nullptr, nullptr, k, per, st, rows,
                                     cubic_lean_taken(c, 0))
                   : launch_cubic<T>(1, SP_HEUN, CP, np, nullptr, q, out, nullptr, k, per, st, rows,
                                     cubic_lean_taken(c, 1));
    };
    int user = c->zc, user_corr = c->zc_corr, user_rows[2] = {c->rows[0], c->rows[1]};
    c->zc = 0;
    c->zc_corr = 0;
    int best_of[2] = {1, 1}, best_rows[2] = {1, 1};
    cudaError_t e = cudaSuccess;
    // each pass and tile height (one or two columns per thread; two in FP32
    // only): the balanced single-wave split for its own occupancy and finer
    // ones (more CTAs, shorter runs of planes), plus fixed run lengths
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
        float best = 1e30f;
        for (int rows = 1; rows <= 2 && e == cudaSuccess; ++rows) {
            c->rows[pass] = rows;
            if (cubic_rows(c, pass) != rows) continue;
            (pass == 0 ? c->zc_auto : c->zc_auto_corr) = 0;
            int bal = cubic_per(c, pass);
            std::vector<int> cands = {bal, (bal + 1) / 2, (bal + 2) / 3, (bal + 3) / 4, (bal + 5) / 6, 4, 8, 16, 32};
            std::sort(cands.begin(), cands.end());
            cands.erase(std::unique(cands.begin(), cands.end()), cands.end());
            if (pass == 1) e = launch(0, cubic_per(c, 0), cubic_rows(c, 0));  // the corrector reads its output
            if (rows == 1) best_of[pass] = bal;
            for (int per : cands) {
                if (per < 1 || e != cudaSuccess) continue;
                e = launch(pass, per, rows);  // warm-up
                // the best of three runs of kTuneRun back-to-back launches
                // (the steady state of a long call, launch overlap included)
                constexpr int kTuneRun = 8;
                float t = 1e30f;
                for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
                    e = cudaEventRecord(e0, st);
                    for (int l = 0; l < kTuneRun && e == cudaSuccess; ++l) e = launch(pass, per, rows);
                    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                    float ms = 0;
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                    if (e == cudaSuccess) t = std::min(t, ms);
                }
                if (e == cudaSuccess && t < best) {
                    best = t;
                    best_of[pass] = per;
                    best_rows[pass] = rows;
                }
            }
        }
        c->rows[pass] = best_rows[pass];
        (pass == 0 ? c->zc_auto : c->zc_auto_corr) = 0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        c->zc = user;
        c->zc_corr = user_corr;
        c->rows[0] = user_rows[0];
        c->rows[1] = user_rows[1];
        c->zc_auto = c->zc_auto_corr = 0;
        return cuda_fail(c, e, "autotune");
    }
    c->zc = best_of[0];
    c->zc_corr = best_of[1];
    if (chosen) *chosen = best_of[0];
    return SP_OK;
}

}  // namespace

// ===================================================================== status word
unsigned *status_word(sp_ctx *c)
{
    if (c->status_d) return c->status_d;
    void *h = nullptr, *d = nullptr;
    cudaError_t e = cudaHostAlloc(&h, 4 * sizeof(unsigned), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        std::memset(h, 0, 4 * sizeof(unsigned));
        e = cudaHostGetDevicePointer(&d, h, 0);
        if (e != cudaSuccess) cudaFreeHost(h);
    }
    if (e != cudaSuccess) {
        cuda_fail(c, e, "status word allocation");
        return nullptr;
    }
    c->status_h = (unsigned *)h;
    c->status_d = (unsigned *)d;
    return c->status_d;
}

namespace {
std::string site_names(unsigned bits)
{
    static const char *names[] = {"spin state", "effective field", "energy or torque", "GNEB energies or forces",
                                  "observables", "Hessian product"};
    std::string s;
    for (int k = 0; k < 6; ++k)
        if (bits & (1u << k)) s += std::string(s.empty() ? "" : ", ") + names[k];
    return s.empty() ? std::string("unknown") : s;
}

// Read and clear the status word; the error it stands for (SP_OK if clear).
int status_take(sp_ctx *c)
{
    if (!c->status_h) return SP_OK;
    volatile unsigned *w = c->status_h;
    unsigned nan = w[0], tmo = w[1];
    if (!nan && !tmo) return SP_OK;
    w[0] = 0;
    w[1] = 0;
    if (tmo) return fail(c, SP_ERR_TIMEOUT, "a bounded device-side wait gave up (sites 0x%x)", tmo);
    return fail(c, SP_ERR_NAN, "a non-finite value was detected in the %s of an earlier call", site_names(nan).c_str());
}
}  // namespace

int status_enter(sp_ctx *c) { return status_take(c); }

int status_check_records(sp_ctx *c, const void *recs, long n_rec, unsigned site, cudaStream_t st)
{
    unsigned *w = status_word(c);
    if (!w) return SP_ERR_CUDA;
    cudaError_t e = c->prec == SP_F64 ? launch_check_records<double>((const dq4 *)recs, n_rec, w, site, st)
                                      : launch_check_records<float>((const float4 *)recs, n_rec, w, site, st);
    return e == cudaSuccess ? SP_OK : cuda_fail(c, e, "finiteness check launch");
}

int status_check_doubles(sp_ctx *c, const double *v, long n_val, unsigned site, cudaStream_t st)
{
    unsigned *w = status_word(c);
    if (!w) return SP_ERR_CUDA;
    cudaError_t e = launch_check_doubles(v, n_val, w, site, st);
    return e == cudaSuccess ? SP_OK : cuda_fail(c, e, "finiteness check launch");
}

// ===================================================================== C ABI
extern "C" {

int sp_create(sp_ctx **out, int precision)
{
    if (!out) return SP_ERR_ARG;
    *out = nullptr;
    if (precision != SP_F32 && precision != SP_F64) return SP_ERR_ARG;
    sp_ctx *c = new (std::nothrow) sp_ctx();
    if (!c) return SP_ERR_STATE;
    c->prec = precision;
    cudaGetDevice(&c->device);
    *out = c;
    return SP_OK;
}

int sp_destroy(sp_ctx *c)
{
    if (!c) return SP_OK;
    bool any = c->pred.p || c->partials.p || c->bdd.p || c->dip || c->mins || c->hess || c->htst || c->mc;
    if (any) cudaDeviceSynchronize();
    if (c->pred.p) cudaFree(c->pred.p);
    if (c->partials.p) cudaFree(c->partials.p);
    if (c->bdd.p) cudaFree(c->bdd.p);
    if (c->qbuf.p) cudaFree(c->qbuf.p);
    if (c->rsig.p) cudaFree(c->rsig.p);
    if (c->step_ctr.p) cudaFree(c->step_ctr.p);
    if (c->lb_tab.p) cudaFree(c->lb_tab.p);
    if (c->status_h) cudaFreeHost(c->status_h);
    for (auto &g : c->lg_graphs) cudaGraphExecDestroy(g.exec);
    if (c->lg_stream) cudaStreamDestroy(c->lg_stream);
    mc_scratch_destroy(c->mc);
    hess_scratch_destroy(c->hess);
    htst_scratch_destroy(c->htst);
    dipole_destroy(c->dip);
    min_scratch_destroy(c->mins);
    delete c;
    return SP_OK;
}

const char *sp_last_error(const sp_ctx *c)
{
    if (!c) return "no context";
    return c->err.c_str();
}

int sp_set_geometry(sp_ctx *c, const double *bravais, int n_basis, const double *basis, const int *n_cells,
                    const int *periodic, double lattice_constant, const double *mu_s)
{
    if (!c) return SP_ERR_ARG;
    if (!bravais || !basis || !n_cells || !periodic || !mu_s) return fail(c, SP_ERR_ARG, "NULL geometry argument");
    if (n_basis < 1 || n_basis > SP_MAX_BASIS) return fail(c, SP_ERR_ARG, "n_basis %d out of 1..%d", n_basis, SP_MAX_BASIS);
    if (!(lattice_constant > 0) || !std::isfinite(lattice_constant))
        return fail(c, SP_ERR_ARG, "lattice constant must be positive");
    long long N = n_basis;
    for (int k = 0; k < 3; ++k) {
        if (n_cells[k] < 1) return fail(c, SP_ERR_ARG, "n_cells[%d] = %d < 1", k, n_cells[k]);
        N *= n_cells[k];
        if (N >= (1LL << 31)) return fail(c, SP_ERR_ARG, "more than 2^31 - 1 spins");
    }
    for (int b = 0; b < n_basis; ++b)
        if (!(mu_s[b] > 0) || !std::isfinite(mu_s[b])) return fail(c, SP_ERR_ARG, "mu_s[%d] must be positive", b);
    for (int k = 0; k < 9; ++k)
        if (!std::isfinite(bravais[k])) return fail(c, SP_ERR_ARG, "non-finite Bravais vector");
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) c->A[k][l] = bravais[3 * k + l];
    c->nb = n_basis;
    for (int b = 0; b < n_basis; ++b) {
        for (int l = 0; l < 3; ++l) c->basis[b][l] = basis[3 * b + l];
        c->mu_s[b] = mu_s[b];
    }
    for (int k = 0; k < 3; ++k) {
        c->nc[k] = n_cells[k];
        c->per[k] = periodic[k] ? 1 : 0;
    }
    c->a = lattice_constant;
    c->N = (int)N;
    c->have_geom = true;
    c->have_ham = false;
    return SP_OK;
}

int sp_set_hamiltonian(sp_ctx *c, const sp_hamiltonian *h)
{
    if (!c) return SP_ERR_ARG;
    if (!c->have_geom) return fail(c, SP_ERR_STATE, "set the geometry before the Hamiltonian");
    if (!h) return fail(c, SP_ERR_ARG, "NULL Hamiltonian");
    if (h->n_shells < 0 || h->n_shells > SP_MAX_SHELLS) return fail(c, SP_ERR_ARG, "n_shells out of range");
    if (h->n_dmi_shells < 0 || h->n_dmi_shells > SP_MAX_SHELLS) return fail(c, SP_ERR_ARG, "n_dmi_shells out of range");
    if (h->dmi_kind < SP_DMI_NONE || h->dmi_kind > SP_DMI_INTERFACIAL) return fail(c, SP_ERR_ARG, "bad dmi_kind");
    if (h->dipole != SP_DIPOLE_NONE && h->dipole != SP_DIPOLE_FFT) return fail(c, SP_ERR_ARG, "bad dipole mode");
    if (h->n_pairs < 0 || (h->n_pairs > 0 && !h->pairs)) return fail(c, SP_ERR_ARG, "bad explicit pair list");
    for (int p = 0; p < h->n_pairs; ++p) {
        const sp_pair &q = h->pairs[p];
        if (q.i < 0 || q.i >= c->nb || q.j < 0 || q.j >= c->nb) return fail(c, SP_ERR_ARG, "pair %d: bad basis index", p);
        if (q.i == q.j && q.d[0] == 0 && q.d[1] == 0 && q.d[2] == 0) return fail(c, SP_ERR_ARG, "pair %d: self pair", p);
    }
    if (h->dipole == SP_DIPOLE_FFT)
        for (int k = 0; k < 3; ++k)
            if (c->per[k] && c->nc[k] > 1)
                return fail(c, SP_ERR_UNSUPPORTED, "dipole term with a periodic direction is not implemented");
    c->h = *h;
    c->pairs.assign(h->pairs, h->pairs + h->n_pairs);
    c->h.pairs = nullptr;
    c->have_ham = false;
    int rc = build_stencil(c);
    if (rc) return rc;
    fill_stencil(c, c->Sf);
    fill_stencil(c, c->Sd);
    detect_cubic(c);
    dipole_destroy(c->dip);
    c->dip = nullptr;
    if (h->dipole == SP_DIPOLE_FFT) {
        DipoleGeom g;
        for (int k = 0; k < 3; ++k) {
            g.nc[k] = c->nc[k];
            for (int l = 0; l < 3; ++l) g.A[k][l] = c->A[k][l] * c->a;
        }
        g.nb = c->nb;
        for (int b = 0; b < c->nb; ++b) {
            g.mu[b] = c->mu_s[b];
            for (int l = 0; l < 3; ++l) g.basis[b][l] = c->basis[b][l];
        }
        int e = dipole_create(&c->dip, g);
        if (!e) dipole_force_generic(c->dip, c->generic_fft);
        if (e == SP_ERR_UNSUPPORTED) return fail(c, e, "dipole FFT supports one basis atom and 2D grids up to 4096");
        if (e) return fail(c, e, "dipole plan creation failed");
    }
    c->have_ham = true;
    return SP_OK;
}

int sp_n_spins(const sp_ctx *c, int *n)
{
    if (!c || !n) return SP_ERR_ARG;
    if (!c->have_geom) return SP_ERR_STATE;
    *n = c->N;
    return SP_OK;
}

static int field_common(sp_ctx *c, const void *n, void *out, double sign, void *stream)
{
    int rc = enter(c);
    if (rc) return rc;
    if ((rc = check_spins(c, n, "spins")) || (rc = check_spins(c, out, "output"))) return rc;
    if (n == out) return fail(c, SP_ERR_ARG, "input and output must not overlap");
    cudaStream_t st = (cudaStream_t)stream;
    const void *bd;
    if ((rc = dipole(c, n, &bd, st))) return rc;
    cudaError_t e = c->prec == SP_F64
                        ? launch_field<double>(c->Sd, (const dq4 *)n, (const dq4 *)bd, (dq4 *)out, sign, st)
                        : launch_field<float>(c->Sf, (const float4 *)n, (const float4 *)bd, (float4 *)out, (float)sign, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "field launch");
    return status_check_records(c, out, c->N, SITE_FIELD, st);
}

int sp_effective_field(sp_ctx *c, const void *n_dev, void *B_dev, void *stream)
{
    return field_common(c, n_dev, B_dev, 1.0, stream);
}

int sp_gradient(sp_ctx *c, const void *n_dev, void *grad_dev, void *stream)
{
    return field_common(c, n_dev, grad_dev, -1.0, stream);
}

static int energy_common(sp_ctx *c, const void *n, double *e_out, double *t_out, void *stream)
{
    int rc = enter(c);
    if (rc) return rc;
    if ((rc = check_spins(c, n, "spins"))) return rc;
    if (!e_out && !t_out) return fail(c, SP_ERR_ARG, "NULL output");
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = ensure(c, c->partials, sizeof(double) * 8 * (size_t)blocks_for(c->N > 0 ? c->N : 1)))) return rc;
    const void *bd;
    if ((rc = dipole(c, n, &bd, st))) return rc;
    cudaError_t e = c->prec == SP_F64
                        ? launch_energy<double>(c->Sd, (const dq4 *)n, (const dq4 *)bd, (double *)c->partials.p, e_out, t_out, st)
                        : launch_energy<float>(c->Sf, (const float4 *)n, (const float4 *)bd, (double *)c->partials.p, e_out, t_out, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "energy launch");
    return e_out ? status_check_doubles(c, e_out, 6, SITE_ENERGY, st) : status_check_doubles(c, t_out, 1, SITE_ENERGY, st);
}

int sp_energy(sp_ctx *c, const void *n_dev, double *e_dev, void *stream)
{
    if (c && !e_dev) return fail(c, SP_ERR_ARG, "NULL energy output");
    return energy_common(c, n_dev, e_dev, nullptr, stream);
}

int sp_max_torque(sp_ctx *c, const void *n_dev, double *torque_dev, void *stream)
{
    if (c && !torque_dev) return fail(c, SP_ERR_ARG, "NULL torque output");
    return energy_common(c, n_dev, nullptr, torque_dev, stream);
}

int sp_llg_step(sp_ctx *c, void *n_dev, const sp_llg_params *p, int n_steps, void *stream)
{
    int rc = enter(c);
    if (rc) return rc;
    if ((rc = check_spins(c, n_dev, "spins"))) return rc;
    if (!p) return fail(c, SP_ERR_ARG, "NULL parameters");
    if (p->solver < SP_DEPONDT || p->solver > SP_RK4) return fail(c, SP_ERR_ARG, "unknown solver %d", p->solver);
    if (!(p->dt > 0) || !std::isfinite(p->dt)) return fail(c, SP_ERR_ARG, "dt must be positive");
    if (!(p->alpha >= 0) || !std::isfinite(p->alpha)) return fail(c, SP_ERR_ARG, "alpha must be >= 0");
    if (!(p->T >= 0) || !std::isfinite(p->T)) return fail(c, SP_ERR_ARG, "T must be >= 0");
    if (n_steps < 0) return fail(c, SP_ERR_ARG, "n_steps must be >= 0");
    if (n_steps == 0 || c->N == 0) return SP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    rc = c->prec == SP_F64 ? llg_run<double>(c, n_dev, p, n_steps, st) : llg_run<float>(c, n_dev, p, n_steps, st);
    return rc ? rc : status_check_records(c, n_dev, c->N, SITE_STATE, st);
}

int sp_llg_step_replicas(sp_ctx *c, void *spins_dev, int n_rep, const double *T, const sp_llg_params *p, int n_steps,
                         void *stream)
{
    int rc = enter(c);
    if (rc) return rc;
    if ((rc = check_spins(c, spins_dev, "spins"))) return rc;
    if (!p || !T) return fail(c, SP_ERR_ARG, "NULL parameters or temperatures");
    if (n_rep < 1) return fail(c, SP_ERR_ARG, "n_rep must be >= 1");
    if (p->solver < SP_DEPONDT || p->solver > SP_RK4) return fail(c, SP_ERR_ARG, "unknown solver %d", p->solver);
    if (!(p->dt > 0) || !std::isfinite(p->dt)) return fail(c, SP_ERR_ARG, "dt must be positive");
    if (!(p->alpha >= 0) || !std::isfinite(p->alpha)) return fail(c, SP_ERR_ARG, "alpha must be >= 0");
    for (int r = 0; r < n_rep; ++r)
        if (!(T[r] >= 0) || !std::isfinite(T[r])) return fail(c, SP_ERR_ARG, "replica %d: T must be >= 0", r);
    if (n_steps < 0) return fail(c, SP_ERR_ARG, "n_steps must be >= 0");
    if ((long long)n_rep * c->N >= (1LL << 31)) return fail(c, SP_ERR_ARG, "replicas larger than 2^31 spins");
    if ((unsigned long long)p->replica + (unsigned long long)n_rep > (1ULL << 29))
        return fail(c, SP_ERR_ARG, "thermal streams replica .. replica + n_rep - 1 must stay below 2^29");
    if (c->h.dipole != SP_DIPOLE_NONE) return fail(c, SP_ERR_UNSUPPORTED, "replicas with the dipole term");
    if (n_steps == 0 || c->N == 0) return SP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (n_rep == 1) {  // one replica is a plain call at its own temperature
        sp_llg_params one = *p;
        one.T = T[0];
        rc = c->prec == SP_F64 ? llg_run<double>(c, spins_dev, &one, n_steps, st)
                               : llg_run<float>(c, spins_dev, &one, n_steps, st);
    } else {
        rc = c->prec == SP_F64 ? replicas_run<double>(c, spins_dev, p, n_steps, st, n_rep, T)
                               : replicas_run<float>(c, spins_dev, p, n_steps, st, n_rep, T);
    }
    return rc ? rc : status_check_records(c, spins_dev, (long)n_rep * c->N, SITE_STATE, st);
}

int sp_llg_step_batch(sp_ctx *const *ctxs, int n_sys, void *spins_dev, const long long *offsets, const double *T,
                      const sp_llg_params *p, int n_steps, void *stream)
{
    if (!ctxs || n_sys < 1 || !ctxs[0]) return SP_ERR_ARG;
    sp_ctx *c0 = ctxs[0];
    int rc = status_enter(c0);
    if (rc) return rc;
    if (!offsets || !T || !p) return fail(c0, SP_ERR_ARG, "NULL batch argument");
    if ((rc = check_spins(c0, spins_dev, "spins"))) return rc;
    if (p->solver != SP_DEPONDT && p->solver != SP_HEUN && p->solver != SP_SIB)
        return fail(c0, p->solver == SP_RK4 ? SP_ERR_UNSUPPORTED : SP_ERR_ARG,
                    "batched LLG steps take the Depondt, Heun or SIB solver");
    if (!(p->dt > 0) || !std::isfinite(p->dt)) return fail(c0, SP_ERR_ARG, "dt must be positive");
    if (!(p->alpha >= 0) || !std::isfinite(p->alpha)) return fail(c0, SP_ERR_ARG, "alpha must be >= 0");
    if (n_steps < 0) return fail(c0, SP_ERR_ARG, "n_steps must be >= 0");
    if ((unsigned long long)p->replica + (unsigned long long)n_sys > (1ULL << 29))
        return fail(c0, SP_ERR_ARG, "thermal streams replica .. replica + n_sys - 1 must stay below 2^29");
    std::vector<std::pair<long long, long long>> spans;
    for (int k = 0; k < n_sys; ++k) {
        sp_ctx *c = ctxs[k];
        if (!c) return fail(c0, SP_ERR_ARG, "NULL context for system %d", k);
        if (!c->have_geom || !c->have_ham) return fail(c0, SP_ERR_STATE, "system %d: context not configured", k);
        if (c->prec != c0->prec) return fail(c0, SP_ERR_ARG, "system %d: precision differs from system 0", k);
        if (c->h.dipole != SP_DIPOLE_NONE) return fail(c0, SP_ERR_UNSUPPORTED, "system %d: dipole term", k);
        if (!(T[k] >= 0) || !std::isfinite(T[k])) return fail(c0, SP_ERR_ARG, "system %d: T must be >= 0", k);
        if (offsets[k] < 0 || offsets[k] + c->N >= (1LL << 31)) return fail(c0, SP_ERR_ARG, "system %d: bad offset", k);
        spans.push_back({offsets[k], offsets[k] + c->N});
    }
    std::sort(spans.begin(), spans.end());
    for (size_t k = 1; k < spans.size(); ++k)
        if (spans[k].first < spans[k - 1].second) return fail(c0, SP_ERR_ARG, "systems overlap in the batch buffer");
    if (n_steps == 0) return SP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    rc = c0->prec == SP_F64 ? llg_batch_run<double>(ctxs, n_sys, spins_dev, offsets, T, p, n_steps, st)
                            : llg_batch_run<float>(ctxs, n_sys, spins_dev, offsets, T, p, n_steps, st);
    if (rc) return rc;
    return status_check_records(c0, spins_dev, (long)spans.back().second, SITE_STATE, st);
}

int sp_minimise(sp_ctx *c, void *n_dev, void *v_dev, double dt, double mass, double tol, int max_iter, int check_every,
                int *iters, double *max_torque, void *stream)
{
    int rc = enter(c);
    if (rc) return rc;
    if ((rc = check_spins(c, n_dev, "spins")) || (rc = check_spins(c, v_dev, "velocities"))) return rc;
    if (n_dev == v_dev) return fail(c, SP_ERR_ARG, "spins and velocities must not overlap");
    if (!(dt > 0) || !(mass > 0) || !std::isfinite(dt) || !std::isfinite(mass))
        return fail(c, SP_ERR_ARG, "dt and mass must be positive");
    if (!(tol >= 0)) return fail(c, SP_ERR_ARG, "tol must be >= 0");
    if (max_iter < 0 || check_every < 1) return fail(c, SP_ERR_ARG, "max_iter >= 0 and check_every >= 1 required");
    if (c->h.dipole != SP_DIPOLE_NONE) return fail(c, SP_ERR_UNSUPPORTED, "minimisation with the dipole term");
    MinArgs a{dt, mass, tol, max_iter, check_every};
    int it = 0;
    double mt = 0;
    int e = c->prec == SP_F64 ? vp_minimise<double>(&c->mins, c->Sd, n_dev, v_dev, a, &it, &mt, (cudaStream_t)stream)
                              : vp_minimise<float>(&c->mins, c->Sf, n_dev, v_dev, a, &it, &mt, (cudaStream_t)stream);
    if (e) return fail(c, e, "minimisation failed (%s)", e == SP_ERR_CUDA ? cudaGetErrorString(cudaGetLastError()) : "");
    if (iters) *iters = it;
    if (max_torque) *max_torque = mt;
    if (!std::isfinite(mt)) return fail(c, SP_ERR_NAN, "minimisation: the max torque is not finite");
    return SP_OK;
}

int sp_gneb_step(sp_ctx *c, void *chain_dev, void *vel_dev, int n_images, const sp_gneb_params *p, int n_iter,
                 double *energies_dev, double *max_force_dev, void *stream)
{
    int rc = enter(c);
    if (rc) return rc;
    if ((rc = check_spins(c, chain_dev, "chain")) || (rc = check_spins(c, vel_dev, "velocities"))) return rc;
    if (!p) return fail(c, SP_ERR_ARG, "NULL parameters");
    if (n_images < 3) return fail(c, SP_ERR_ARG, "a chain needs at least 3 images");
    if (n_iter < 0) return fail(c, SP_ERR_ARG, "n_iter must be >= 0");
    if (!(p->dt > 0) || !(p->mass > 0)) return fail(c, SP_ERR_ARG, "dt and mass must be positive");
    if (!energies_dev || !max_force_dev) return fail(c, SP_ERR_ARG, "NULL output");
    if ((long long)n_images * c->N >= (1LL << 31)) return fail(c, SP_ERR_ARG, "chain larger than 2^31 spins");
    if (c->h.dipole != SP_DIPOLE_NONE) return fail(c, SP_ERR_UNSUPPORTED, "GNEB with the dipole term");
    if (!(p->energy_weight >= 0 && p->energy_weight < 1)) return fail(c, SP_ERR_ARG, "energy_weight must be in [0, 1)");
    if (p->image_types)
        for (int v = 0; v < n_images; ++v)
            if (p->image_types[v] < SP_IMAGE_NORMAL || p->image_types[v] > SP_IMAGE_FALLING)
                return fail(c, SP_ERR_ARG, "image %d: unknown image type %d", v, p->image_types[v]);
    GnebArgs a{p->dt, p->mass, p->k_spring, p->climbing ? 1 : 0, n_images, n_iter, p->image_types, p->energy_weight};
    a.persistent = c->gneb_persistent;
    a.wait_limit = c->wait_limit;
    if (a.persistent && !(a.status = status_word(c))) return SP_ERR_CUDA;
    int e = c->prec == SP_F64
                ? gneb_run<double>(&c->mins, c->Sd, chain_dev, vel_dev, a, energies_dev, max_force_dev, (cudaStream_t)stream)
                : gneb_run<float>(&c->mins, c->Sf, chain_dev, vel_dev, a, energies_dev, max_force_dev, (cudaStream_t)stream);
    if (e) return fail(c, e, "GNEB failed");
    if ((rc = status_check_doubles(c, energies_dev, n_images, SITE_RELAX, (cudaStream_t)stream))) return rc;
    return status_check_doubles(c, max_force_dev, 1, SITE_RELAX, (cudaStream_t)stream);
}

int sp_gneb_path(sp_ctx *c, const void *chain_dev, int n_images, int n_interp, double *r, double *E, double *slope,
                 double *Q, double *r_interp, double *E_interp, void *stream)
{
    int rc = enter(c);
    if (rc) return rc;
    if ((rc = check_spins(c, chain_dev, "chain"))) return rc;
    if (n_images < 2) return fail(c, SP_ERR_ARG, "a chain needs at least 2 images");
    if (n_interp < 1) return fail(c, SP_ERR_ARG, "n_interp must be >= 1");
    if (!r || !E || !slope) return fail(c, SP_ERR_ARG, "NULL output");
    if ((long long)n_images * c->N >= (1LL << 31)) return fail(c, SP_ERR_ARG, "chain larger than 2^31 spins");
    if (c->h.dipole != SP_DIPOLE_NONE) return fail(c, SP_ERR_UNSUPPORTED, "path analysis with the dipole term");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<double> dist(n_images - 1);
    int e = c->prec == SP_F64 ? gneb_path_scalars<double>(&c->mins, c->Sd, chain_dev, n_images, E, dist.data(), slope, st)
                              : gneb_path_scalars<float>(&c->mins, c->Sf, chain_dev, n_images, E, dist.data(), slope, st);
    if (e) return fail(c, e, "path analysis failed");
    r[0] = 0;
    for (int v = 1; v < n_images; ++v) r[v] = r[v - 1] + dist[v - 1];
    if (r_interp && E_interp) {
        // cubic Hermite interpolation of E(r) on every segment
        for (int v = 0; v + 1 < n_images; ++v) {
            double h = dist[v];
            for (int q = 0; q < n_interp; ++q) {
                double t = (double)q / n_interp;
                double h00 = 2 * t * t * t - 3 * t * t + 1, h10 = t * t * t - 2 * t * t + t;
                double h01 = -2 * t * t * t + 3 * t * t, h11 = t * t * t - t * t;
                r_interp[v * n_interp + q] = r[v] + t * h;
                E_interp[v * n_interp + q] = h00 * E[v] + h10 * h * slope[v] + h01 * E[v + 1] + h11 * h * slope[v + 1];
            }
        }
        r_interp[(n_images - 1) * n_interp] = r[n_images - 1];
        E_interp[(n_images - 1) * n_interp] = E[n_images - 1];
    }
    if (Q) {
        size_t rb = c->prec == SP_F64 ? 32 : 16;
        if ((rc = ensure(c, c->qbuf, sizeof(double) * (size_t)n_images))) return rc;
        for (int v = 0; v < n_images; ++v) {
            rc = sp_topological_charge(c, (const char *)chain_dev + rb * (size_t)v * c->N, (double *)c->qbuf.p + v, stream);
            if (rc) return rc;
        }
        cudaError_t ce = cudaMemcpyAsync(Q, c->qbuf.p, sizeof(double) * n_images, cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) return cuda_fail(c, ce, "topological charge copy");
        for (int v = 0; v < n_images; ++v)
            if (!std::isfinite(Q[v])) return fail(c, SP_ERR_NAN, "path analysis: image %d has a non-finite charge", v);
    }
    for (int v = 0; v < n_images; ++v)
        if (!std::isfinite(E[v]) || !std::isfinite(r[v]) || !std::isfinite(slope[v]))
            return fail(c, SP_ERR_NAN, "path analysis: image %d has a non-finite energy, distance or slope", v);
    return SP_OK;
}

int sp_topological_charge(sp_ctx *c, const void *n_dev, double *Q_dev, void *stream)
{
    int rc = enter(c);
    if (rc) return rc;
    if ((rc = check_spins(c, n_dev, "spins"))) return rc;
    if (!Q_dev) return fail(c, SP_ERR_ARG, "NULL output");
    if (c->nb != 1 || c->nc[2] != 1) return fail(c, SP_ERR_UNSUPPORTED, "topological charge needs a 2D one-atom lattice");
    double cz = c->A[0][0] * c->A[1][1] - c->A[0][1] * c->A[1][0];
    if ((rc = ensure(c, c->partials, sizeof(double) * 8 * (size_t)blocks_for(c->N)))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = c->prec == SP_F64
                        ? launch_topo<double>(c->Sd, (const dq4 *)n_dev, cz < 0, (double *)c->partials.p, Q_dev, st)
                        : launch_topo<float>(c->Sf, (const float4 *)n_dev, cz < 0, (double *)c->partials.p, Q_dev, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "topological charge launch");
    return status_check_doubles(c, Q_dev, 1, SITE_SAMPLE, st);
}

int sp_minimise_batch(sp_ctx *const *ctxs, int n_sys, void *spins_dev, void *vel_dev, const long long *offsets,
                      double dt, double mass, double tol, int max_iter, int check_every, int *iters,
                      double *max_torque, void *stream)
{
    if (!ctxs || n_sys < 1 || !ctxs[0]) return SP_ERR_ARG;
    sp_ctx *c0 = ctxs[0];
    if (!offsets || !iters || !max_torque) return fail(c0, SP_ERR_ARG, "NULL batch argument");
    int rc = status_enter(c0);
    if (rc) return rc;
    if ((rc = check_spins(c0, spins_dev, "spins")) || (rc = check_spins(c0, vel_dev, "velocities"))) return rc;
    if (spins_dev == vel_dev) return fail(c0, SP_ERR_ARG, "spins and velocities must not overlap");
    if (!(dt > 0) || !(mass > 0) || !(tol >= 0) || max_iter < 0 || check_every < 1)
        return fail(c0, SP_ERR_ARG, "bad minimiser parameters");
    std::vector<std::pair<long long, long long>> spans;
    std::vector<long long> off;
    for (int k = 0; k < n_sys; ++k) {
        sp_ctx *c = ctxs[k];
        if (!c) return fail(c0, SP_ERR_ARG, "NULL context for system %d", k);
        if (!c->have_geom || !c->have_ham) return fail(c0, SP_ERR_STATE, "system %d: context not configured", k);
        if (c->prec != c0->prec) return fail(c0, SP_ERR_ARG, "system %d: precision differs from system 0", k);
        if (c->h.dipole != SP_DIPOLE_NONE) return fail(c0, SP_ERR_UNSUPPORTED, "system %d: dipole term", k);
        if (offsets[k] < 0 || offsets[k] + c->N >= (1LL << 31)) return fail(c0, SP_ERR_ARG, "system %d: bad offset", k);
        spans.push_back({offsets[k], offsets[k] + c->N});
        off.push_back(offsets[k]);
    }
    std::sort(spans.begin(), spans.end());
    for (size_t k = 1; k < spans.size(); ++k)
        if (spans[k].first < spans[k - 1].second) return fail(c0, SP_ERR_ARG, "systems overlap in the batch buffer");
    MinArgs a{dt, mass, tol, max_iter, check_every};
    int e;
    if (c0->prec == SP_F64) {
        std::vector<Stencil<double>> S;
        for (int k = 0; k < n_sys; ++k) S.push_back(ctxs[k]->Sd);
        e = vp_batch_run<double>(&c0->mins, S, off, spins_dev, vel_dev, a, iters, max_torque, (cudaStream_t)stream);
    } else {
        std::vector<Stencil<float>> S;
        for (int k = 0; k < n_sys; ++k) S.push_back(ctxs[k]->Sf);
        e = vp_batch_run<float>(&c0->mins, S, off, spins_dev, vel_dev, a, iters, max_torque, (cudaStream_t)stream);
    }
    if (e) return fail(c0, e, "batched minimisation failed");
    for (int k = 0; k < n_sys; ++k)
        if (!std::isfinite(max_torque[k]))
            return fail(c0, SP_ERR_NAN, "batched minimisation: system %d has a non-finite max torque", k);
    return SP_OK;
}

int sp_gneb_batch_step(sp_ctx *const *ctxs, int n_chains, void *chains_dev, void *vel_dev, const long long *offsets,
                       const int *n_images, const sp_gneb_params *p, int n_iter, double *energies_dev,
                       double *max_force_dev, void *stream)
{
    if (!ctxs || n_chains < 1 || !ctxs[0]) return SP_ERR_ARG;
    sp_ctx *c0 = ctxs[0];
    if (!offsets || !n_images || !p) return fail(c0, SP_ERR_ARG, "NULL batch description");
    if (!energies_dev || !max_force_dev) return fail(c0, SP_ERR_ARG, "NULL output");
    int rc = status_enter(c0);
    if (rc) return rc;
    if ((rc = check_spins(c0, chains_dev, "chains")) || (rc = check_spins(c0, vel_dev, "velocities"))) return rc;
    if (n_iter < 0 || !(p->dt > 0) || !(p->mass > 0)) return fail(c0, SP_ERR_ARG, "bad iteration parameters");
    struct Span {
        long long a, b;
    };
    std::vector<Span> spans;
    std::vector<int> M;
    std::vector<long long> off;
    for (int k = 0; k < n_chains; ++k) {
        sp_ctx *c = ctxs[k];
        if (!c) return fail(c0, SP_ERR_ARG, "NULL context for chain %d", k);
        if (!c->have_geom || !c->have_ham) return fail(c0, SP_ERR_STATE, "chain %d: context not configured", k);
        if (c->prec != c0->prec) return fail(c0, SP_ERR_ARG, "chain %d: precision differs from chain 0", k);
        if (c->h.dipole != SP_DIPOLE_NONE) return fail(c0, SP_ERR_UNSUPPORTED, "chain %d: GNEB with the dipole term", k);
        if (n_images[k] < 3) return fail(c0, SP_ERR_ARG, "chain %d: at least 3 images", k);
        if (offsets[k] < 0) return fail(c0, SP_ERR_ARG, "chain %d: negative offset", k);
        long long len = (long long)n_images[k] * c->N;
        if (offsets[k] + len >= (1LL << 31)) return fail(c0, SP_ERR_ARG, "batch larger than 2^31 records");
        spans.push_back({offsets[k], offsets[k] + len});
        M.push_back(n_images[k]);
        off.push_back(offsets[k]);
    }
    std::vector<Span> sorted = spans;
    std::sort(sorted.begin(), sorted.end(), [](const Span &x, const Span &y) { return x.a < y.a; });
    for (size_t k = 1; k < sorted.size(); ++k)
        if (sorted[k].a < sorted[k - 1].b) return fail(c0, SP_ERR_ARG, "chains overlap in the batch buffer");
    if (!(p->energy_weight >= 0 && p->energy_weight < 1)) return fail(c0, SP_ERR_ARG, "energy_weight must be in [0, 1)");
    if (p->image_types) {
        long long tot = 0;
        for (int k = 0; k < n_chains; ++k) tot += n_images[k];
        for (long long g = 0; g < tot; ++g)
            if (p->image_types[g] < SP_IMAGE_NORMAL || p->image_types[g] > SP_IMAGE_FALLING)
                return fail(c0, SP_ERR_ARG, "image %lld: unknown image type %d", g, p->image_types[g]);
    }
    GnebArgs a{p->dt, p->mass, p->k_spring, p->climbing ? 1 : 0, 0, n_iter, p->image_types, p->energy_weight};
    a.persistent = c0->gneb_persistent;
    a.wait_limit = c0->wait_limit;
    if (a.persistent && !(a.status = status_word(c0))) return SP_ERR_CUDA;
    int e;
    if (c0->prec == SP_F64) {
        std::vector<Stencil<double>> S;
        for (int k = 0; k < n_chains; ++k) S.push_back(ctxs[k]->Sd);
        e = gneb_batch_run<double>(&c0->mins, S, M, off, chains_dev, vel_dev, a, energies_dev, max_force_dev,
                                   (cudaStream_t)stream);
    } else {
        std::vector<Stencil<float>> S;
        for (int k = 0; k < n_chains; ++k) S.push_back(ctxs[k]->Sf);
        e = gneb_batch_run<float>(&c0->mins, S, M, off, chains_dev, vel_dev, a, energies_dev, max_force_dev,
                                  (cudaStream_t)stream);
    }
    if (e) return fail(c0, e, "batched GNEB failed");
    long long tot = 0;
    for (int k = 0; k < n_chains; ++k) tot += n_images[k];
    if ((rc = status_check_doubles(c0, energies_dev, (long)tot, SITE_RELAX, (cudaStream_t)stream))) return rc;
    return status_check_doubles(c0, max_force_dev, n_chains, SITE_RELAX, (cudaStream_t)stream);
}

int sp_sync_status(sp_ctx *c)
{
    if (!c) return SP_ERR_ARG;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess && dev != c->device) e = cudaSetDevice(c->device);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (dev != c->device) cudaSetDevice(dev);
    if (e != cudaSuccess) return cuda_fail(c, e, "device synchronisation");
    return status_take(c);
}

int sp_gneb_batch_autotune(sp_ctx *const *ctxs, int n_chains, const void *chains_dev, const void *vel_dev,
                           const long long *offsets, const int *n_images, const sp_gneb_params *p, int n_trial,
                           int *persistent, double *ms, void *stream)
{
    if (!ctxs || n_chains < 1 || !ctxs[0]) return SP_ERR_ARG;
    sp_ctx *c0 = ctxs[0];
    if (!offsets || !n_images || !p || !chains_dev || !vel_dev) return fail(c0, SP_ERR_ARG, "NULL batch description");
    if (n_trial < 1) return fail(c0, SP_ERR_ARG, "n_trial must be >= 1");
    long long total = 0, n_img = 0;
    for (int k = 0; k < n_chains; ++k) {
        if (!ctxs[k] || !ctxs[k]->have_geom) return fail(c0, SP_ERR_STATE, "chain %d: context not configured", k);
        total = std::max(total, offsets[k] + (long long)n_images[k] * ctxs[k]->N);
        n_img += n_images[k];
    }
    const size_t bytes = rec_bytes(c0) * (size_t)std::max(total, 1LL);
    cudaStream_t st = (cudaStream_t)stream;
    void *x = nullptr, *v = nullptr;
    double *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int keep = c0->gneb_persistent, rc = SP_OK;
    double t[2] = {0, 0};
    cudaError_t e = cudaMalloc(&x, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&v, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(double) * (size_t)(n_img + n_chains));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // each mode: a warm-up call, then n_trial iterations timed, both from
    // copies of the caller's chains and velocities
    for (int mode = 0; mode < 2 && e == cudaSuccess && rc == SP_OK; ++mode) {
        c0->gneb_persistent = mode;
        for (int pass = 0; pass < 2 && e == cudaSuccess && rc == SP_OK; ++pass) {
            e = cudaMemcpyAsync(x, chains_dev, bytes, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(v, vel_dev, bytes, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaEventRecord(e0, st);
            if (e != cudaSuccess) break;
            rc = sp_gneb_batch_step(ctxs, n_chains, x, v, offsets, n_images, p, pass ? n_trial : 2, out, out + n_img,
                                    stream);
            if (rc == SP_OK) e = cudaEventRecord(e1, st);
            if (rc == SP_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
            float f = 0;
            if (rc == SP_OK && e == cudaSuccess && pass) e = cudaEventElapsedTime(&f, e0, e1);
            t[mode] = f;
        }
    }
    c0->gneb_persistent = keep;
    if (x) cudaFree(x);
    if (v) cudaFree(v);
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(c0, e, "GNEB batch autotune");
    if ((rc = status_enter(c0))) return rc;  // a trial that timed out or met a non-finite value
    c0->gneb_persistent = t[1] < t[0] ? 1 : 0;
    if (persistent) *persistent = c0->gneb_persistent;
    if (ms) {
        ms[0] = t[0];
        ms[1] = t[1];
    }
    return SP_OK;
}

int sp_set_option(sp_ctx *c, int option, int value)
{
    if (!c) return SP_ERR_ARG;
    switch (option) {
    case SP_OPT_SMALL_PATH:
        if (value != 0 && value != 1) return fail(c, SP_ERR_ARG, "small_path takes 0 or 1");
        c->use_small = value == 1;
        return SP_OK;
    case SP_OPT_GENERIC_STENCIL:
        c->use_cubic = value == 0;
        return SP_OK;
    case SP_OPT_GENERIC_FFT:
        c->generic_fft = value != 0;
        dipole_force_generic(c->dip, c->generic_fft);
        return SP_OK;
    case SP_OPT_PLANES_PER_CTA:
        if (value < 0) return fail(c, SP_ERR_ARG, "units per CTA must be >= 0 (0: balanced)");
        c->zc = value;
        c->zc_corr = 0;  // the user's value applies to both passes
        return SP_OK;
    case SP_OPT_PLANES_PER_CTA_CORR:
        if (value < 0) return fail(c, SP_ERR_ARG, "units per CTA must be >= 0 (0: as the predictor)");
        c->zc_corr = value;
        return SP_OK;
    case SP_OPT_MC_RESIDENT:
        if (value != 0 && value != 1) return fail(c, SP_ERR_ARG, "mc_resident takes 0 or 1");
        c->use_mc_resident = value == 1;
        return SP_OK;
    case SP_OPT_CUBIC_ROWS:
    case SP_OPT_CUBIC_ROWS_CORR:
        if (value != 1 && value != 2) return fail(c, SP_ERR_ARG, "columns per thread: 1 or 2");
        if (option == SP_OPT_CUBIC_ROWS) c->rows[0] = value;
        c->rows[1] = value;
        c->zc_auto = c->zc_auto_corr = 0;
        return SP_OK;
    case SP_OPT_CUBIC_LEAN:
        if (value != 0 && value != 1) return fail(c, SP_ERR_ARG, "cubic_lean takes 0 or 1");
        c->lean = value;
        c->zc_auto = c->zc_auto_corr = 0;
        return SP_OK;
    case SP_OPT_GNEB_PERSISTENT:
        if (value != 0 && value != 1) return fail(c, SP_ERR_ARG, "gneb_persistent takes 0 or 1");
        c->gneb_persistent = value;
        return SP_OK;
    case SP_OPT_WAIT_LIMIT:
        if (value < 0) return fail(c, SP_ERR_ARG, "wait limit must be >= 0 (0: default)");
        c->wait_limit = value;
        return SP_OK;
    default:
        return fail(c, SP_ERR_ARG, "unknown option %d", option);
    }
}

int sp_autotune(sp_ctx *c, const void *n_dev, int *chosen, void *stream)
{
    int rc = ready(c);
    if (rc) return rc;
    if ((rc = check_spins(c, n_dev, "spins"))) return rc;
    if (!c->cubic || c->N == 0) {
        if (chosen) *chosen = c->zc;
        return SP_OK;
    }
    cudaStream_t st = (cudaStream_t)stream;
    return c->prec == SP_F64 ? autotune_run<double>(c, n_dev, chosen, st) : autotune_run<float>(c, n_dev, chosen, st);
}

int sp_get_option(const sp_ctx *c, int option, int *value)
{
    if (!c || !value) return SP_ERR_ARG;
    switch (option) {
    case SP_OPT_GENERIC_STENCIL:
        *value = c->use_cubic ? 0 : 1;
        return SP_OK;
    case SP_OPT_PLANES_PER_CTA:
        *value = c->zc > 0 ? c->zc : c->zc_auto;
        return SP_OK;
    case SP_OPT_HAS_CUBIC_PATH:
        *value = c->cubic ? 1 : 0;
        return SP_OK;
    case SP_OPT_GENERIC_FFT:
        *value = c->generic_fft ? 1 : 0;
        return SP_OK;
    case SP_OPT_SMALL_PATH:
        *value = c->use_small ? 1 : 0;
        return SP_OK;
    case SP_OPT_PLANES_PER_CTA_CORR:
        *value = c->zc_corr > 0 ? c->zc_corr : (c->zc > 0 ? c->zc : c->zc_auto_corr);
        return SP_OK;
    case SP_OPT_MC_RESIDENT:
        *value = c->use_mc_resident ? 1 : 0;
        return SP_OK;
    case SP_OPT_GNEB_PERSISTENT:
        *value = c->gneb_persistent;
        return SP_OK;
    case SP_OPT_CUBIC_ROWS:
        *value = cubic_rows(c, 0);
        return SP_OK;
    case SP_OPT_CUBIC_ROWS_CORR:
        *value = cubic_rows(c, 1);
        return SP_OK;
    case SP_OPT_CUBIC_LEAN:
        *value = cubic_lean_taken(c, 0) ? 1 : 0;
        return SP_OK;
    case SP_OPT_WAIT_LIMIT:
        *value = c->wait_limit;
        return SP_OK;
    case SP_OPT_SCRATCH_KIB: {
        size_t b = c->pred.bytes + c->partials.bytes + c->bdd.bytes + c->qbuf.bytes + c->rsig.bytes + c->step_ctr.bytes +
               c->lb_tab.bytes;
        *value = (int)std::min<size_t>((b + 1023) / 1024, 0x7fffffff);
        return SP_OK;
    }
    default:
        return SP_ERR_ARG;
    }
}

int sp_profile_enable(sp_ctx *c, int on)
{
    if (!c) return SP_ERR_ARG;
    if (!on && c->prof.on) {
        cudaError_t e = c->prof.drain();
        if (e != cudaSuccess) return cuda_fail(c, e, "profile drain");
    }
    c->prof.on = on != 0;
    return SP_OK;
}

int sp_profile_read(sp_ctx *c, int kind, double *total_ms, long long *launches)
{
    if (!c) return SP_ERR_ARG;
    if (kind < 0 || kind >= SP_PROF_KINDS || !total_ms || !launches) return fail(c, SP_ERR_ARG, "bad profile query");
    cudaError_t e = c->prof.drain();
    if (e != cudaSuccess) return cuda_fail(c, e, "profile drain");
    *total_ms = c->prof.ms[kind];
    *launches = c->prof.count[kind];
    c->prof.ms[kind] = 0;
    c->prof.count[kind] = 0;
    return SP_OK;
}

}  // extern "C"
