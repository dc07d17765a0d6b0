// htst.cu -- harmonic transition-state theory (Sec. "Harmonic Transition-State
// Theory" and the appendix on the curved manifold): the full spectrum of the
// covariant Hessian and the rate prefactor of a transition from a minimum
// over a first-order saddle point.  sp_hessian_spectrum, sp_htst.
//
// Rate (Sec. HTST):  Gamma = v / (2 pi) Omega_0 exp(-dE / kB T) with
//   Omega_0 = sqrt(prod' lambda^M / prod' lambda^S)            (positive eigenvalues)
//   v       = sqrt(2 pi kB T)^(N0^M - N0^S) V^S / V^M sqrt(sum'_i a_i^2 / lambda^S_i)
// a_i the first row of the dynamical matrix in the Hessian's eigenbasis: the
// velocity along the unstable mode e_1 that a displacement along mode e_i
// causes.  The linearised precession at a stationary point is
//   d(dn_i)/dt = (gamma / mu_i) n_i x (H dn)_i
// (the Landau-Lifshitz equation without damping, the dynamics of the
// harmonic rate), so in the eigenbasis a_i = (e_1 . W e_i) lambda_i with
// W dn|_i = (gamma / mu_i) n_i x dn_i.  W is antisymmetric per spin, so
// e_1 . W e_1 = 0 and
//   sum_{lambda_i > 0} a_i^2 / lambda_i = u . H u - sum_{zero modes} lambda_z (u . e_z)^2,
//   u_i = (gamma / mu_i) n_i x e_1,i
// -- one Hessian-vector product with the unstable mode turned by 90 degrees
// per spin replaces the sum over all 2N modes (the zero modes' share is
// below zero_tol |u|^2 and is not subtracted).
//
// Spectrum: Lanczos on the 2N-dimensional tangent space with classical
// Gram-Schmidt reorthogonalisation done twice against every stored vector;
// where the Krylov space closes (an invariant subspace: the residual falls to
// the rounding level) the iteration restarts from a new pseudo-random tangent
// field orthogonalised against all vectors so far, so that degenerate
// eigenvalues are found with their multiplicity.  After 2N steps the
// tridiagonal matrix (block diagonal at the restarts) is similar to the
// Hessian; its eigenvalues come from bisection on Sturm counts, one thread
// per eigenvalue.  FP64 contexts only.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ctx.h"

struct HtstScratch {
    DevBuf Q, w, u, Hu, part, upd, dots, coef, tri, eig, epart;
};

namespace {

constexpr int kB = 256;
constexpr int kDotChunk = 1024;  // spins per block of the Gram-Schmidt dot products
constexpr int kAxpyChunk = 64;   // basis vectors per block of the Gram-Schmidt update

int grow(DevBuf &b, size_t bytes)
{
    if (b.p && b.bytes >= bytes) return 0;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) return SP_ERR_CUDA;
    b.bytes = bytes;
    return 0;
}

// part[sb * m + k] = sum over the spins of block row sb of a_i . q_k,i (k < m);
// warp w of block x takes basis vector k = 8 x + w.
__global__ void __launch_bounds__(kB) k_gs_dots(int N, const dq4 *__restrict__ a, const dq4 *__restrict__ Q, int m,
                                                double *__restrict__ part)
{
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int k = blockIdx.x * (kB / 32) + warp;
    if (k >= m) return;
    int i0 = blockIdx.y * kDotChunk, i1 = min(N, i0 + kDotChunk);
    const dq4 *q = Q + (size_t)k * N;
    double s = 0;
    for (int i = i0 + lane; i < i1; i += 32) s += ddot(ld(a, i), ld(q, i));
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) part[(size_t)blockIdx.y * m + k] = s;
}

// out[k] = sum over block rows (fixed order)
__global__ void k_gs_sum(const double *__restrict__ part, int nsb, int m, double *__restrict__ out)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    double s = 0;
    for (int b = 0; b < nsb; ++b) s += part[(size_t)b * m + k];
    out[k] = s;
}

// P[kc][i] = sum over the basis vectors k of chunk kc of c_k q_k,i
__global__ void __launch_bounds__(kB) k_gs_axpy(int N, const dq4 *__restrict__ Q, const double *__restrict__ c, int m,
                                                dq4 *__restrict__ P)
{
    int i = blockIdx.x * kB + threadIdx.x;
    if (i >= N) return;
    int k0 = blockIdx.y * kAxpyChunk, k1 = min(m, k0 + kAxpyChunk);
    v3<double> s = mk(0.0, 0.0, 0.0);
    for (int k = k0; k < k1; ++k) s = axpy(c[k], ld(Q + (size_t)k * N, i), s);
    st(P + (size_t)blockIdx.y * N, i, s);
}

// w_i <- P_{n_i}(a w_i - sum_kc P[kc][i])  (fixed order over the chunks)
__global__ void __launch_bounds__(kB) k_gs_apply(int N, const dq4 *__restrict__ n, dq4 *__restrict__ w, double a,
                                                 const dq4 *__restrict__ P, int nkc)
{
    int i = blockIdx.x * kB + threadIdx.x;
    if (i >= N) return;
    v3<double> x = a * ld(w, i);
    for (int kc = 0; kc < nkc; ++kc) x = x - ld(P + (size_t)kc * N, i);
    v3<double> ni = ld(n, i);
    st(w, i, x - dot(x, ni) * ni);
}

// out = s * v projected onto the tangent planes
__global__ void k_scale_project(int N, const dq4 *__restrict__ n, const dq4 *__restrict__ v, double s,
                                dq4 *__restrict__ out)
{
    int i = blockIdx.x * kB + threadIdx.x;
    if (i >= N) return;
    v3<double> x = s * ld(v, i), ni = ld(n, i);
    st(out, i, x - dot(x, ni) * ni);
}

// a pseudo-random tangent field (integer hash of index and salt)
__global__ void k_seed(int N, const dq4 *__restrict__ n, dq4 *__restrict__ v, uint32_t salt)
{
    int i = blockIdx.x * kB + threadIdx.x;
    if (i >= N) return;
    double h[3];
    for (int k = 0; k < 3; ++k) {
        uint32_t z = (uint32_t)i * 2654435761u + (uint32_t)k * 40503u + salt * 2246822519u + 12345u;
        z ^= z >> 15;
        z *= 2246822519u;
        z ^= z >> 13;
        z *= 3266489917u;
        z ^= z >> 16;
        h[k] = (double)z * 2.3283064365386963e-10 - 0.5;
    }
    v3<double> x = mk(h[0], h[1], h[2]), ni = ld(n, i);
    st(v, i, x - dot(x, ni) * ni);
}

// u_i = (gamma / mu_i) n_i x e_i: the unstable mode turned by the precession
__global__ void k_precess(const __grid_constant__ Stencil<double> S, const dq4 *__restrict__ n,
                          const dq4 *__restrict__ e, dq4 *__restrict__ u)
{
    int i = blockIdx.x * kB + threadIdx.x;
    if (i >= S.N) return;
    int b, c0, c1, c2;
    decode_site(S, i, b, c0, c1, c2);
    st(u, i, (kGamma / S.mu[b]) * cross(ld(n, i), ld(e, i)));
}

// Eigenvalue number k (ascending) of the symmetric tridiagonal matrix with
// diagonal a[0..m) and squared couplings b2[0..m-1), by bisection of
// [lo, hi] on the Sturm count (the number of negative pivots of T - x I).
__global__ void k_tri_bisect(const double *__restrict__ a, const double *__restrict__ b2, int m, double lo,
                             double hi, double pivmin, double *__restrict__ eig)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    double l = lo, h = hi;
    for (int it = 0; it < 128; ++it) {
        double x = 0.5 * (l + h);
        if (!(x > l && x < h)) break;  // the interval cannot shrink further
        int cnt = 0;
        double d = 1.0;
        for (int i = 0; i < m; ++i) {
            d = a[i] - x - (i ? b2[i - 1] / d : 0.0);
            if (fabs(d) < pivmin) d = -pivmin;
            cnt += d < 0;
        }
        if (cnt > k)
            h = x;
        else
            l = x;
    }
    eig[k] = 0.5 * (l + h);
}

struct Spec {
    const Stencil<double> &S;
    HtstScratch &h;
    cudaStream_t st;
    int N;
    unsigned nb;

    dq4 *q(int k) { return (dq4 *)h.Q.p + (size_t)k * N; }

    // device dots[k] = a . q_k (k < m), from the vectors at Qb
    void dots(const dq4 *a, const dq4 *Qb, int m)
    {
        int nsb = (N + kDotChunk - 1) / kDotChunk;
        k_gs_dots<<<dim3((m + kB / 32 - 1) / (kB / 32), nsb), kB, 0, st>>>(N, a, Qb, m, (double *)h.part.p);
        k_gs_sum<<<(m + 127) / 128, 128, 0, st>>>((const double *)h.part.p, nsb, m, (double *)h.dots.p);
    }
    // w <- P(a w - sum_k dots[k] q_k), k < m
    void update(const dq4 *n, dq4 *w, double a, int m)
    {
        int nkc = (m + kAxpyChunk - 1) / kAxpyChunk;
        if (nkc > 0)
            k_gs_axpy<<<dim3(nb, nkc), kB, 0, st>>>(N, (const dq4 *)h.Q.p, (const double *)h.dots.p, m, (dq4 *)h.upd.p);
        k_gs_apply<<<nb, kB, 0, st>>>(N, n, w, a, (const dq4 *)h.upd.p, nkc);
    }
    // w <- w minus its components along q_0..q_{m-1}, twice; *first (may be
    // null) receives the first pass's coefficient of q_{m-1}; *nrm2 = |w|^2
    int orthogonalise(const dq4 *n, dq4 *w, int m, double *first, double *nrm2)
    {
        double host[2] = {0, 0};
        for (int pass = 0; pass < 2 && m > 0; ++pass) {
            dots(w, q(0), m);
            if (pass == 0 && first &&
                cudaMemcpyAsync(&host[0], (double *)h.dots.p + (m - 1), sizeof(double), cudaMemcpyDeviceToHost, st) !=
                    cudaSuccess)
                return SP_ERR_CUDA;
            update(n, w, 1.0, m);
        }
        dots(w, w, 1);
        if (cudaMemcpyAsync(&host[1], h.dots.p, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return SP_ERR_CUDA;
        if (first) *first = host[0];
        *nrm2 = host[1];
        return cudaGetLastError() == cudaSuccess ? 0 : SP_ERR_CUDA;
    }

    // Lanczos over the whole tangent space (2N steps, restarts at invariant
    // subspaces): diagonal alpha, couplings beta (0 at a restart).
    int tridiagonal(const dq4 *n, std::vector<double> &alpha, std::vector<double> &beta)
    {
        const int M = 2 * N;
        dq4 *w = (dq4 *)h.w.p;
        uint32_t salt = 1;
        double nrm2 = 0;
        k_seed<<<nb, kB, 0, st>>>(N, n, q(0), salt);
        int rc = orthogonalise(n, q(0), 0, nullptr, &nrm2);
        if (rc) return rc;
        if (!(nrm2 > 0)) return SP_ERR_STATE;
        k_scale_project<<<nb, kB, 0, st>>>(N, n, q(0), 1.0 / sqrt(nrm2), q(0));
        double tnorm = 0;
        for (int k = 0; k < M; ++k) {
            launch_hvp<double>(S, n, q(k), w, st);
            double a, b2;
            if ((rc = orthogonalise(n, w, k + 1, &a, &b2))) return rc;
            alpha.push_back(a);
            double b = sqrt(b2);
            tnorm = std::max(tnorm, fabs(a) + b + (k ? beta[k - 1] : 0.0));
            if (k == M - 1) break;
            if (b > 1e-12 * tnorm) {
                beta.push_back(b);
                k_scale_project<<<nb, kB, 0, st>>>(N, n, w, 1.0 / b, q(k + 1));
                continue;
            }
            // the Krylov space closed: restart from a fresh direction
            beta.push_back(0.0);
            bool ok = false;
            for (int tries = 0; tries < 8 && !ok; ++tries) {
                k_seed<<<nb, kB, 0, st>>>(N, n, q(k + 1), ++salt);
                if ((rc = orthogonalise(n, q(k + 1), k + 1, nullptr, &nrm2))) return rc;
                if (nrm2 > 1e-20) {
                    k_scale_project<<<nb, kB, 0, st>>>(N, n, q(k + 1), 1.0 / sqrt(nrm2), q(k + 1));
                    ok = true;
                }
            }
            if (!ok) return SP_ERR_STATE;
        }
        return cudaGetLastError() == cudaSuccess ? 0 : SP_ERR_CUDA;
    }
};

// Eigenvalues of the tridiagonal (alpha, beta) on the device, ascending.
int tri_eigenvalues(HtstScratch &h, const std::vector<double> &alpha, const std::vector<double> &beta,
                    std::vector<double> &eig, cudaStream_t st)
{
    int m = (int)alpha.size();
    std::vector<double> host(2 * (size_t)m, 0.0);
    double lo = 1e300, hi = -1e300, bmax = 0;
    for (int i = 0; i < m; ++i) {
        double r = (i ? fabs(beta[i - 1]) : 0.0) + (i + 1 < m ? fabs(beta[i]) : 0.0);
        lo = std::min(lo, alpha[i] - r);
        hi = std::max(hi, alpha[i] + r);
        host[i] = alpha[i];
        if (i + 1 < m) {
            host[m + i] = beta[i] * beta[i];
            bmax = std::max(bmax, fabs(beta[i]));
        }
    }
    double span = std::max(hi - lo, std::max(fabs(lo), fabs(hi))) + 1e-300;
    lo -= 1e-12 * span;
    hi += 1e-12 * span;
    double pivmin = std::max(1e-300, 1e-290 * std::max(1.0, bmax * bmax));
    eig.assign(m, 0.0);
    double *a = (double *)h.tri.p, *b2 = a + m;
    if (cudaMemcpyAsync(a, host.data(), sizeof(double) * 2 * m, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return SP_ERR_CUDA;
    k_tri_bisect<<<(m + 127) / 128, 128, 0, st>>>(a, b2, m, lo, hi, pivmin, (double *)h.eig.p);
    if (cudaMemcpyAsync(eig.data(), h.eig.p, sizeof(double) * m, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SP_ERR_CUDA;
    std::sort(eig.begin(), eig.end());
    return 0;
}

// Eigenvector y (unit) of the tridiagonal for the eigenvalue lam, by inverse
// iteration with a shift just below lam (tridiagonal LU with partial
// pivoting).
void tri_eigenvector(const std::vector<double> &alpha, const std::vector<double> &beta, double lam,
                     std::vector<double> &y)
{
    int m = (int)alpha.size();
    double scale = 0;
    for (int i = 0; i < m; ++i) scale = std::max(scale, fabs(alpha[i]) + (i < m - 1 ? fabs(beta[i]) : 0.0));
    double sigma = lam - 1e-10 * std::max(scale, 1e-300);
    y.assign(m, 0.0);
    for (int i = 0; i < m; ++i) y[i] = 1.0 + 0.1 * std::sin(1.0 + i);  // a generic start
    // LU of T - sigma I with row interchanges: rows hold (l, d, u, u2)
    std::vector<double> dl(m, 0), d(m), du(m, 0), du2(m, 0);
    std::vector<int> piv(m, 0);
    for (int i = 0; i < m; ++i) {
        d[i] = alpha[i] - sigma;
        if (i + 1 < m) du[i] = beta[i], dl[i + 1] = beta[i];
    }
    for (int i = 0; i + 1 < m; ++i) {
        if (fabs(d[i]) >= fabs(dl[i + 1])) {
            double f = d[i] != 0 ? dl[i + 1] / d[i] : 0.0;
            dl[i + 1] = f;
            d[i + 1] -= f * du[i];
            piv[i] = 0;
        } else {
            double f = d[i] / dl[i + 1];
            d[i] = dl[i + 1];
            dl[i + 1] = f;
            double t = du[i];
            du[i] = d[i + 1];
            d[i + 1] = t - f * d[i + 1];
            if (i + 2 < m) {
                du2[i] = du[i + 1];
                du[i + 1] = -f * du[i + 1];
            }
            piv[i] = 1;
        }
    }
    const double tiny = 1e-300;
    for (int it = 0; it < 4; ++it) {
        // forward: apply the interchanges and L
        for (int i = 0; i + 1 < m; ++i) {
            if (piv[i]) std::swap(y[i], y[i + 1]);
            y[i + 1] -= dl[i + 1] * y[i];
        }
        // back substitution with U
        for (int i = m - 1; i >= 0; --i) {
            double s = y[i];
            if (i + 1 < m) s -= du[i] * y[i + 1];
            if (i + 2 < m) s -= du2[i] * y[i + 2];
            y[i] = s / (fabs(d[i]) > tiny ? d[i] : tiny);
        }
        double nr = 0;
        for (double v : y) nr += v * v;
        nr = sqrt(nr);
        for (double &v : y) v /= nr;
    }
}

int setup(sp_ctx *c)
{
    if (!c->htst) c->htst = new HtstScratch;
    HtstScratch &h = *c->htst;
    size_t N = (size_t)c->N, M = 2 * N, rec = sizeof(dq4) * N;
    size_t nsb = (N + kDotChunk - 1) / kDotChunk, nkc = (M + 1 + kAxpyChunk - 1) / kAxpyChunk;
    if (grow(h.Q, rec * (M + 1)) || grow(h.w, rec) || grow(h.u, rec) || grow(h.Hu, rec) ||
        grow(h.part, sizeof(double) * nsb * (M + 1)) || grow(h.upd, rec * nkc) || grow(h.dots, sizeof(double) * (M + 1)) ||
        grow(h.coef, sizeof(double) * (M + 1)) || grow(h.tri, sizeof(double) * 2 * M) || grow(h.eig, sizeof(double) * M) ||
        grow(h.epart, sizeof(double) * (16 + 8 * ((N + kBlock - 1) / kBlock))))
        return SP_ERR_CUDA;
    return 0;
}

int spectrum_run(sp_ctx *c, const void *n, std::vector<double> &alpha, std::vector<double> &beta,
                 std::vector<double> &eig, cudaStream_t st)
{
    int rc = setup(c);
    if (rc) return rc;
    Spec sp{c->Sd, *c->htst, st, c->N, (unsigned)((c->N + kB - 1) / kB)};
    alpha.clear();
    beta.clear();
    if ((rc = sp.tridiagonal((const dq4 *)n, alpha, beta))) return rc;
    return tri_eigenvalues(*c->htst, alpha, beta, eig, st);
}

int hfail2(sp_ctx *c, int code, const char *msg)
{
    c->err = msg;
    return code;
}

int check(sp_ctx *c)
{
    if (!c) return SP_ERR_ARG;
    if (!c->have_geom || !c->have_ham) return hfail2(c, SP_ERR_STATE, "context not configured");
    if (c->prec != SP_F64) return hfail2(c, SP_ERR_UNSUPPORTED, "the Hessian spectrum needs an SP_F64 context");
    if (c->h.dipole != SP_DIPOLE_NONE) return hfail2(c, SP_ERR_UNSUPPORTED, "Hessian with the dipole term");
    if (c->N < 1 || c->N > SP_HTST_MAX_SPINS)
        return hfail2(c, SP_ERR_ARG, "the Hessian spectrum takes 1..SP_HTST_MAX_SPINS (2048) spins");
    return status_enter(c);
}

bool rec_aligned(const void *p) { return p && ((uintptr_t)p % 32) == 0; }

}  // namespace

void htst_scratch_destroy(HtstScratch *h)
{
    if (!h) return;
    DevBuf *bufs[] = {&h->Q, &h->w, &h->u, &h->Hu, &h->part, &h->upd, &h->dots, &h->coef, &h->tri, &h->eig, &h->epart};
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    delete h;
}

extern "C" {

int sp_hessian_spectrum(sp_ctx *c, const void *n_dev, double *eig, void *stream)
{
    int rc = check(c);
    if (rc) return rc;
    if (!rec_aligned(n_dev) || !eig) return hfail2(c, SP_ERR_ARG, "NULL or misaligned argument");
    std::vector<double> alpha, beta, ev;
    rc = spectrum_run(c, n_dev, alpha, beta, ev, (cudaStream_t)stream);
    if (rc) return hfail2(c, rc, "Hessian spectrum failed");
    std::copy(ev.begin(), ev.end(), eig);
    for (double x : ev)
        if (!std::isfinite(x)) return hfail2(c, SP_ERR_NAN, "Hessian spectrum: a non-finite eigenvalue");
    return SP_OK;
}

int sp_htst(sp_ctx *c, const void *n_min_dev, const void *n_sad_dev, const sp_htst_params *p, sp_htst_result *out,
            void *stream)
{
    int rc = check(c);
    if (rc) return rc;
    if (!rec_aligned(n_min_dev) || !rec_aligned(n_sad_dev) || !p || !out)
        return hfail2(c, SP_ERR_ARG, "NULL or misaligned argument");
    if (!(p->zero_tol >= 0) || !(p->V_min > 0) || !(p->V_sad > 0))
        return hfail2(c, SP_ERR_ARG, "zero_tol >= 0 and positive zero-mode volumes required");
    cudaStream_t st = (cudaStream_t)stream;
    const int N = c->N;
    const unsigned nb = (unsigned)((N + kB - 1) / kB);
    sp_htst_result r{};
    // energies of both states (FP64 sums)
    if ((rc = setup(c))) return hfail2(c, rc, "HTST scratch");
    HtstScratch &h = *c->htst;
    {
        double e[2][6];
        double *E = (double *)h.epart.p, *part = E + 16;
        cudaError_t ce = launch_energy<double>(c->Sd, (const dq4 *)n_min_dev, nullptr, part, E, nullptr, st);
        if (ce == cudaSuccess) ce = launch_energy<double>(c->Sd, (const dq4 *)n_sad_dev, nullptr, part, E + 8, nullptr, st);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(e[0], E, 6 * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(e[1], E + 8, 6 * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) return hfail2(c, SP_ERR_CUDA, "HTST energies");
        r.E_min = e[0][0];
        r.E_sad = e[1][0];
        r.dE = r.E_sad - r.E_min;
    }
    // spectra: log det' and the mode counts
    std::vector<double> alpha, beta, ev;
    double logdet[2];
    int nzero[2], nneg[2];
    const void *states[2] = {n_min_dev, n_sad_dev};
    for (int s = 0; s < 2; ++s) {
        if ((rc = spectrum_run(c, states[s], alpha, beta, ev, st))) return hfail2(c, rc, "Hessian spectrum failed");
        logdet[s] = 0;
        nzero[s] = nneg[s] = 0;
        for (double x : ev) {
            if (!std::isfinite(x)) return hfail2(c, SP_ERR_NAN, "HTST: a non-finite eigenvalue");
            if (x > p->zero_tol)
                logdet[s] += std::log(x);
            else if (x < -p->zero_tol)
                ++nneg[s];
            else
                ++nzero[s];
        }
        if (s == 1) r.lambda_unstable = ev[0];
    }
    // the saddle's unstable mode: Ritz vector of the lowest eigenvalue from
    // the saddle's Lanczos basis (still in h.Q), then u = W e_1 and u . H u
    std::vector<double> y;
    tri_eigenvector(alpha, beta, r.lambda_unstable, y);
    const int m = (int)alpha.size();
    Spec sp{c->Sd, h, st, N, nb};
    dq4 *e1 = (dq4 *)h.w.p, *u = (dq4 *)h.u.p, *Hu = (dq4 *)h.Hu.p;
    if (cudaMemsetAsync(e1, 0, sizeof(dq4) * (size_t)N, st) != cudaSuccess ||
        cudaMemcpyAsync(h.dots.p, y.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return hfail2(c, SP_ERR_CUDA, "HTST mode");
    sp.update((const dq4 *)n_sad_dev, e1, 0.0, m);  // e1 = -sum y_k q_k (the sign is immaterial)
    k_precess<<<nb, kB, 0, st>>>(c->Sd, (const dq4 *)n_sad_dev, e1, u);
    launch_hvp<double>(c->Sd, (const dq4 *)n_sad_dev, u, Hu, st);
    sp.dots(u, Hu, 1);
    double uHu = 0;
    if (cudaMemcpyAsync(&uHu, h.dots.p, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return hfail2(c, SP_ERR_CUDA, "HTST velocity");
    r.log_det_min = logdet[0];
    r.log_det_sad = logdet[1];
    r.n_zero_min = nzero[0];
    r.n_zero_sad = nzero[1];
    r.n_neg_min = nneg[0];
    r.n_neg_sad = nneg[1];
    r.omega0 = std::exp(0.5 * (logdet[0] - logdet[1]));
    r.v = std::sqrt(std::max(0.0, uHu));
    r.prefactor = r.v / (2.0 * M_PI) * r.omega0 * p->V_sad / p->V_min;
    *out = r;
    if (!std::isfinite(r.omega0) || !std::isfinite(r.v) || !std::isfinite(r.dE))
        return hfail2(c, SP_ERR_NAN, "HTST: a non-finite result");
    return SP_OK;
}

}  // extern "C"
