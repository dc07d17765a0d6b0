// hessian.cu -- covariant Hessian on the spin manifold, its lowest mode and
// minimum mode following (Sec. MMF and the appendix on the manifold of
// constant-length spins): sp_hessian_apply, sp_lowest_mode, sp_mmf.
//
// Hessian-vector product, per spin i, for a tangent field w:
//   H w|_i = P_i (Hbar w)_i - (n_i . grad_i Hbar) w_i
// where Hbar are the second derivatives of the Hamiltonian continued to
// R^{3N}: (Hbar w)_i = -(sum_j J_ij w_j + w_j x D_ij + 2 K (Khat.w_i) Khat),
// i.e. minus the local field evaluated on w without the Zeeman term, and
// grad_i Hbar = -B_i.  The lowest mode comes from Lanczos with full
// reorthogonalisation (kernels for the operator, dot products and updates;
// the small tridiagonal eigenproblem on the host by cyclic Jacobi).  MMF
// moves with the effective force F - 2 (F.l) l (-(F.l) l where the lowest
// eigenvalue is not negative) by the velocity projection of Appendix D.
#include <algorithm>
#include <cmath>
#include <initializer_list>
#include <vector>

#include "ctx.h"

struct HessScratch {
    DevBuf Q, w, F, Fe, F2, Fe2, y, mode2, part, dots, coef;
    int m = 0;
};

namespace {

constexpr int kHB = 256;
constexpr int kMaxKrylov = 256;

int grow_h(DevBuf &b, size_t bytes)
{
    if (b.p && b.bytes >= bytes) return 0;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) return SP_ERR_CUDA;
    b.bytes = bytes;
    return 0;
}

// H v with v projected onto the tangent planes on the fly: one pass over
// the stencil loads n_j and v_j together and accumulates the field of n and
// the field of the projected w without the Zeeman term.
template <typename T>
__global__ void __launch_bounds__(kHB) k_hvp(const __grid_constant__ Stencil<T> S, const rec_t<T> *__restrict__ n,
                                             const rec_t<T> *__restrict__ v, rec_t<T> *__restrict__ out,
                                             unsigned *status = nullptr)
{
    allow_dependents();
    wait_prerequisite();  // n and v may come from the kernels before
    int i = blockIdx.x * kHB + threadIdx.x;
    if (i >= S.N) return;
    int b, c0, c1, c2;
    decode_site(S, i, b, c0, c1, c2);
    const bool inner = interior_site(S, c0, c1, c2);
    v3<T> ni = ld(n, i), vi = ld(v, i);
    v3<T> wi = vi - dot(vi, ni) * ni;
    v3<T> kh = mk(S.Kh[b][0], S.Kh[b][1], S.Kh[b][2]);
    v3<T> Bn = mk(S.Bz[b][0], S.Bz[b][1], S.Bz[b][2]) + (T(2) * S.K[b] * dot(kh, ni)) * kh;
    v3<T> Lw = (T(2) * S.K[b] * dot(kh, wi)) * kh;
    for (int q = S.off[b]; q < S.off[b + 1]; ++q) {
        const NbrEntry<T> &E = S.e[q];
        int j = nbr_index(S, E, i, inner, c0, c1, c2);
        if (j < 0) continue;
        v3<T> nj = ld(n, j), vj = ld(v, j);
        v3<T> wj = vj - dot(vj, nj) * nj;
        v3<T> D = mk(E.Dx, E.Dy, E.Dz);
        Bn = axpy(E.J, nj, Bn + cross(nj, D));
        Lw = axpy(E.J, wj, Lw + cross(wj, D));
    }
    // P (Hbar w) with Hbar w = -Lw, plus the Weingarten term (n . B) w
    v3<T> r3 = (dot(Lw, ni) * ni - Lw) + dot(ni, Bn) * wi;
    st(out, i, r3);
    // status != null: a non-finite product sets the Hessian bit of the
    // context's status word (the check of the output, without a second pass)
    if (status) {
        const bool bad = !(isfinite(r3.x) && isfinite(r3.y) && isfinite(r3.z));
        const unsigned act = __activemask();
        if (__any_sync(act, bad) && (threadIdx.x & 31) == __ffs(act) - 1) atomicOr_system(status, (unsigned)SITE_HESSIAN);
    }
}

// out = v projected per spin onto the tangent plane of n
template <typename T>
__global__ void k_project(int N, const rec_t<T> *__restrict__ n, const rec_t<T> *__restrict__ v, rec_t<T> *__restrict__ out)
{
    int i = blockIdx.x * kHB + threadIdx.x;
    if (i >= N) return;
    v3<T> ni = ld(n, i), vi = ld(v, i);
    st(out, i, vi - dot(vi, ni) * ni);
}

// part[blk][k] = sum over the block's spins of a . q_k, k < m (q_k = Q + k N)
template <typename T>
__global__ void __launch_bounds__(kHB) k_dots(int N, const rec_t<T> *__restrict__ a, const rec_t<T> *__restrict__ Q, int m,
                                              double *__restrict__ part)
{
    __shared__ double sh[kHB / 32];
    int i = blockIdx.x * kHB + threadIdx.x;
    v3<T> ai = i < N ? ld(a, i) : mk(T(0), T(0), T(0));
    for (int k = 0; k < m; ++k) {
        double v = 0;
        if (i < N) v = ddot(ai, ld(Q + (size_t)k * N, i));
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0;
            for (int w = 0; w < kHB / 32; ++w) s += sh[w];
            part[(size_t)blockIdx.x * m + k] = s;
        }
        __syncthreads();
    }
}

__global__ void k_dots_final(const double *__restrict__ part, int nblk, int m, double *__restrict__ out)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    double s = 0;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)b * m + k];
    out[k] = s;
}

// w = a w + sum_k c_k q_k (c on the device), then per-spin projection onto T_n
template <typename T>
__global__ void k_combine(int N, const rec_t<T> *__restrict__ n, rec_t<T> *__restrict__ w, double a,
                          const rec_t<T> *__restrict__ Q, const double *__restrict__ c, int m)
{
    int i = blockIdx.x * kHB + threadIdx.x;
    if (i >= N) return;
    v3<T> wi = (T)a * ld(w, i);
    for (int k = 0; k < m; ++k) wi = axpy((T)c[k], ld(Q + (size_t)k * N, i), wi);
    v3<T> ni = ld(n, i);
    st(w, i, wi - dot(wi, ni) * ni);
}

// F = B - (B.n) n
template <typename T>
__global__ void __launch_bounds__(kHB) k_force(const __grid_constant__ Stencil<T> S, const rec_t<T> *__restrict__ n,
                                               rec_t<T> *__restrict__ F)
{
    int i = blockIdx.x * kHB + threadIdx.x;
    if (i >= S.N) return;
    int b;
    v3<T> ni = ld(n, i);
    v3<T> B = local_field(S, n, i, ni, b);
    st(F, i, B - dot(B, ni) * ni);
}

// y = normalise(x + dt v + dt^2/(2m) Fe)
template <typename T>
__global__ void k_mmf_move(int N, const rec_t<T> *__restrict__ x, const rec_t<T> *__restrict__ v,
                           const rec_t<T> *__restrict__ Fe, rec_t<T> *__restrict__ y, double dt, double dt2_2m)
{
    int i = blockIdx.x * kHB + threadIdx.x;
    if (i >= N) return;
    st(y, i, normalised(axpy((T)dt2_2m, ld(Fe, i), axpy((T)dt, ld(v, i), ld(x, i)))));
}

// v += dt/(2m) (Fe + Fe2)
template <typename T>
__global__ void k_mmf_vel(int N, rec_t<T> *__restrict__ v, const rec_t<T> *__restrict__ Fe,
                          const rec_t<T> *__restrict__ Fe2, double dth_m)
{
    int i = blockIdx.x * kHB + threadIdx.x;
    if (i >= N) return;
    st(v, i, axpy((T)dth_m, ld(Fe, i) + ld(Fe2, i), ld(v, i)));
}

// out = a u + b z (plain records)
template <typename T>
__global__ void k_lin(int N, rec_t<T> *__restrict__ out, double a, const rec_t<T> *__restrict__ u, double b,
                      const rec_t<T> *__restrict__ z)
{
    int i = blockIdx.x * kHB + threadIdx.x;
    if (i >= N) return;
    st(out, i, axpy((T)b, ld(z, i), (T)a * ld(u, i)));
}

// max_i |F_i|
template <typename T>
__global__ void k_maxnorm(int N, const rec_t<T> *__restrict__ F, double *__restrict__ part)
{
    __shared__ double sh[kHB / 32];
    int i = blockIdx.x * kHB + threadIdx.x;
    double v = i < N ? sqrt(ddot(ld(F, i), ld(F, i))) : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < kHB / 32; ++w) s = fmax(s, sh[w]);
        part[blockIdx.x] = s;
    }
}

// Eigen-decomposition of a small symmetric matrix (row-major m x m) by the
// cyclic Jacobi method: rotations annihilate off-diagonal entries until
// their norm is below 1e-15 of the matrix norm.  Eigenvalues in d, vectors
// in the columns of V.
void jacobi_eigen(std::vector<double> A, int m, std::vector<double> &d, std::vector<double> &V)
{
    V.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) V[(size_t)i * m + i] = 1.0;
    double norm = 0;
    for (double a : A) norm += a * a;
    norm = sqrt(norm);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0;
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) off += A[(size_t)p * m + q] * A[(size_t)p * m + q];
        if (sqrt(off) <= 1e-15 * norm || norm == 0) break;
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) {
                double apq = A[(size_t)p * m + q];
                if (apq == 0) continue;
                double app = A[(size_t)p * m + p], aqq = A[(size_t)q * m + q];
                double theta = (aqq - app) / (2 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1));
                double c = 1 / sqrt(t * t + 1), s = t * c;
                for (int k = 0; k < m; ++k) {  // A <- A R (columns p, q)
                    double akp = A[(size_t)k * m + p], akq = A[(size_t)k * m + q];
                    A[(size_t)k * m + p] = c * akp - s * akq;
                    A[(size_t)k * m + q] = s * akp + c * akq;
                }
                for (int k = 0; k < m; ++k) {  // A <- R^T A (rows p, q)
                    double apk = A[(size_t)p * m + k], aqk = A[(size_t)q * m + k];
                    A[(size_t)p * m + k] = c * apk - s * aqk;
                    A[(size_t)q * m + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < m; ++k) {
                    double vkp = V[(size_t)k * m + p], vkq = V[(size_t)k * m + q];
                    V[(size_t)k * m + p] = c * vkp - s * vkq;
                    V[(size_t)k * m + q] = s * vkp + c * vkq;
                }
            }
    }
    d.resize(m);
    for (int i = 0; i < m; ++i) d[i] = A[(size_t)i * m + i];
}

unsigned hblocks(long long n) { return (unsigned)((n + kHB - 1) / kHB); }

template <typename T>
struct Ops {
    const Stencil<T> &S;
    HessScratch &h;
    cudaStream_t st;
    int N;
    unsigned nb;

    rec_t<T> *q(int k) { return (rec_t<T> *)h.Q.p + (size_t)k * N; }

    // dots[k] = a . q_k, k < m, copied to the host
    int dots(const rec_t<T> *a, const rec_t<T> *Qb, int m, double *host)
    {
        k_dots<T><<<nb, kHB, 0, st>>>(N, a, Qb, m, (double *)h.part.p);
        k_dots_final<<<(m + 127) / 128, 128, 0, st>>>((double *)h.part.p, (int)nb, m, (double *)h.dots.p);
        if (cudaMemcpyAsync(host, h.dots.p, sizeof(double) * m, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return SP_ERR_CUDA;
        return 0;
    }

    // w = a w + sum_k c_k q_k (c from the host), projected
    int combine(const rec_t<T> *n, rec_t<T> *w, double a, const rec_t<T> *Qb, const double *c, int m)
    {
        if (m > 0 && cudaMemcpyAsync(h.coef.p, c, sizeof(double) * m, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return SP_ERR_CUDA;
        k_combine<T><<<nb, kHB, 0, st>>>(N, n, w, a, Qb, (const double *)h.coef.p, m);
        // the host array c must stay valid until the copy ran
        return cudaStreamSynchronize(st) == cudaSuccess ? 0 : SP_ERR_CUDA;
    }

    // Lowest eigenpair of H at n by m Lanczos steps from `start` (zero: a
    // fixed pseudo-random tangent field).  mode receives the unit Ritz vector.
    int lowest(const rec_t<T> *n, const rec_t<T> *start, rec_t<T> *mode, int m, double *lam)
    {
        rec_t<T> *w = (rec_t<T> *)h.w.p;
        // q_0 = start projected and normalised
        k_project<T><<<nb, kHB, 0, st>>>(N, n, start, q(0));
        double nrm2;
        int rc = dots(q(0), q(0), 1, &nrm2);
        if (rc) return rc;
        if (nrm2 != nrm2) return SP_ERR_NAN;  // a non-finite state or start vector
        if (!(nrm2 > 0)) return SP_ERR_ARG;
        double inv = 1.0 / sqrt(nrm2);
        k_lin<T><<<nb, kHB, 0, st>>>(N, q(0), inv, q(0), 0.0, q(0));
        std::vector<double> alpha, beta, c(kMaxKrylov + 1);
        int used = 0;
        // the Krylov space cannot outgrow the 2N-dimensional tangent space;
        // a residual at the rounding level of the stored records (relative
        // to the running estimate of |T|) is an invariant subspace, not a
        // new direction: normalising it would add a dependent vector
        m = (int)std::min<long long>(m, 2LL * N);
        const double brk = sizeof(T) == 4 ? 1e-5 : 1e-13;
        double tnorm = 0;
        for (int k = 0; k < m; ++k) {
            k_hvp<T><<<nb, kHB, 0, st>>>(S, n, q(k), w);
            // full reorthogonalisation, twice: w -= sum_j (q_j . w) q_j
            for (int pass = 0; pass < 2; ++pass) {
                if ((rc = dots(w, q(0), k + 1, c.data()))) return rc;
                if (pass == 0) alpha.push_back(c[k]);
                for (int j = 0; j <= k; ++j) c[j] = -c[j];
                if ((rc = combine(n, w, 1.0, q(0), c.data(), k + 1))) return rc;
            }
            used = k + 1;
            double b2;
            if ((rc = dots(w, w, 1, &b2))) return rc;
            double b = sqrt(b2);
            tnorm = std::max(tnorm, fabs(alpha[k]) + b + (k ? beta[k - 1] : 0.0));
            if (k == m - 1 || !(b > brk * tnorm)) break;
            beta.push_back(b);
            k_lin<T><<<nb, kHB, 0, st>>>(N, q(k + 1), 1.0 / b, w, 0.0, w);
        }
        // tridiagonal Rayleigh quotient: alpha on the diagonal, beta beside it
        std::vector<double> Tm((size_t)used * used, 0.0), d, V;
        for (int k = 0; k < used; ++k) {
            Tm[(size_t)k * used + k] = alpha[k];
            if (k + 1 < used) Tm[(size_t)k * used + k + 1] = Tm[(size_t)(k + 1) * used + k] = beta[k];
        }
        jacobi_eigen(Tm, used, d, V);
        int lo = (int)(std::min_element(d.begin(), d.end()) - d.begin());
        std::vector<double> y(used);
        for (int k = 0; k < used; ++k) y[k] = V[(size_t)k * used + lo];
        if (cudaMemsetAsync(mode, 0, sizeof(rec_t<T>) * (size_t)N, st) != cudaSuccess) return SP_ERR_CUDA;
        if ((rc = combine(n, mode, 0.0, q(0), y.data(), used))) return rc;
        if ((rc = dots(mode, mode, 1, &nrm2))) return rc;
        k_lin<T><<<nb, kHB, 0, st>>>(N, mode, 1.0 / sqrt(nrm2), mode, 0.0, mode);
        *lam = d[lo];
        return cudaGetLastError() == cudaSuccess ? 0 : SP_ERR_CUDA;
    }

    // F, the lowest mode (warm-started from `mode`, updated) and Fe at x
    int effective(const rec_t<T> *x, rec_t<T> *F, rec_t<T> *mode, rec_t<T> *Fe, int m, double *lam)
    {
        k_force<T><<<nb, kHB, 0, st>>>(S, x, F);
        int rc = lowest(x, mode, mode, m, lam);
        if (rc) return rc;
        double fl;
        if ((rc = dots(F, mode, 1, &fl))) return rc;
        if (*lam < 0)
            k_lin<T><<<nb, kHB, 0, st>>>(N, Fe, 1.0, F, -2.0 * fl, mode);
        else
            k_lin<T><<<nb, kHB, 0, st>>>(N, Fe, 0.0, F, -fl, mode);
        return cudaGetLastError() == cudaSuccess ? 0 : SP_ERR_CUDA;
    }
};

template <typename T>
int setup(sp_ctx *c, int m)
{
    HessScratch *&h = c->hess;
    if (!h) h = new HessScratch;
    size_t rec = sizeof(rec_t<T>) * (size_t)c->N;
    unsigned nb = hblocks(c->N);
    if (grow_h(h->Q, rec * (m + 1)) || grow_h(h->w, rec) || grow_h(h->F, rec) || grow_h(h->Fe, rec) ||
        grow_h(h->F2, rec) || grow_h(h->Fe2, rec) || grow_h(h->y, rec) || grow_h(h->mode2, rec) ||
        grow_h(h->part, sizeof(double) * (size_t)nb * (kMaxKrylov + 1)) ||
        grow_h(h->dots, sizeof(double) * (kMaxKrylov + 1)) || grow_h(h->coef, sizeof(double) * (kMaxKrylov + 1)))
        return SP_ERR_CUDA;
    return 0;
}

// a fixed pseudo-random field (integer hash of the index), for a cold start
template <typename T>
__global__ void k_seed_field(int N, rec_t<T> *v)
{
    int i = blockIdx.x * kHB + threadIdx.x;
    if (i >= N) return;
    uint32_t h[3];
    for (int k = 0; k < 3; ++k) {
        uint32_t z = (uint32_t)i * 2654435761u + (uint32_t)k * 40503u + 12345u;
        z ^= z >> 16;
        z *= 2246822519u;
        z ^= z >> 13;
        h[k] = z;
    }
    st(v, i, mk((T)((int)(h[0] >> 8) - (1 << 23)), (T)((int)(h[1] >> 8) - (1 << 23)), (T)((int)(h[2] >> 8) - (1 << 23))));
}

template <typename T>
int lowest_mode_run(sp_ctx *c, const Stencil<T> &S, const void *n, void *mode, int m, double *lam, cudaStream_t st)
{
    int rc = setup<T>(c, m);
    if (rc) return rc;
    Ops<T> op{S, *c->hess, st, c->N, hblocks(c->N)};
    rec_t<T> *md = (rec_t<T> *)mode;
    double z;
    if ((rc = op.dots(md, md, 1, &z))) return rc;
    if (!(z > 0)) k_seed_field<T><<<op.nb, kHB, 0, st>>>(c->N, md);
    return op.lowest((const rec_t<T> *)n, md, md, m, lam);
}

template <typename T>
int mmf_run(sp_ctx *c, const Stencil<T> &S, void *n, void *vel, void *mode, const sp_mmf_params *p, int n_iter,
            double *max_force, double *lam, cudaStream_t st)
{
    int rc = setup<T>(c, p->krylov);
    if (rc) return rc;
    HessScratch &h = *c->hess;
    Ops<T> op{S, h, st, c->N, hblocks(c->N)};
    int N = c->N;
    rec_t<T> *x = (rec_t<T> *)n, *v = (rec_t<T> *)vel, *md = (rec_t<T> *)mode;
    rec_t<T> *F = (rec_t<T> *)h.F.p, *Fe = (rec_t<T> *)h.Fe.p, *F2 = (rec_t<T> *)h.F2.p, *Fe2 = (rec_t<T> *)h.Fe2.p,
             *y = (rec_t<T> *)h.y.p;
    double z;
    if ((rc = op.dots(md, md, 1, &z))) return rc;
    if (!(z > 0)) k_seed_field<T><<<op.nb, kHB, 0, st>>>(N, md);
    double dth_m = p->dt / (2.0 * p->mass), dt2_2m = p->dt * p->dt / (2.0 * p->mass);
    if ((rc = op.effective(x, F, md, Fe, p->krylov, lam))) return rc;
    for (int it = 0; it < n_iter; ++it) {
        k_mmf_move<T><<<op.nb, kHB, 0, st>>>(N, x, v, Fe, y, p->dt, dt2_2m);
        if ((rc = op.effective(y, F2, md, Fe2, p->krylov, lam))) return rc;
        k_mmf_vel<T><<<op.nb, kHB, 0, st>>>(N, v, Fe, Fe2, dth_m);
        double vf, ff;
        if ((rc = op.dots(v, Fe2, 1, &vf)) || (rc = op.dots(Fe2, Fe2, 1, &ff))) return rc;
        double cpr = (vf > 0 && ff > 0) ? vf / ff : 0.0;
        k_lin<T><<<op.nb, kHB, 0, st>>>(N, v, 0.0, v, cpr, Fe2);
        if (cudaMemcpyAsync(x, y, sizeof(rec_t<T>) * (size_t)N, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(F, F2, sizeof(rec_t<T>) * (size_t)N, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(Fe, Fe2, sizeof(rec_t<T>) * (size_t)N, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return SP_ERR_CUDA;
    }
    k_maxnorm<T><<<op.nb, kHB, 0, st>>>(N, F, (double *)h.part.p);
    std::vector<double> pm(op.nb);
    if (cudaMemcpyAsync(pm.data(), h.part.p, sizeof(double) * op.nb, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SP_ERR_CUDA;
    *max_force = *std::max_element(pm.begin(), pm.end());
    return 0;
}

int hfail(sp_ctx *c, int code, const char *msg)
{
    c->err = msg;
    return code;
}

int hcheck(sp_ctx *c)
{
    if (!c) return SP_ERR_ARG;
    if (!c->have_geom || !c->have_ham) return hfail(c, SP_ERR_STATE, "context not configured");
    if (c->h.dipole != SP_DIPOLE_NONE) return hfail(c, SP_ERR_UNSUPPORTED, "Hessian with the dipole term");
    return status_enter(c);
}

// Device record arrays start on a record boundary (16 B in FP32, 32 B in FP64).
bool hrecords_aligned(const sp_ctx *c, std::initializer_list<const void *> ptrs)
{
    const uintptr_t a = c->prec == SP_F64 ? 32 : 16;
    for (const void *p : ptrs)
        if ((uintptr_t)p % a) return false;
    return true;
}

}  // namespace

namespace spgb {
template <typename T>
cudaError_t launch_hvp(const Stencil<T> &S, const rec_t<T> *n, const rec_t<T> *v, rec_t<T> *out, cudaStream_t st)
{
    if (S.N <= 0) return cudaSuccess;
    k_hvp<T><<<hblocks(S.N), kHB, 0, st>>>(S, n, v, out);
    return cudaGetLastError();
}
template cudaError_t launch_hvp<float>(const Stencil<float> &, const float4 *, const float4 *, float4 *, cudaStream_t);
template cudaError_t launch_hvp<double>(const Stencil<double> &, const dq4 *, const dq4 *, dq4 *, cudaStream_t);
}  // namespace spgb

void hess_scratch_destroy(HessScratch *h)
{
    if (!h) return;
    DevBuf *bufs[] = {&h->Q, &h->w, &h->F, &h->Fe, &h->F2, &h->Fe2, &h->y, &h->mode2, &h->part, &h->dots, &h->coef};
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    delete h;
}

extern "C" {

int sp_hessian_apply(sp_ctx *c, const void *n_dev, const void *v_dev, void *out_dev, void *stream)
{
    int rc = hcheck(c);
    if (rc) return rc;
    if (!n_dev || !v_dev || !out_dev) return hfail(c, SP_ERR_ARG, "NULL argument");
    if (v_dev == out_dev) return hfail(c, SP_ERR_ARG, "v and out must differ");
    if (!hrecords_aligned(c, {n_dev, v_dev, out_dev})) return hfail(c, SP_ERR_ARG, "misaligned record array");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned nb = hblocks(c->N);
    unsigned *w = status_word(c);
    if (!w) return hfail(c, SP_ERR_CUDA, "status word");
    cudaError_t e = c->prec == SP_F64 ? launch_pdl(k_hvp<double>, dim3(nb), dim3(kHB), 0, st, c->Sd, (const dq4 *)n_dev,
                                                   (const dq4 *)v_dev, (dq4 *)out_dev, w)
                                      : launch_pdl(k_hvp<float>, dim3(nb), dim3(kHB), 0, st, c->Sf,
                                                   (const float4 *)n_dev, (const float4 *)v_dev, (float4 *)out_dev, w);
    if (e != cudaSuccess) return hfail(c, SP_ERR_CUDA, "Hessian launch failed");
    return SP_OK;
}

int sp_lowest_mode(sp_ctx *c, const void *n_dev, void *mode_dev, int krylov, double *lambda, void *stream)
{
    int rc = hcheck(c);
    if (rc) return rc;
    if (!n_dev || !mode_dev || !lambda) return hfail(c, SP_ERR_ARG, "NULL argument");
    if (krylov < 1 || krylov > kMaxKrylov) return hfail(c, SP_ERR_ARG, "krylov must be in 1..256");
    if (!hrecords_aligned(c, {n_dev, mode_dev})) return hfail(c, SP_ERR_ARG, "misaligned record array");
    cudaStream_t st = (cudaStream_t)stream;
    rc = c->prec == SP_F64 ? lowest_mode_run<double>(c, c->Sd, n_dev, mode_dev, krylov, lambda, st)
                           : lowest_mode_run<float>(c, c->Sf, n_dev, mode_dev, krylov, lambda, st);
    if (rc == SP_ERR_NAN) return hfail(c, rc, "lowest mode: a non-finite value in the state or the start vector");
    if (rc) return hfail(c, rc, "Lanczos failed");
    return std::isfinite(*lambda) ? SP_OK : hfail(c, SP_ERR_NAN, "lowest mode: the eigenvalue is not finite");
}

int sp_mmf(sp_ctx *c, void *n_dev, void *vel_dev, void *mode_dev, const sp_mmf_params *p, int n_iter,
           double *max_force, double *lambda, void *stream)
{
    int rc = hcheck(c);
    if (rc) return rc;
    if (!n_dev || !vel_dev || !mode_dev || !p || !max_force || !lambda) return hfail(c, SP_ERR_ARG, "NULL argument");
    if (!(p->dt > 0) || !(p->mass > 0) || p->krylov < 1 || p->krylov > kMaxKrylov || n_iter < 0)
        return hfail(c, SP_ERR_ARG, "bad MMF parameters");
    if (!hrecords_aligned(c, {n_dev, vel_dev, mode_dev})) return hfail(c, SP_ERR_ARG, "misaligned record array");
    cudaStream_t st = (cudaStream_t)stream;
    rc = c->prec == SP_F64 ? mmf_run<double>(c, c->Sd, n_dev, vel_dev, mode_dev, p, n_iter, max_force, lambda, st)
                           : mmf_run<float>(c, c->Sf, n_dev, vel_dev, mode_dev, p, n_iter, max_force, lambda, st);
    if (rc == SP_ERR_NAN) return hfail(c, rc, "minimum mode following: a non-finite value");
    if (rc) return hfail(c, rc, "minimum mode following failed");
    return std::isfinite(*max_force) && std::isfinite(*lambda)
               ? SP_OK
               : hfail(c, SP_ERR_NAN, "minimum mode following: the force or eigenvalue is not finite");
}

}  // extern "C"
