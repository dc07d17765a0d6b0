// minimise.cu -- velocity projection (Appendix D) and GNEB (Sec. GNEB,
// Appendix F) on the GPU.
//
// Work is cut into blocks of kBlock spins of one image ("image" = one system
// of one chain; a plain minimisation is one image).  Per-image scalars
// (energy, geodesic distance, tangent norm, projections, max force) are
// reduced deterministically: every block writes its partial, and the last
// block of the image to finish (atomic ticket) sums the image's partials in
// a fixed order and re-arms the ticket.  Kernels of one iteration:
//   move    v <- projection of v on F (from the previous force pass),
//           x <- normalise(x + dt v + dt^2/(2m) F)          (interior images)
//   field   B(x), E_v, Pg = -(B - (B.x)x), theta^2 to image v+1
//   tangent improved tangent, per-spin projection, |tau|^2, Pg.tau
//   force   F' (spring / climbing image), v <- v + dt/(2m)(F + F'),
//           v.F', F'.F', max |F'|
#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "minimise.h"

namespace spgb {

namespace {

struct ImgInfo {
    long long spin0;  // record offset of image 0 of the chain
    int N, chain, nu, M, g0, blk0, bpi;
    int kind;  // SP_IMAGE_* or -1: climbing decided by the climbing flag
};
struct BlkInfo {
    int g, t;
};

// per-image scalar slots (kS doubles per image): energy, squared geodesic
// distance to the next image, |tau|^2, Pg.tau, v.F, F.F, max_i |F_i|^2,
// energy-weighted segment length, tangent weights of the forward and
// backward differences, force coefficient a (F = -Pg + a tau), velocity
// projection coefficient v.F / F.F
enum { kE = 0, kL2, kTT, kGT, kVF, kFF, kFMAX, kLW, kWP, kWM, kA, kC, kS = 16 };

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

int grow(Buf &b, size_t bytes)
{
    if (b.p && b.bytes >= bytes) return 0;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) return SP_ERR_CUDA;
    b.bytes = bytes;
    return 0;
}

}  // namespace

struct MinScratch {
    Buf F, G, Tau, scal, part, cnt, blk, img, sten, state, aux, sync;
    int *host_state = nullptr;  // pinned: iters, active
    double *host_fmax = nullptr;
    // batch layout last uploaded (block/image tables and stencils)
    std::vector<char> layout;
    int n_img = 0, n_blk = 0, n_chains = 0;
    // CUDA graph of kGraphIters steady-state GNEB iterations
    cudaStream_t gstream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<char> gkey;
};

constexpr int kGraphIters = 8;

void min_scratch_destroy(MinScratch *s)
{
    if (!s) return;
    Buf *bufs[] = {&s->F, &s->G, &s->Tau, &s->scal, &s->part, &s->cnt, &s->blk, &s->img, &s->sten, &s->state, &s->aux,
                   &s->sync};
    for (Buf *b : bufs)
        if (b->p) cudaFree(b->p);
    if (s->host_state) cudaFreeHost(s->host_state);
    if (s->host_fmax) cudaFreeHost(s->host_fmax);
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    if (s->gstream) cudaStreamDestroy(s->gstream);
    if (s->ev0) cudaEventDestroy(s->ev0);
    if (s->ev1) cudaEventDestroy(s->ev1);
    delete s;
}

namespace {

int scratch(MinScratch **s)
{
    if (!*s) {
        *s = new (std::nothrow) MinScratch();
        if (!*s) return SP_ERR_STATE;
        if (cudaMallocHost(&(*s)->host_state, 4 * sizeof(int)) != cudaSuccess) return SP_ERR_CUDA;
        if (cudaMallocHost(&(*s)->host_fmax, sizeof(double)) != cudaSuccess) return SP_ERR_CUDA;
    }
    return 0;
}

// Counters must start at zero; the reduction leaves them at zero.
int grow_counters(Buf &b, size_t n, cudaStream_t st)
{
    size_t bytes = n * sizeof(unsigned);
    if (b.p && b.bytes >= bytes) return 0;
    if (grow(b, bytes)) return SP_ERR_CUDA;
    return cudaMemsetAsync(b.p, 0, b.bytes, st) == cudaSuccess ? 0 : SP_ERR_CUDA;
}

// Per-image dot-product accumulators: float-float for FP32 (the FP64 sum of
// the same exact products to ~1e-14), plain FP64 for FP64.
template <typename T> struct Acc {
    using type = double;
};
template <> struct Acc<float> {
    using type = f2sum;
};
__device__ __forceinline__ f2sum acc_dot(v3<float> a, v3<float> b) { return exact_dot(a, b); }
__device__ __forceinline__ double acc_dot(v3<double> a, v3<double> b) { return dot(a, b); }

template <int NV, typename V>
__device__ __forceinline__ V combine(int k, unsigned maxmask, V a, V b)
{
    return ((maxmask >> k) & 1u) ? nan_max(a, b) : a + b;
}

struct NoPost {
    __device__ void operator()(double *) const {}
};

// Deterministic per-image reduction of NV values (bit k of maxmask: max
// instead of sum; maxima are of non-negative values, 0 is their identity).
// Every thread of every block of the image must call it.  The warp-level
// step runs in the values' own type V (float, double or f2sum); from the warp
// results on everything is FP64.  After one barrier warps 1.. leave; warp 0
// combines the warp results by a fixed shuffle tree into the block's partial
// and takes a ticket; warp 0 of the image's last block sums the partials
// (lane l takes partials l, l + 32, ..., then a shuffle tree), writes the
// totals to out[] and calls post(out).
template <int NV, typename V, typename Post = NoPost>
__device__ void image_reduce(V (&v)[NV], unsigned maxmask, double *__restrict__ part, int blk, int blk0, int bpi,
                             unsigned *counter, double *out, Post post = Post())
{
    constexpr int NW = kBlock / 32;
    static_assert(NW <= 32, "one warp combines the warp results");
    __shared__ double sh[NW][NV];
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] = combine<NV>(k, maxmask, v[k], shfl_down(v[k], o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
        for (int k = 0; k < NV; ++k) sh[w][k] = to_double(v[k]);
    __syncthreads();
    if (w != 0) return;
    double a[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        a[k] = l < NW ? sh[l][k] : 0.0;
        for (int o = NW / 2; o > 0; o >>= 1) a[k] = combine<NV, double>(k, maxmask, a[k], shfl_down(a[k], o));
    }
    int last = 0;
    if (l == 0) {
        for (int k = 0; k < NV; ++k) part[(size_t)blk * NV + k] = a[k];
        __threadfence();
        unsigned ticket = atomicAdd(counter, 1u);
        last = ticket == (unsigned)(bpi - 1);
    }
    if (!__shfl_sync(0xffffffffu, last, 0)) return;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    for (int p = l; p < bpi; p += 32)
        for (int k = 0; k < NV; ++k)
            acc[k] = combine<NV, double>(k, maxmask, acc[k], __ldcg(&part[(size_t)(blk0 + p) * NV + k]));
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) acc[k] = combine<NV, double>(k, maxmask, acc[k], shfl_down(acc[k], o));
    if (l == 0) {
        for (int k = 0; k < NV; ++k) out[k] = acc[k];
        post(out);
        atomicExch(counter, 0u);
    }
}

// After a force pass (out = scal + kS g + kVF): the projection coefficient
// v.F / F.F (0 unless both are positive) of the next move.
struct ProjectionPost {
    __device__ void operator()(double *out) const
    {
        double vf = out[kVF - kVF], ff = out[kFF - kVF];
        out[kC - kVF] = (vf > 0 && ff > 0) ? vf / ff : 0.0;
    }
};

// ============================================================ VP minimiser
// state (ints): [0] iterations performed, [1] active flag
// scal (doubles): v.F, F.F, max|F|^2, projection-valid flag
// (max |F|^2 rather than max |F|: one square root per image instead of one
// per spin; sqrt is monotonic and correctly rounded, so sqrt(max |F|^2) is
// exactly max |F| in FP64)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_vp_force(const __grid_constant__ Stencil<T> S, const rec_t<T> *__restrict__ x,
                                                     rec_t<T> *__restrict__ v, rec_t<T> *__restrict__ F, T dth_m,
                                                     int mode, double *part, unsigned *cnt, double *scal,
                                                     const int *state)
{
    allow_dependents();
    wait_prerequisite();  // state, scalars and records come from the kernels before
    if (mode == 1 && state[1] == 0) return;
    int i = blockIdx.x * kBlock + threadIdx.x;
    T r[3] = {0, 0, 0};
    if (i < S.N) {
        int b;
        v3<T> ni = ld(x, i);
        v3<T> B = local_field(S, x, i, ni, b);
        v3<T> Fn = B - dot(B, ni) * ni;
        if (mode == 1) {
            v3<T> vi = axpy(dth_m, ldc(F, i) + Fn, ldc(v, i));
            st(v, i, vi);
            r[0] = dot(vi, Fn);
        }
        st(F, i, Fn);
        r[1] = dot(Fn, Fn);
        r[2] = r[1];
    }
    image_reduce<3>(r, 4u, part, blockIdx.x, 0, gridDim.x, cnt, scal);
    if (blockIdx.x == 0 && threadIdx.x == 0) scal[3] = mode;
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_vp_move(int N, rec_t<T> *__restrict__ x, rec_t<T> *__restrict__ v,
                                                    const rec_t<T> *__restrict__ F, T dt, T dt2_2m, double tol,
                                                    int k, int max_iter, const double *scal, int *state)
{
    allow_dependents();
    wait_prerequisite();  // state, scalars and records come from the kernels before
    __shared__ T s_c;
    __shared__ int s_done;
    if (threadIdx.x == 0) {
        double vf = scal[0], ff = scal[1];
        s_c = (vf > 0 && ff > 0) ? (T)(vf / ff) : T(0);
        s_done = (sqrt(scal[2]) < tol) || (k >= max_iter);
    }
    __syncthreads();
    bool done = s_done;
    bool proj = scal[3] != 0.0;
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i < N) {
        v3<T> vi;
        if (proj) {
            T c = s_c;
            vi = c * ldc(F, i);
            st(v, i, vi);
        } else {
            vi = ldc(v, i);
        }
        if (!done) st(x, i, normalised(axpy(dt2_2m, ldc(F, i), axpy(dt, vi, ldc(x, i)))));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        state[1] = done ? 0 : 1;
        if (!done) state[0] = k + 1;
    }
}

// ============================================================ GNEB
// The GNEB passes are written as bodies for one work block `vb` (an entry of
// the block table), so that the per-pass kernels (vb = blockIdx.x) and the
// persistent kernel (a CTA takes several vb in turn) run the same code.
// R: the record type the mutable buffers are read through -- rec_t<T> (the
// per-pass kernels: spins by the read-only path) or the plain-load record
// type of ShRec<T> (the persistent kernel, which reads what other blocks
// wrote earlier in the same launch).
template <typename T, typename R>
__device__ __forceinline__ void g_field_body(int vb, const BlkInfo *__restrict__ blk, const ImgInfo *__restrict__ img,
                                             const Stencil<T> *__restrict__ S, const R *x, R *G, double *part,
                                             unsigned *cnt, double *scal)
{
    BlkInfo bi = blk[vb];
    ImgInfo im = img[bi.g];
    // the chain's stencil, staged in shared memory for the neighbour loop
    __shared__ __align__(16) unsigned char st_raw[sizeof(Stencil<T>)];
    Stencil<T> &St = *reinterpret_cast<Stencil<T> *>(st_raw);
    stage_stencil(S + im.chain, &St);
    int i = bi.t * kBlock + threadIdx.x;
    const R *xb = x + im.spin0 + (long long)im.nu * im.N;
    // energy and squared angle sums: FP64, or float-float for FP32 (the
    // same sums of the same products to ~1e-14, off the FP64 pipe)
    using A = typename Acc<T>::type;
    A r[2] = {A{}, A{}};
    if (i < im.N) {
        int b;
        v3<T> ni = ld(xb, i);
        v3<T> B = local_field(St, xb, i, ni, b);
        v3<T> Bz = mk(St.Bz[b][0], St.Bz[b][1], St.Bz[b][2]);
        v3<T> pg = dot(B, ni) * ni - B;  // tangent-space part of dH/dn = -B
        st(G, im.spin0 + (long long)im.nu * im.N + i, pg);
        T th = T(0);
        if (im.nu < im.M - 1) {
            v3<T> nj = ld(xb + im.N, i);
            v3<T> c = cross(ni, nj);
            th = atan2(sqrt(dot(c, c)), dot(ni, nj));
        }
        if constexpr (std::is_same<T, float>::value) {
            f2sum e = exact_dot(ni, B + Bz);
            r[0] = f2sum{-0.5f * e.hi, -0.5f * e.lo};
            r[1] = exact_square(th);
        } else {
            r[0] = -0.5 * ddot(ni, B + Bz);
            r[1] = th * th;
        }
    }
    image_reduce<2>(r, 0u, part, vb, im.blk0, im.bpi, cnt + bi.g, scal + kS * bi.g + kE);
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_g_field(const BlkInfo *__restrict__ blk, const ImgInfo *__restrict__ img,
                                                    const Stencil<T> *__restrict__ S, const rec_t<T> *__restrict__ x,
                                                    rec_t<T> *__restrict__ G, double *part, unsigned *cnt, double *scal)
{
    g_field_body<T>(blockIdx.x, blk, img, S, x, G, part, cnt, scal);
}

// Weights (w+, w-) of the forward and backward differences in the improved
// tangent (Henkelman and Jonsson 2000) of interior image g, from the image
// energies of the field pass.
__device__ __forceinline__ void tangent_weights(const double *scal, int g, double *wp_out, double *wm_out)
{
    double Ep = scal[kS * (g + 1) + kE], E0 = scal[kS * g + kE], Em = scal[kS * (g - 1) + kE];
    double wp, wm;
    if (Ep > E0 && E0 > Em) {
        wp = 1;
        wm = 0;
    } else if (Ep < E0 && E0 < Em) {
        wp = 0;
        wm = 1;
    } else {
        double dmax = fmax(fabs(Ep - E0), fabs(Em - E0)), dmin = fmin(fabs(Ep - E0), fabs(Em - E0));
        if (Ep > Em) {
            wp = dmax;
            wm = dmin;
        } else {
            wp = dmin;
            wm = dmax;
        }
    }
    *wp_out = wp;
    *wm_out = wm;
}

// LOCALW: the weights are computed here from the energies (persistent
// kernel) instead of read from the slots k_g_weights filled -- the same
// function of the same values.
template <typename T, bool LOCALW, typename R>
__device__ __forceinline__ void g_tangent_body(int vb, const BlkInfo *__restrict__ blk, const ImgInfo *__restrict__ img,
                                               const R *x, const R *G, R *Tau, double *part, unsigned *cnt,
                                               double *scal)
{
    BlkInfo bi = blk[vb];
    ImgInfo im = img[bi.g];
    int i = bi.t * kBlock + threadIdx.x;
    long long p = im.spin0 + (long long)im.nu * im.N + i;
    bool end = im.nu == 0 || im.nu == im.M - 1;
    // weights of the forward and backward differences, read (or computed
    // from the three energies) by every thread: no block barrier
    T s_wp = T(0), s_wm = T(0);
    if (!end) {
        if (LOCALW) {
            double wp, wm;
            tangent_weights(scal, bi.g, &wp, &wm);
            s_wp = (T)wp;
            s_wm = (T)wm;
        } else {
            s_wp = (T)scal[kS * bi.g + kWP];
            s_wm = (T)scal[kS * bi.g + kWM];
        }
    }
    using A = typename Acc<T>::type;
    A r[2] = {A{}, A{}};
    if (i < im.N && end) {
        // endpoints: one-sided difference to the neighbouring image (only its
        // slope dE/dr is used, for the interpolated path energy)
        v3<T> xi = ld(x, p);
        v3<T> t = im.nu == 0 ? ld(x, p + im.N) - xi : xi - ld(x, p - im.N);
        t = t - dot(t, xi) * xi;
        st(Tau, p, t);
        r[0] = acc_dot(t, t);
        r[1] = acc_dot(ldc(G, p), t);
    } else if (i < im.N) {
        v3<T> xi = ld(x, p), xp = ld(x, p + im.N), xm = ld(x, p - im.N);
        v3<T> t = axpy(s_wp, xp - xi, s_wm * (xi - xm));
        t = t - dot(t, xi) * xi;
        st(Tau, p, t);
        r[0] = acc_dot(t, t);
        r[1] = acc_dot(ldc(G, p), t);
    }
    image_reduce<2>(r, 0u, part, vb, im.blk0, im.bpi, cnt + bi.g, scal + kS * bi.g + kTT);
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_g_tangent(const BlkInfo *__restrict__ blk, const ImgInfo *__restrict__ img,
                                                      const rec_t<T> *__restrict__ x, const rec_t<T> *__restrict__ G,
                                                      rec_t<T> *__restrict__ Tau, double *part, unsigned *cnt,
                                                      double *scal)
{
    g_tangent_body<T, false>(blockIdx.x, blk, img, x, G, Tau, part, cnt, scal);
}

// Tangent weights of every interior image into its slots; one thread per image.
__global__ void k_g_weights(const ImgInfo *__restrict__ img, int n_img, double *scal)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_img) return;
    ImgInfo im = img[g];
    if (im.nu == 0 || im.nu == im.M - 1) return;
    tangent_weights(scal, g, &scal[kS * g + kWP], &scal[kS * g + kWM]);
}

// Slope dE/dr of image g along its normalised tangent.
__device__ __forceinline__ double slope_of(const double *scal, int g)
{
    double tt = scal[kS * g + kTT];
    return tt > 0 ? scal[kS * g + kGT] / sqrt(tt) : 0.0;
}

// Energy-weighted length of the segment from image a to a+1 (reading of the
// paper's spring modulation: arc length of the curve ((1-w) r, w E(r)) over
// the geodesic distance h, E(r) the cubic Hermite interpolant of the two
// images' energies and slopes), by adaptive Simpson with Lyness' criterion
// and Richardson correction to 1e-13 h, subdivision depth at most 40 (an
// explicit stack of at most 41 intervals).
// The per-image scalars below are computed both by one-thread-per-image
// kernels and inside the persistent kernel; every product and sum is written
// with the non-contracting intrinsics, so that the two give the same bits
// whatever fused multiply-adds the compiler would otherwise form.
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }

__device__ double seg_integrand(double Ea, double Eb, double da, double db, double h, double w, double s)
{
    double t = s / h, t2 = dmul(t, t);
    double c6 = dadd(dmul(6.0, t2), -dmul(6.0, t));  // 6 t^2 - 6 t
    double ce = dadd(dmul(c6, Ea), dmul(-c6, Eb)) / h;
    double ca = dadd(dadd(dmul(3.0, t2), -dmul(4.0, t)), 1.0);  // 3 t^2 - 4 t + 1
    double cb = dadd(dmul(3.0, t2), -dmul(2.0, t));            // 3 t^2 - 2 t
    double dE = dadd(dadd(ce, dmul(ca, da)), dmul(cb, db));
    double u = 1.0 - w;
    return sqrt(dadd(dmul(u, u), dmul(dmul(w, w), dmul(dE, dE))));
}

__device__ double seg_length(double Ea, double Eb, double da, double db, double h, double w)
{
    if (w == 0.0) return h;
    if (!(h > 0)) return 0.0;
    struct Iv {
        double a, b, fa, fm, fb, whole, eps;
        int depth;
    } stk[44];
    int sp = 0;
    double fa = seg_integrand(Ea, Eb, da, db, h, w, 0.0), fm = seg_integrand(Ea, Eb, da, db, h, w, 0.5 * h),
           fb = seg_integrand(Ea, Eb, da, db, h, w, h);
    stk[sp++] = Iv{0.0, h, fa, fm, fb, dmul(h / 6, dadd(dadd(fa, dmul(4.0, fm)), fb)), 1e-13 * h, 40};
    double total = 0.0;
    while (sp > 0) {
        Iv c = stk[--sp];
        double m = 0.5 * (c.a + c.b), lm = 0.5 * (c.a + m), rm = 0.5 * (m + c.b);
        double flm = seg_integrand(Ea, Eb, da, db, h, w, lm), frm = seg_integrand(Ea, Eb, da, db, h, w, rm);
        double left = dmul((m - c.a) / 6, dadd(dadd(c.fa, dmul(4.0, flm)), c.fm));
        double right = dmul((c.b - m) / 6, dadd(dadd(c.fm, dmul(4.0, frm)), c.fb));
        double d = dadd(dadd(left, right), -c.whole);
        if (c.depth <= 0 || fabs(d) <= 15 * c.eps) {
            total = dadd(total, dadd(dadd(left, right), d / 15));
        } else {
            // right half below the left one: the left half is finished first
            stk[sp++] = Iv{m, c.b, c.fm, frm, c.fb, right, 0.5 * c.eps, c.depth - 1};
            stk[sp++] = Iv{c.a, m, c.fa, flm, c.fm, left, 0.5 * c.eps, c.depth - 1};
        }
    }
    return total;
}

// Energy-weighted length of segment (g, g+1) from the image slots.
__device__ __forceinline__ double segment_of(const double *scal, int g, double w)
{
    return seg_length(scal[kS * g + kE], scal[kS * (g + 1) + kE], slope_of(scal, g), slope_of(scal, g + 1),
                      sqrt(scal[kS * g + kL2]), w);
}

// scal[8g + kLW] = energy-weighted length of segment (g, g+1), one thread per image.
__global__ void k_g_seglen(const ImgInfo *__restrict__ img, int n_img, double w, double *scal)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_img) return;
    ImgInfo im = img[g];
    if (im.nu >= im.M - 1) return;
    scal[kS * g + kLW] = segment_of(scal, g, w);
}

// The force coefficient a of every interior image (F = -Pg + a tau):
// climbing image (the chain's highest interior image when climbing is on and
// the image has no fixed kind): a = 2 Pg.tau / |tau|^2; falling image: 0;
// otherwise (Pg.tau / |tau| + k (l_g - l_{g-1})) / |tau|, l the geodesic or
// energy-weighted segment lengths.  One thread per image.
// lw_g, lw_gm: the energy-weighted lengths of segments (g, g+1) and
// (g-1, g) (used when `weighted`).
__device__ __forceinline__ double force_coef(const ImgInfo &im, int g, double kspring, int climbing, int weighted,
                                             const double *scal, double lw_g, double lw_gm)
{
    int ci = -1;
    if (climbing && im.kind < 0) {
        ci = 1;
        double best = scal[kS * (im.g0 + 1) + kE];
        for (int nu = 2; nu < im.M - 1; ++nu) {
            double e = scal[kS * (im.g0 + nu) + kE];
            if (e > best) {
                best = e;
                ci = nu;
            }
        }
    }
    double tt = scal[kS * g + kTT];
    double inv = tt > 0 ? 1.0 / sqrt(tt) : 0.0;
    double gt = dmul(scal[kS * g + kGT], inv);
    double fs = weighted ? dmul(kspring, lw_g - lw_gm)
                         : dmul(kspring, sqrt(scal[kS * g + kL2]) - sqrt(scal[kS * (g - 1) + kL2]));
    int kind = im.kind >= 0 ? im.kind : (im.nu == ci ? SP_IMAGE_CLIMBING : SP_IMAGE_NORMAL);
    // climbing: tangential component inverted, no spring; falling: the full
    // projected gradient, no spring (descends to a minimum along the path)
    double coef = kind == SP_IMAGE_CLIMBING ? 2.0 * gt : (kind == SP_IMAGE_FALLING ? 0.0 : dadd(gt, fs));
    return dmul(coef, inv);
}

__global__ void k_g_coef(const ImgInfo *__restrict__ img, int n_img, double kspring, int climbing, int weighted,
                         double *scal)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_img) return;
    ImgInfo im = img[g];
    if (im.nu == 0 || im.nu == im.M - 1) return;
    scal[kS * g + kA] = force_coef(im, g, kspring, climbing, weighted, scal, weighted ? scal[kS * g + kLW] : 0.0,
                                   weighted ? scal[kS * (g - 1) + kLW] : 0.0);
}

// Coefficients of the force pass when computed in place (persistent kernel).
struct CoefArgs {
    double kspring, w;
    int climbing, weighted;
};

template <typename T, bool LOCALC, typename R>
__device__ __forceinline__ void g_force_body(int vb, const BlkInfo *__restrict__ blk, const ImgInfo *__restrict__ img,
                                             R *v, R *F, const R *G, const R *Tau, T dth_m, int mode, double *part,
                                             unsigned *cnt, double *scal, CoefArgs ca)
{
    BlkInfo bi = blk[vb];
    ImgInfo im = img[bi.g];
    if (im.nu == 0 || im.nu == im.M - 1) return;
    // the image's force is -G + a Tau (a from k_g_coef, or computed here from
    // the same slots by the same function)
    // (k_g_coef's slot: every thread reads it, no block barrier; computed in
    // place: thread 0 evaluates it once and the block waits)
    __shared__ T sh_a;
    T s_a;
    if (LOCALC) {
        if (threadIdx.x == 0) {
            double lw = 0, lwm = 0;
            if (ca.weighted) {
                lw = segment_of(scal, bi.g, ca.w);
                lwm = segment_of(scal, bi.g - 1, ca.w);
            }
            sh_a = (T)force_coef(im, bi.g, ca.kspring, ca.climbing, ca.weighted, scal, lw, lwm);
        }
        __syncthreads();
        s_a = sh_a;
    } else {
        s_a = (T)scal[kS * bi.g + kA];
    }
    int i = bi.t * kBlock + threadIdx.x;
    long long p = im.spin0 + (long long)im.nu * im.N + i;
    using A = typename Acc<T>::type;
    A r[3] = {A{}, A{}, A{}};
    if (i < im.N) {
        v3<T> Fn = axpy(s_a, ld(Tau, p), -ldc(G, p));
        if (mode == 1) {
            v3<T> vi = axpy(dth_m, ldc(F, p) + Fn, ldc(v, p));
            st(v, p, vi);
            r[0] = acc_dot(vi, Fn);
        }
        st(F, p, Fn);
        r[1] = acc_dot(Fn, Fn);
        r[2] = r[1];  // max |F|^2; the image's max |F| is its square root
    }
    image_reduce<3>(r, 4u, part, vb, im.blk0, im.bpi, cnt + bi.g, scal + kS * bi.g + kVF, ProjectionPost());
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_g_force(const BlkInfo *__restrict__ blk, const ImgInfo *__restrict__ img,
                                                    rec_t<T> *__restrict__ v, rec_t<T> *__restrict__ F,
                                                    const rec_t<T> *__restrict__ G, const rec_t<T> *__restrict__ Tau,
                                                    T dth_m, int mode, double *part, unsigned *cnt, double *scal)
{
    g_force_body<T, false>(blockIdx.x, blk, img, v, F, G, Tau, dth_m, mode, part, cnt, scal, CoefArgs{});
}

// mode 0: move; 1: project then move; 2: project only
template <typename T, typename R>
__device__ __forceinline__ void g_move_body(int vb, const BlkInfo *__restrict__ blk, const ImgInfo *__restrict__ img,
                                            R *x, R *v, const R *F, T dt, T dt2_2m, int mode, const double *scal)
{
    BlkInfo bi = blk[vb];
    ImgInfo im = img[bi.g];
    if (im.nu == 0 || im.nu == im.M - 1) return;
    // projection coefficient of the last force pass: every thread reads the
    // image's slot (one broadcast load, no block barrier)
    const T c = mode >= 1 ? (T)scal[kS * bi.g + kC] : T(0);
    int i = bi.t * kBlock + threadIdx.x;
    if (i >= im.N) return;
    long long p = im.spin0 + (long long)im.nu * im.N + i;
    v3<T> vi;
    if (mode >= 1) {
        vi = c * ldc(F, p);
        st(v, p, vi);
    } else {
        vi = ldc(v, p);
    }
    if (mode <= 1) st(x, p, normalised(axpy(dt2_2m, ldc(F, p), axpy(dt, vi, ldc(x, p)))));
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_g_move(const BlkInfo *__restrict__ blk, const ImgInfo *__restrict__ img,
                                                   rec_t<T> *__restrict__ x, rec_t<T> *__restrict__ v,
                                                   const rec_t<T> *__restrict__ F, T dt, T dt2_2m, int mode,
                                                   const double *scal)
{
    g_move_body<T>(blockIdx.x, blk, img, x, v, F, dt, dt2_2m, mode, scal);
}

// ------------------------------------------------------------ persistent GNEB
// Grid-wide barrier of a cooperative launch, with a bounded wait: the arrival
// counter *bar only grows (by gridDim.x per barrier; the host zeroes it before
// the launch).  A block polls at most `limit` times; a block that gives up
// raises *abort_flag and ORs `site` into status[1] (the context's status word,
// timeouts), and every block that sees the abort flag while waiting leaves
// too, so no block waits unboundedly.  Returns false when the kernel must
// return.
__device__ bool grid_sync(unsigned *bar, unsigned *abort_flag, unsigned &gen, long long limit, unsigned *status,
                          unsigned site)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        gen += 1;
        const unsigned target = gen * gridDim.x;
        __threadfence();  // this block's writes before its arrival
        atomicAdd(bar, 1u);
        int ok = 1;
        long long polls = 0;
        while (*(volatile unsigned *)bar < target) {
            if (*(volatile unsigned *)abort_flag) {
                ok = 0;
                break;
            }
            if (++polls > limit) {
                ok = 0;
                atomicExch(abort_flag, 1u);
                if (status) atomicOr_system(status + 1, site);
                break;
            }
            __nanosleep(64);
        }
        __threadfence();  // the other blocks' writes after the barrier
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename T> struct PersistArgs {
    const BlkInfo *blk;
    const ImgInfo *img;
    const Stencil<T> *S;
    rec_t<T> *x, *v, *F, *G, *Tau;
    double *part, *scal;
    unsigned *cnt;
    T dt, dt2_2m, dth_m;
    int n_blk, n_iter, first_mode;  // first_mode: move mode of the first iteration (0 or 1)
    CoefArgs ca;
    unsigned *bar, *abort_flag, *status;
    long long limit;
};

// n_iter GNEB iterations (move, field, tangent, force) of every image of
// every chain in one cooperative launch: each pass is a grid-stride loop over
// the block table, the passes are separated by grid barriers, and the
// per-image tangent weights and force coefficients are computed by each work
// block from the slots the previous pass filled (the same functions of the
// same values as the per-pass kernels, so the iterates are bit-identical).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_g_persistent(const __grid_constant__ PersistArgs<T> a)
{
    // every spin, velocity and pass buffer is read with plain (coherent)
    // loads: other blocks wrote them earlier in this launch
    using R = typename ShRec<T>::type;
    static_assert(sizeof(R) == sizeof(rec_t<T>), "plain-load records have the record layout");
    R *x = reinterpret_cast<R *>(a.x), *v = reinterpret_cast<R *>(a.v), *F = reinterpret_cast<R *>(a.F),
      *G = reinterpret_cast<R *>(a.G), *Tau = reinterpret_cast<R *>(a.Tau);
    unsigned gen = 0;
    for (int it = 0; it < a.n_iter; ++it) {
        const int mode = it == 0 ? a.first_mode : 1;
        for (int vb = blockIdx.x; vb < a.n_blk; vb += gridDim.x) {
            g_move_body<T>(vb, a.blk, a.img, x, v, (const R *)F, a.dt, a.dt2_2m, mode, a.scal);
            __syncthreads();
        }
        if (!grid_sync(a.bar, a.abort_flag, gen, a.limit, a.status, 1u)) return;
        for (int vb = blockIdx.x; vb < a.n_blk; vb += gridDim.x) {
            g_field_body<T>(vb, a.blk, a.img, a.S, (const R *)x, G, a.part, a.cnt, a.scal);
            __syncthreads();
        }
        if (!grid_sync(a.bar, a.abort_flag, gen, a.limit, a.status, 1u)) return;
        for (int vb = blockIdx.x; vb < a.n_blk; vb += gridDim.x) {
            g_tangent_body<T, true>(vb, a.blk, a.img, (const R *)x, (const R *)G, Tau, a.part, a.cnt, a.scal);
            __syncthreads();
        }
        if (!grid_sync(a.bar, a.abort_flag, gen, a.limit, a.status, 1u)) return;
        for (int vb = blockIdx.x; vb < a.n_blk; vb += gridDim.x) {
            g_force_body<T, true>(vb, a.blk, a.img, v, F, (const R *)G, (const R *)Tau, a.dth_m, 1, a.part, a.cnt,
                                  a.scal, a.ca);
            __syncthreads();
        }
        if (!grid_sync(a.bar, a.abort_flag, gen, a.limit, a.status, 1u)) return;
    }
}

__global__ void k_g_finish(const ImgInfo *__restrict__ img, int n_img, const double *scal, double *E, double *fmax_out,
                           int n_chains)
{
    // one thread per image; the thread of each chain's image 0 also takes the
    // chain's max force over its interior images (in image order)
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n_img; g += gridDim.x * blockDim.x) {
        E[g] = scal[kS * g + kE];
        const ImgInfo im = img[g];
        if (im.nu != 0 || im.chain >= n_chains) continue;
        double m = 0;
        for (int nu = 1; nu < im.M - 1; ++nu) m = nan_max(m, scal[kS * (im.g0 + nu) + kFMAX]);
        fmax_out[im.chain] = sqrt(m);  // the slot holds max |F|^2
    }
}

}  // namespace

// ------------------------------------------------------------ VP host loop
template <typename T>
int vp_minimise(MinScratch **sp, const Stencil<T> &S, void *n, void *v, const MinArgs &a, int *iters, double *max_torque,
                cudaStream_t st)
{
    int rc = scratch(sp);
    if (rc) return rc;
    MinScratch *s = *sp;
    int N = S.N;
    int nblk = blocks_for(N > 0 ? N : 1);
    if (grow(s->F, sizeof(rec_t<T>) * (size_t)(N > 0 ? N : 1)) || grow(s->scal, 8 * sizeof(double)) ||
        grow(s->part, 3 * sizeof(double) * (size_t)nblk) || grow_counters(s->cnt, 1, st) ||
        grow(s->state, 4 * sizeof(int)))
        return SP_ERR_CUDA;
    rec_t<T> *x = (rec_t<T> *)n, *vv = (rec_t<T> *)v, *F = (rec_t<T> *)s->F.p;
    double *scal = (double *)s->scal.p, *part = (double *)s->part.p;
    unsigned *cnt = (unsigned *)s->cnt.p;
    int *state = (int *)s->state.p;
    double dth_m = a.dt / (2.0 * a.mass), dt2_2m = a.dt * a.dt / (2.0 * a.mass);
    if (cudaMemsetAsync(state, 0, 4 * sizeof(int), st) != cudaSuccess) return SP_ERR_CUDA;
    launch_pdl(k_vp_force<T>, dim3(nblk), dim3(kBlock), 0, st, S, x, vv, F, (T)dth_m, 0, part, cnt, scal, (const int *)state);
    int k = 0;
    while (k < a.max_iter) {
        int chunk = std::min(a.check_every, a.max_iter - k);
        for (int c = 0; c < chunk; ++c, ++k) {
            launch_pdl(k_vp_move<T>, dim3(nblk), dim3(kBlock), 0, st, N, x, vv, (const rec_t<T> *)F, (T)a.dt, (T)dt2_2m, a.tol, k,
                       a.max_iter, (const double *)scal, state);
            launch_pdl(k_vp_force<T>, dim3(nblk), dim3(kBlock), 0, st, S, x, vv, F, (T)dth_m, 1, part, cnt, scal, (const int *)state);
        }
        if (cudaGetLastError() != cudaSuccess) return SP_ERR_CUDA;
        if (cudaMemcpyAsync(s->host_state, state, 2 * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return SP_ERR_CUDA;
        if (s->host_state[1] == 0) break;
    }
    // final projection of the velocity (or nothing when no iteration ran)
    launch_pdl(k_vp_move<T>, dim3(nblk), dim3(kBlock), 0, st, N, x, vv, (const rec_t<T> *)F, (T)a.dt, (T)dt2_2m, a.tol,
               a.max_iter, a.max_iter, (const double *)scal, state);
    if (cudaMemcpyAsync(s->host_state, state, 2 * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(s->host_fmax, scal + 2, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SP_ERR_CUDA;
    *iters = s->host_state[0];
    *max_torque = sqrt(*s->host_fmax);
    return 0;
}

// ------------------------------------------------------------ batched VP
// One image per system.  Per system g: scal[8g + kVF, kFF, kFMAX] from the
// last force pass, state[2g] iterations moved, state[2g+1] active flag,
// proj[g] whether the last force pass updated the velocity.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_bvp_force(const BlkInfo *__restrict__ blk, const ImgInfo *__restrict__ img,
                                                      const Stencil<T> *__restrict__ S, const rec_t<T> *__restrict__ x,
                                                      rec_t<T> *__restrict__ v, rec_t<T> *__restrict__ F, T dth_m,
                                                      int mode, double *part, unsigned *cnt, double *scal,
                                                      const int *state, int *proj)
{
    allow_dependents();
    wait_prerequisite();  // state, scalars and records come from the kernels before
    BlkInfo bi = blk[blockIdx.x];
    ImgInfo im = img[bi.g];
    if (mode == 1 && state[2 * bi.g + 1] == 0) return;
    const Stencil<T> &St = S[im.chain];
    int i = bi.t * kBlock + threadIdx.x;
    const rec_t<T> *xb = x + im.spin0;
    T r[3] = {0, 0, 0};
    if (i < im.N) {
        int b;
        long long p = im.spin0 + i;
        v3<T> ni = ld(xb, i);
        v3<T> B = local_field(St, xb, i, ni, b);
        v3<T> Fn = B - dot(B, ni) * ni;
        if (mode == 1) {
            v3<T> vi = axpy(dth_m, ldc(F, p) + Fn, ldc(v, p));
            st(v, p, vi);
            r[0] = dot(vi, Fn);
        }
        st(F, p, Fn);
        r[1] = dot(Fn, Fn);
        r[2] = r[1];
    }
    image_reduce<3>(r, 4u, part, blockIdx.x, im.blk0, im.bpi, cnt + bi.g, scal + kS * bi.g + kVF, ProjectionPost());
    if (bi.t == 0 && threadIdx.x == 0) proj[bi.g] = mode;
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_bvp_move(const BlkInfo *__restrict__ blk, const ImgInfo *__restrict__ img,
                                                     rec_t<T> *__restrict__ x, rec_t<T> *__restrict__ v,
                                                     const rec_t<T> *__restrict__ F, T dt, T dt2_2m, double tol,
                                                     int k, int max_iter, const double *scal, int *state,
                                                     const int *proj)
{
    allow_dependents();
    wait_prerequisite();  // state, scalars and records come from the kernels before
    BlkInfo bi = blk[blockIdx.x];
    ImgInfo im = img[bi.g];
    const double *sc = scal + kS * bi.g;
    __shared__ T s_c;
    __shared__ int s_done;
    if (threadIdx.x == 0) {
        s_c = (T)sc[kC];
        s_done = (sqrt(sc[kFMAX]) < tol) || (k >= max_iter);
    }
    __syncthreads();
    bool done = s_done;
    int i = bi.t * kBlock + threadIdx.x;
    if (i < im.N) {
        long long p = im.spin0 + i;
        v3<T> vi;
        if (proj[bi.g]) {
            T c = s_c;
            vi = c * ldc(F, p);
            st(v, p, vi);
        } else {
            vi = ldc(v, p);
        }
        if (!done) st(x, p, normalised(axpy(dt2_2m, ldc(F, p), axpy(dt, vi, ldc(x, p)))));
    }
    if (bi.t == 0 && threadIdx.x == 0) {
        state[2 * bi.g + 1] = done ? 0 : 1;
        if (!done) state[2 * bi.g] = k + 1;
    }
}

template <typename T>
int vp_batch_run(MinScratch **sp, const std::vector<Stencil<T>> &stencils, const std::vector<long long> &spin0,
                 void *spins, void *vel, const MinArgs &a, int *iters, double *max_torque, cudaStream_t st)
{
    int rc = scratch(sp);
    if (rc) return rc;
    MinScratch *s = *sp;
    int C = (int)stencils.size();
    std::vector<ImgInfo> img;
    std::vector<BlkInfo> blk;
    long long total = 0;
    for (int c = 0; c < C; ++c) {
        int N = stencils[c].N;
        int bpi = blocks_for(N > 0 ? N : 1);
        ImgInfo im{spin0[c], N, c, 0, 1, c, (int)blk.size(), bpi, -1};
        for (int t = 0; t < bpi; ++t) blk.push_back(BlkInfo{c, t});
        img.push_back(im);
        total = std::max(total, spin0[c] + (long long)N);
    }
    int n_full = (int)blk.size();
    size_t rb = sizeof(rec_t<T>) * (size_t)std::max(total, 1LL);
    // blk holds the full table followed by room for a compacted copy
    if (grow(s->F, rb) || grow(s->scal, kS * sizeof(double) * C) || grow(s->part, 3 * sizeof(double) * (size_t)n_full) ||
        grow_counters(s->cnt, C, st) || grow(s->blk, 2 * sizeof(BlkInfo) * n_full) ||
        grow(s->img, sizeof(ImgInfo) * C) || grow(s->sten, sizeof(Stencil<T>) * C) ||
        grow(s->state, sizeof(int) * 3 * C))
        return SP_ERR_CUDA;
    BlkInfo *Bfull = (BlkInfo *)s->blk.p, *Bact = Bfull + n_full;
    ImgInfo *I = (ImgInfo *)s->img.p;
    if (cudaMemcpyAsync(Bfull, blk.data(), sizeof(BlkInfo) * n_full, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(Bact, blk.data(), sizeof(BlkInfo) * n_full, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(I, img.data(), sizeof(ImgInfo) * C, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(s->sten.p, stencils.data(), sizeof(Stencil<T>) * C, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(s->state.p, 0, sizeof(int) * 3 * C, st) != cudaSuccess)
        return SP_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return SP_ERR_CUDA;
    s->layout.clear();  // the GNEB tables were overwritten
    const Stencil<T> *Sd = (const Stencil<T> *)s->sten.p;
    rec_t<T> *x = (rec_t<T> *)spins, *v = (rec_t<T> *)vel, *F = (rec_t<T> *)s->F.p;
    double *scal = (double *)s->scal.p, *part = (double *)s->part.p;
    unsigned *cnt = (unsigned *)s->cnt.p;
    int *state = (int *)s->state.p, *proj = state + 2 * C;
    double dth_m = a.dt / (2.0 * a.mass), dt2_2m = a.dt * a.dt / (2.0 * a.mass);
    std::vector<int> hs(2 * C);
    launch_pdl(k_bvp_force<T>, dim3(n_full), dim3(kBlock), 0, st, (const BlkInfo *)Bfull, (const ImgInfo *)I, Sd,
               (const rec_t<T> *)x, v, F, (T)dth_m, 0, part, cnt, scal, (const int *)state, proj);
    int k = 0, n_act = n_full;
    while (k < a.max_iter) {
        int chunk = std::min(a.check_every, a.max_iter - k);
        for (int c = 0; c < chunk; ++c, ++k) {
            launch_pdl(k_bvp_move<T>, dim3(n_act), dim3(kBlock), 0, st, (const BlkInfo *)Bact, (const ImgInfo *)I, x, v,
                       (const rec_t<T> *)F, (T)a.dt, (T)dt2_2m, a.tol, k, a.max_iter, (const double *)scal, state,
                       (const int *)proj);
            launch_pdl(k_bvp_force<T>, dim3(n_act), dim3(kBlock), 0, st, (const BlkInfo *)Bact, (const ImgInfo *)I, Sd,
                       (const rec_t<T> *)x, v, F, (T)dth_m, 1, part, cnt, scal, (const int *)state, proj);
        }
        if (cudaGetLastError() != cudaSuccess) return SP_ERR_CUDA;
        if (cudaMemcpyAsync(hs.data(), state, sizeof(int) * 2 * C, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return SP_ERR_CUDA;
        // Drop converged systems from the launch tables once a quarter of the
        // launched blocks belongs to them.  A converged system is frozen: its
        // force pass returns at once and its move re-applies the same
        // projection, so leaving it out changes no result.
        std::vector<BlkInfo> act;
        for (int c = 0; c < C; ++c)
            if (hs[2 * c + 1]) {
                img[c].blk0 = (int)act.size();
                for (int t = 0; t < img[c].bpi; ++t) act.push_back(BlkInfo{c, t});
            }
        if (act.empty()) break;
        if (4 * (long long)act.size() <= 3LL * n_act) {
            n_act = (int)act.size();
            if (cudaMemcpyAsync(Bact, act.data(), sizeof(BlkInfo) * n_act, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                cudaMemcpyAsync(I, img.data(), sizeof(ImgInfo) * C, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                return SP_ERR_CUDA;
        }
    }
    // final projection (where the last force pass updated the velocity)
    launch_pdl(k_bvp_move<T>, dim3(n_full), dim3(kBlock), 0, st, (const BlkInfo *)Bfull, (const ImgInfo *)I, x, v,
               (const rec_t<T> *)F, (T)a.dt, (T)dt2_2m, a.tol, a.max_iter, a.max_iter, (const double *)scal, state,
               (const int *)proj);
    std::vector<double> hsc(kS * C);
    if (cudaMemcpyAsync(hs.data(), state, sizeof(int) * 2 * C, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(hsc.data(), scal, sizeof(double) * kS * C, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SP_ERR_CUDA;
    for (int c = 0; c < C; ++c) {
        iters[c] = hs[2 * c];
        max_torque[c] = sqrt(hsc[kS * c + kFMAX]);
    }
    return 0;
}

// ------------------------------------------------------------ GNEB host side
template <typename T>
int gneb_batch_run(MinScratch **sp, const std::vector<Stencil<T>> &stencils, const std::vector<int> &M,
                   const std::vector<long long> &spin0, void *chain, void *vel, const GnebArgs &a, double *E_dev,
                   double *fmax_dev, cudaStream_t st)
{
    int rc = scratch(sp);
    if (rc) return rc;
    MinScratch *s = *sp;
    int C = (int)stencils.size();
    std::vector<ImgInfo> img;
    std::vector<BlkInfo> blk;
    long long total = 0;
    for (int c = 0; c < C; ++c) {
        int N = stencils[c].N;
        int bpi = blocks_for(N > 0 ? N : 1);
        int g0 = (int)img.size();
        for (int nu = 0; nu < M[c]; ++nu) {
            int kind = a.kinds ? a.kinds[g0 + nu] : -1;
            ImgInfo im{spin0[c], N, c, nu, M[c], g0, (int)blk.size(), bpi, kind};
            for (int t = 0; t < bpi; ++t) blk.push_back(BlkInfo{(int)img.size(), t});
            img.push_back(im);
        }
        total = std::max(total, spin0[c] + (long long)M[c] * N);
    }
    int n_img = (int)img.size(), n_blk = (int)blk.size();
    size_t rb = sizeof(rec_t<T>) * (size_t)std::max(total, 1LL);
    if (grow(s->F, rb) || grow(s->G, rb) || grow(s->Tau, rb) || grow(s->scal, kS * sizeof(double) * n_img) ||
        grow(s->part, 3 * sizeof(double) * (size_t)n_blk) || grow_counters(s->cnt, n_img, st) ||
        grow(s->blk, sizeof(BlkInfo) * n_blk) || grow(s->img, sizeof(ImgInfo) * n_img) ||
        grow(s->sten, sizeof(Stencil<T>) * C))
        return SP_ERR_CUDA;
    // upload the tables only when the layout changed (a call with an
    // unchanged layout launches kernels only, so it can be stream-captured)
    std::vector<char> key(sizeof(int) + img.size() * sizeof(ImgInfo) + stencils.size() * sizeof(Stencil<T>));
    int tsz = (int)sizeof(T);
    memcpy(key.data(), &tsz, sizeof(int));
    memcpy(key.data() + sizeof(int), img.data(), img.size() * sizeof(ImgInfo));
    memcpy(key.data() + sizeof(int) + img.size() * sizeof(ImgInfo), stencils.data(), stencils.size() * sizeof(Stencil<T>));
    if (key != s->layout) {
        if (cudaMemcpyAsync(s->blk.p, blk.data(), sizeof(BlkInfo) * n_blk, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(s->img.p, img.data(), sizeof(ImgInfo) * n_img, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(s->sten.p, stencils.data(), sizeof(Stencil<T>) * C, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return SP_ERR_CUDA;
        // the host vectors must outlive the copies above
        if (cudaStreamSynchronize(st) != cudaSuccess) return SP_ERR_CUDA;
        s->layout.swap(key);
    }
    const BlkInfo *B = (const BlkInfo *)s->blk.p;
    const ImgInfo *I = (const ImgInfo *)s->img.p;
    const Stencil<T> *Sd = (const Stencil<T> *)s->sten.p;
    rec_t<T> *x = (rec_t<T> *)chain, *v = (rec_t<T> *)vel;
    rec_t<T> *F = (rec_t<T> *)s->F.p, *G = (rec_t<T> *)s->G.p, *Tau = (rec_t<T> *)s->Tau.p;
    double *scal = (double *)s->scal.p, *part = (double *)s->part.p;
    unsigned *cnt = (unsigned *)s->cnt.p;
    double dth_m = a.dt / (2.0 * a.mass), dt2_2m = a.dt * a.dt / (2.0 * a.mass);
    const int weighted = a.w != 0.0;
    const int ib = (n_img + 127) / 128;
    auto forces = [&](int mode, cudaStream_t ss) {
        k_g_field<T><<<n_blk, kBlock, 0, ss>>>(B, I, Sd, x, G, part, cnt, scal);
        k_g_weights<<<ib, 128, 0, ss>>>(I, n_img, scal);
        k_g_tangent<T><<<n_blk, kBlock, 0, ss>>>(B, I, x, G, Tau, part, cnt, scal);
        if (weighted) k_g_seglen<<<ib, 128, 0, ss>>>(I, n_img, a.w, scal);
        k_g_coef<<<ib, 128, 0, ss>>>(I, n_img, a.k, a.climbing, weighted, scal);
        k_g_force<T><<<n_blk, kBlock, 0, ss>>>(B, I, v, F, G, Tau, dth_m, mode, part, cnt, scal);
    };
    auto iteration = [&](cudaStream_t ss) {
        k_g_move<T><<<n_blk, kBlock, 0, ss>>>(B, I, x, v, F, a.dt, dt2_2m, 1, scal);
        forces(1, ss);
    };
    forces(0, st);
    int remaining = a.n_iter;
    if (remaining > 0 && a.persistent) {
        // every iteration of the call in one cooperative launch; the barrier
        // counter, abort flag and the image tickets start at zero (a launch
        // that gave up may have left tickets behind)
        if (grow(s->sync, 4 * sizeof(unsigned))) return SP_ERR_CUDA;
        int dev = 0, nsm = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_g_persistent<T>, kBlock, 0) != cudaSuccess ||
            per_sm < 1)
            return SP_ERR_CUDA;
        int grid = (int)std::min<long long>((long long)nsm * per_sm, n_blk);
        PersistArgs<T> pa{B, I, Sd, x, v, F, G, Tau, part, scal, cnt, (T)a.dt, (T)dt2_2m, (T)dth_m, n_blk, remaining,
                          0, CoefArgs{a.k, a.w, a.climbing, weighted}, (unsigned *)s->sync.p,
                          (unsigned *)s->sync.p + 1, a.status, a.wait_limit > 0 ? a.wait_limit : (1LL << 21)};
        void *args[] = {&pa};
        if (cudaMemsetAsync(s->sync.p, 0, 4 * sizeof(unsigned), st) != cudaSuccess ||
            cudaMemsetAsync(cnt, 0, sizeof(unsigned) * n_img, st) != cudaSuccess ||
            cudaLaunchCooperativeKernel((const void *)k_g_persistent<T>, dim3(grid), dim3(kBlock), args, 0, st) !=
                cudaSuccess)
            return SP_ERR_CUDA;
        // leave the tickets at zero for the next call whatever happened
        if (cudaMemsetAsync(cnt, 0, sizeof(unsigned) * n_img, st) != cudaSuccess) return SP_ERR_CUDA;
        remaining = 0;
    }
    if (remaining > 0) {
        k_g_move<T><<<n_blk, kBlock, 0, st>>>(B, I, x, v, F, a.dt, dt2_2m, 0, scal);
        forces(1, st);
        --remaining;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return SP_ERR_CUDA;
    if (remaining >= kGraphIters && cap == cudaStreamCaptureStatusNone) {
        // replay kGraphIters iterations per graph launch on a private stream
        if (!s->gstream) {
            if (cudaStreamCreateWithFlags(&s->gstream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&s->ev0, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&s->ev1, cudaEventDisableTiming) != cudaSuccess)
                return SP_ERR_CUDA;
        }
        struct GKey {
            const void *x, *v, *F, *G, *Tau, *scal, *part, *cnt, *blk, *img, *sten;
            double dt, mass, k, w;
            int climbing, n_blk;
        } gk{x, v, F, G, Tau, scal, part, cnt, B, I, Sd, a.dt, a.mass, a.k, a.w, a.climbing, n_blk};
        std::vector<char> gkey(sizeof gk + s->layout.size());
        memcpy(gkey.data(), &gk, sizeof gk);
        memcpy(gkey.data() + sizeof gk, s->layout.data(), s->layout.size());
        if (!s->gexec || gkey != s->gkey) {
            if (s->gexec) cudaGraphExecDestroy(s->gexec);
            s->gexec = nullptr;
            cudaGraph_t graph;
            if (cudaStreamBeginCapture(s->gstream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SP_ERR_CUDA;
            for (int r = 0; r < kGraphIters; ++r) iteration(s->gstream);
            if (cudaStreamEndCapture(s->gstream, &graph) != cudaSuccess) return SP_ERR_CUDA;
            cudaError_t e = cudaGraphInstantiate(&s->gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return SP_ERR_CUDA;
            s->gkey.swap(gkey);
        }
        if (cudaEventRecord(s->ev0, st) != cudaSuccess || cudaStreamWaitEvent(s->gstream, s->ev0, 0) != cudaSuccess)
            return SP_ERR_CUDA;
        for (; remaining >= kGraphIters; remaining -= kGraphIters)
            if (cudaGraphLaunch(s->gexec, s->gstream) != cudaSuccess) return SP_ERR_CUDA;
        if (cudaEventRecord(s->ev1, s->gstream) != cudaSuccess || cudaStreamWaitEvent(st, s->ev1, 0) != cudaSuccess)
            return SP_ERR_CUDA;
    }
    for (; remaining > 0; --remaining) iteration(st);
    if (a.n_iter > 0) k_g_move<T><<<n_blk, kBlock, 0, st>>>(B, I, x, v, F, a.dt, dt2_2m, 2, scal);
    k_g_finish<<<(n_img + 255) / 256, 256, 0, st>>>(I, n_img, scal, E_dev, fmax_dev, C);
    return cudaGetLastError() == cudaSuccess ? 0 : SP_ERR_CUDA;
}

template <typename T>
int gneb_run(MinScratch **s, const Stencil<T> &S, void *chain, void *vel, const GnebArgs &a, double *E_dev,
             double *fmax_dev, cudaStream_t st)
{
    std::vector<Stencil<T>> sv(1, S);
    return gneb_batch_run<T>(s, sv, std::vector<int>{a.M}, std::vector<long long>{0}, chain, vel, a, E_dev, fmax_dev, st);
}

template <typename T>
int gneb_path_scalars(MinScratch **sp, const Stencil<T> &S, const void *chain, int M, double *E, double *dist,
                      double *slope, cudaStream_t st)
{
    int rc = scratch(sp);
    if (rc) return rc;
    if (grow((*sp)->aux, sizeof(double) * (size_t)(M + 1))) return SP_ERR_CUDA;
    double *Ed = (double *)(*sp)->aux.p;
    // zero iterations: energies, distances, tangents and slopes of every
    // image are evaluated and nothing moves (the velocity is not touched)
    GnebArgs a{0.1, 1.0, 0.0, 0, M, 0, nullptr, 0.0};
    std::vector<Stencil<T>> sv(1, S);
    rc = gneb_batch_run<T>(sp, sv, std::vector<int>{M}, std::vector<long long>{0}, const_cast<void *>(chain),
                           const_cast<void *>(chain), a, Ed, Ed + M, st);
    if (rc) return rc;
    std::vector<double> sc(kS * (size_t)M);
    if (cudaMemcpyAsync(sc.data(), (*sp)->scal.p, sizeof(double) * kS * M, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SP_ERR_CUDA;
    for (int g = 0; g < M; ++g) {
        E[g] = sc[kS * g + kE];
        if (g + 1 < M) dist[g] = sqrt(sc[kS * g + kL2]);
        double tt = sc[kS * g + kTT];
        slope[g] = tt > 0 ? sc[kS * g + kGT] / sqrt(tt) : 0.0;
    }
    return 0;
}

#define SPGB_MIN_INST(T)                                                                                               \
    template int gneb_path_scalars<T>(MinScratch **, const Stencil<T> &, const void *, int, double *, double *,         \
                                      double *, cudaStream_t);                                                         \
    template int vp_batch_run<T>(MinScratch **, const std::vector<Stencil<T>> &, const std::vector<long long> &, void *, \
                                 void *, const MinArgs &, int *, double *, cudaStream_t);                              \
    template int vp_minimise<T>(MinScratch **, const Stencil<T> &, void *, void *, const MinArgs &, int *, double *,    \
                                cudaStream_t);                                                                         \
    template int gneb_run<T>(MinScratch **, const Stencil<T> &, void *, void *, const GnebArgs &, double *, double *,   \
                             cudaStream_t);                                                                            \
    template int gneb_batch_run<T>(MinScratch **, const std::vector<Stencil<T>> &, const std::vector<int> &,           \
                                   const std::vector<long long> &, void *, void *, const GnebArgs &, double *,          \
                                   double *, cudaStream_t);
SPGB_MIN_INST(float)
SPGB_MIN_INST(double)

}  // namespace spgb
