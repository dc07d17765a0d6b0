// mc.cu -- Metropolis Monte Carlo with cone trial moves (Sec. Monte Carlo):
// sp_mc_sweeps and sp_mc_colours of include/spirit_gb.h.
//
// A sweep visits the colours of a lattice colouring in order (colour =
// basis atom and, per direction, the cell index modulo 2, or modulo 3 for a
// periodic direction of odd size divisible by 3).  Spins of one colour never
// interact, so one launch updates all spins of a colour of all replicas in
// parallel; each update is a Metropolis step with the rest fixed, so the
// chain samples the Boltzmann distribution (the paper visits the spins in a
// random sequential order instead).  Trial: a direction uniform on the cap of
// half-angle theta_cone around the spin; acceptance min(1, exp(-dE/kT)).
// The three uniforms come from Philox4x32-10 with counter (spin, sweep lo,
// sweep hi, 8 replica + 1) -- the thermal field of the LLG uses word 3 =
// 8 replica, so the streams never overlap.  The sweep index lives in device
// memory and is advanced by the cone kernel, so runs of sweeps are replayed
// from a CUDA graph.
#include <cmath>
#include <vector>

#include "ctx.h"

struct McScratch {
    DevBuf T, acc, sweep, part, cnt, cosc;
    cudaStream_t gs = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<char> gkey;
};

namespace {

constexpr int kMcBlock = 256;
constexpr int kMcGraphSweeps = 16;

struct McColour {
    int m0, m1, m2;        // moduli per direction
    int off0, off1, off2;  // this colour's residues
    int s0, s1, s2;        // cells of this colour per direction
    int b;                 // basis atom
    long long per;         // spins of this colour per replica
};

template <typename T>
__global__ void __launch_bounds__(kMcBlock) k_mc_colour(const __grid_constant__ Stencil<T> S, rec_t<T> *__restrict__ x,
                                                        int n_rep, McColour col, const double *__restrict__ TK,
                                                        const double *__restrict__ cosc,
                                                        const unsigned long long *__restrict__ sweep_dev,
                                                        uint64_t seed, unsigned long long *__restrict__ acc)
{
    __shared__ unsigned cnt[kMcBlock];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    long long t0 = (long long)blockIdx.x * kMcBlock;
    long long t = t0 + threadIdx.x;
    int rep0 = (int)(t0 / col.per);
    if (t < col.per * n_rep) {
        int rep = (int)(t / col.per);
        long long q = t - (long long)rep * col.per;
        int c0 = col.off0 + col.m0 * (int)(q % col.s0);
        q /= col.s0;
        int c1 = col.off1 + col.m1 * (int)(q % col.s1);
        q /= col.s1;
        int c2 = col.off2 + col.m2 * (int)q;
        int i = col.b + S.nb * (c0 + S.n0 * (c1 + S.n1 * c2));
        rec_t<T> *xr = x + (long long)rep * S.N;
        v3<T> ni = ld(xr, i);
        int b;
        v3<T> B = local_field(S, xr, i, ni, b);
        // the field's terms linear in n_i (Zeeman, exchange, DMI): remove the
        // anisotropy part, whose energy change is taken exactly below
        v3<T> kh = mk(S.Kh[b][0], S.Kh[b][1], S.Kh[b][2]);
        T kn = dot(kh, ni);
        v3<T> Bl = B - (T(2) * S.K[b] * kn) * kh;
        uint64_t sweep = *sweep_dev;
        uint4 o = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)sweep, (uint32_t)(sweep >> 32), 8u * (uint32_t)rep + 1u),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
        const T scale = T(2.3283064365386963e-10);
        T u0 = ((T)o.x + T(0.5)) * scale, u1 = ((T)o.y + T(0.5)) * scale, u2 = ((T)o.z + T(0.5)) * scale;
        T ct = (T)cosc[rep];  // cos of the replica's cone angle
        T cth = T(1) - u1 * (T(1) - ct);
        T sth = sqrt(fmax(T(0), T(1) - cth * cth));
        T ph = T(6.283185307179586) * u0;
        v3<T> a = fabs(ni.x) >= T(0.9) ? mk(T(0), T(1), T(0)) : mk(T(1), T(0), T(0));
        v3<T> e1 = normalised(a - dot(a, ni) * ni);
        v3<T> e2 = cross(ni, e1);
        v3<T> nt = normalised(cth * ni + sth * (cos(ph) * e1 + sin(ph) * e2));
        T knt = dot(kh, nt);
        T dE = -(dot(nt, Bl) - dot(ni, Bl)) - S.K[b] * (knt * knt - kn * kn);
        double Tr = TK[rep];
        bool ok = Tr > 0 ? (u2 < exp(-dE / (T)(0.08617333262 * Tr))) : (dE < T(0));
        if (ok) {
            st(xr, i, nt);
            atomicAdd(&cnt[rep - rep0], 1u);
        }
    }
    __syncthreads();
    unsigned c = cnt[threadIdx.x];
    if (c) atomicAdd(&acc[rep0 + threadIdx.x], (unsigned long long)c);
}

// After a sweep: acceptance into the statistics, the cone's feedback
// (theta <- theta exp(ratio - target), kept in [1e-4, pi]) and the sweep
// counter.
__global__ void k_mc_cone(int n_rep, long long N, unsigned long long *acc, double *cone, double *cosc, double target,
                          double *stats, unsigned long long *sweep_dev)
{
    for (int r = threadIdx.x; r < n_rep; r += blockDim.x) {
        double a = (double)acc[r];
        stats[8 * r + 6] += a;
        stats[8 * r + 7] += (double)N;
        if (target > 0) cone[r] = fmin(3.141592653589793, fmax(1e-4, cone[r] * exp(a / (double)N - target)));
        cosc[r] = cos(cone[r]);
        acc[r] = 0;
    }
    if (threadIdx.x == 0) *sweep_dev += 1;
}

__global__ void k_mc_cos(int n_rep, const double *cone, double *cosc)
{
    for (int r = threadIdx.x; r < n_rep; r += blockDim.x) cosc[r] = cos(cone[r]);
}

// Observables of every replica: sum of n (3 components) and the energy
// -1/2 n.(B + mu B_ext) per spin, FP64 sums; the last block of a replica
// reduces its partials in a fixed order and accumulates m, m^2, m^4, E, E^2
// and the sample count.
template <typename T>
__global__ void __launch_bounds__(kMcBlock) k_mc_sample(const __grid_constant__ Stencil<T> S,
                                                        const rec_t<T> *__restrict__ x, int bpr, double *part,
                                                        unsigned *tickets, double *stats)
{
    __shared__ double sh[kMcBlock / 32][4];
    __shared__ int last;
    int rep = blockIdx.x / bpr, blk = blockIdx.x - rep * bpr;
    int i = blk * kMcBlock + threadIdx.x;
    const rec_t<T> *xr = x + (long long)rep * S.N;
    double v[4] = {0, 0, 0, 0};
    if (i < S.N) {
        v3<T> ni = ld(xr, i);
        int b;
        v3<T> B = local_field(S, xr, i, ni, b);
        v3<T> Bz = mk(S.Bz[b][0], S.Bz[b][1], S.Bz[b][2]);
        v[0] = (double)ni.x;
        v[1] = (double)ni.y;
        v[2] = (double)ni.z;
        v[3] = -0.5 * ddot(ni, B + Bz);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
        for (int k = 0; k < 4; ++k) sh[w][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < 4; ++k) {
            double s = 0;
            for (int ww = 0; ww < kMcBlock / 32; ++ww) s += sh[ww][k];
            part[4 * (size_t)blockIdx.x + k] = s;
        }
        __threadfence();
        unsigned tk = atomicAdd(&tickets[rep], 1u);
        last = tk == (unsigned)(bpr - 1);
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double M[4] = {0, 0, 0, 0};
    for (int p = 0; p < bpr; ++p)
        for (int k = 0; k < 4; ++k) M[k] += __ldcg(&part[4 * ((size_t)rep * bpr + p) + k]);
    double m = sqrt(M[0] * M[0] + M[1] * M[1] + M[2] * M[2]) / (double)S.N;
    double *st = stats + 8 * (size_t)rep;
    st[0] += m;
    st[1] += m * m;
    st[2] += m * m * m * m;
    st[3] += M[3];
    st[4] += M[3] * M[3];
    st[5] += 1;
    tickets[rep] = 0;
}

int grow_buf(DevBuf &b, size_t bytes)
{
    if (b.p && b.bytes >= bytes) return 0;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) return SP_ERR_CUDA;
    b.bytes = bytes;
    return 0;
}

// Per-direction moduli of the colouring; false when the lattice has none.
template <typename T>
bool mc_moduli(const Stencil<T> &S, int m[3])
{
    const int n[3] = {S.n0, S.n1, S.n2}, per[3] = {S.per0, S.per1, S.per2};
    for (int d = 0; d < 3; ++d) {
        bool any = false;
        for (int q = 0; q < S.off[S.nb]; ++q) {
            int dd = d == 0 ? S.e[q].d0 : (d == 1 ? S.e[q].d1 : S.e[q].d2);
            if (dd > 1 || dd < -1) return false;
            if (dd) any = true;
        }
        if (n[d] == 1) {
            if (any) return false;
            m[d] = 1;
        } else if (!per[d] || n[d] % 2 == 0) {
            m[d] = 2;
        } else if (n[d] % 3 == 0) {
            m[d] = 3;
        } else {
            return false;
        }
    }
    return true;
}

template <typename T>
std::vector<McColour> mc_colours(const Stencil<T> &S)
{
    std::vector<McColour> out;
    int m[3];
    if (!mc_moduli(S, m)) return out;
    const int n[3] = {S.n0, S.n1, S.n2};
    // colour index = b + nb (r0 + m0 (r1 + m1 r2)), the oracle's order
    for (int r2 = 0; r2 < m[2]; ++r2)
        for (int r1 = 0; r1 < m[1]; ++r1)
            for (int r0 = 0; r0 < m[0]; ++r0)
                for (int b = 0; b < S.nb; ++b) {
                    McColour c;
                    c.m0 = m[0];
                    c.m1 = m[1];
                    c.m2 = m[2];
                    c.off0 = r0;
                    c.off1 = r1;
                    c.off2 = r2;
                    c.s0 = (n[0] - r0 + m[0] - 1) / m[0];
                    c.s1 = (n[1] - r1 + m[1] - 1) / m[1];
                    c.s2 = (n[2] - r2 + m[2] - 1) / m[2];
                    c.b = b;
                    c.per = (long long)c.s0 * c.s1 * c.s2;
                    out.push_back(c);
                }
    return out;
}

template <typename T>
int mc_run(sp_ctx *c, const Stencil<T> &S, void *spins, int n_rep, const double *T_host, const sp_mc_params *p,
           int n_sweeps, double *cone, double *stats, cudaStream_t st)
{
    McScratch *&ms = c->mc;
    if (!ms) ms = new McScratch;
    std::vector<McColour> cols = mc_colours(S);
    if (cols.empty()) return SP_ERR_UNSUPPORTED;
    int bpr = (S.N + kMcBlock - 1) / kMcBlock;
    if (grow_buf(ms->T, sizeof(double) * n_rep) || grow_buf(ms->acc, sizeof(unsigned long long) * (n_rep + kMcBlock)) ||
        grow_buf(ms->sweep, sizeof(unsigned long long)) || grow_buf(ms->part, 4 * sizeof(double) * (size_t)bpr * n_rep) ||
        grow_buf(ms->cnt, sizeof(unsigned) * n_rep) || grow_buf(ms->cosc, sizeof(double) * n_rep))
        return SP_ERR_CUDA;
    unsigned long long s0 = p->sweep0;
    if (cudaMemcpyAsync(ms->T.p, T_host, sizeof(double) * n_rep, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(ms->sweep.p, &s0, sizeof s0, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(ms->acc.p, 0, sizeof(unsigned long long) * (n_rep + kMcBlock), st) != cudaSuccess ||
        cudaMemsetAsync(ms->cnt.p, 0, sizeof(unsigned) * n_rep, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)  // the host values above must outlive the copies
        return SP_ERR_CUDA;
    rec_t<T> *x = (rec_t<T> *)spins;
    const double *TK = (const double *)ms->T.p;
    double *cosc = (double *)ms->cosc.p;
    k_mc_cos<<<1, 256, 0, st>>>(n_rep, cone, cosc);
    unsigned long long *acc = (unsigned long long *)ms->acc.p, *sw = (unsigned long long *)ms->sweep.p;
    double *part = (double *)ms->part.p;
    unsigned *tk = (unsigned *)ms->cnt.p;
    auto sweep = [&](cudaStream_t ss) {
        for (const McColour &col : cols) {
            long long work = col.per * n_rep;
            k_mc_colour<T><<<(unsigned)((work + kMcBlock - 1) / kMcBlock), kMcBlock, 0, ss>>>(S, x, n_rep, col, TK, cosc,
                                                                                            sw, p->seed, acc);
        }
        k_mc_cone<<<1, 256, 0, ss>>>(n_rep, (long long)S.N, acc, cone, cosc, p->target_accept, stats, sw);
        if (p->sample) k_mc_sample<T><<<(unsigned)(bpr * n_rep), kMcBlock, 0, ss>>>(S, x, bpr, part, tk, stats);
    };
    int k = 0;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return SP_ERR_CUDA;
    if (n_sweeps >= kMcGraphSweeps && cap == cudaStreamCaptureStatusNone) {
        if (!ms->gs) {
            if (cudaStreamCreateWithFlags(&ms->gs, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&ms->e0, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&ms->e1, cudaEventDisableTiming) != cudaSuccess)
                return SP_ERR_CUDA;
        }
        struct Key {
            const void *x, *cone, *stats, *temps, *acc, *sw, *part, *cnt, *cosc;
            uint64_t seed;
            double target;
            int sample, n_rep, prec;
        } key{x, cone, stats, TK, acc, sw, part, tk, cosc, p->seed, p->target_accept, p->sample, n_rep, (int)sizeof(T)};
        std::vector<char> gk(sizeof key + sizeof(Stencil<T>));
        memcpy(gk.data(), &key, sizeof key);
        memcpy(gk.data() + sizeof key, &S, sizeof(Stencil<T>));
        if (!ms->gexec || gk != ms->gkey) {
            if (ms->gexec) cudaGraphExecDestroy(ms->gexec);
            ms->gexec = nullptr;
            cudaGraph_t g;
            if (cudaStreamBeginCapture(ms->gs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SP_ERR_CUDA;
            for (int r = 0; r < kMcGraphSweeps; ++r) sweep(ms->gs);
            if (cudaStreamEndCapture(ms->gs, &g) != cudaSuccess) return SP_ERR_CUDA;
            cudaError_t e = cudaGraphInstantiate(&ms->gexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return SP_ERR_CUDA;
            ms->gkey.swap(gk);
        }
        if (cudaEventRecord(ms->e0, st) != cudaSuccess || cudaStreamWaitEvent(ms->gs, ms->e0, 0) != cudaSuccess)
            return SP_ERR_CUDA;
        for (; k + kMcGraphSweeps <= n_sweeps; k += kMcGraphSweeps)
            if (cudaGraphLaunch(ms->gexec, ms->gs) != cudaSuccess) return SP_ERR_CUDA;
        if (cudaEventRecord(ms->e1, ms->gs) != cudaSuccess || cudaStreamWaitEvent(st, ms->e1, 0) != cudaSuccess)
            return SP_ERR_CUDA;
    }
    for (; k < n_sweeps; ++k) sweep(st);
    return cudaGetLastError() == cudaSuccess ? 0 : SP_ERR_CUDA;
}

int mfail(sp_ctx *c, int code, const char *msg)
{
    c->err = msg;
    return code;
}

// Observables of n_rep replicas accumulated into stats (sp_sample).
template <typename T>
int sample_run(sp_ctx *c, const Stencil<T> &S, const void *spins, int n_rep, double *stats, cudaStream_t st)
{
    McScratch *&ms = c->mc;
    if (!ms) ms = new McScratch;
    int bpr = (S.N + kMcBlock - 1) / kMcBlock;
    if (grow_buf(ms->part, 4 * sizeof(double) * (size_t)bpr * n_rep) || grow_buf(ms->cnt, sizeof(unsigned) * n_rep) ||
        cudaMemsetAsync(ms->cnt.p, 0, sizeof(unsigned) * n_rep, st) != cudaSuccess)
        return SP_ERR_CUDA;
    k_mc_sample<T><<<(unsigned)(bpr * n_rep), kMcBlock, 0, st>>>(S, (const rec_t<T> *)spins, bpr, (double *)ms->part.p,
                                                                 (unsigned *)ms->cnt.p, stats);
    return cudaGetLastError() == cudaSuccess ? 0 : SP_ERR_CUDA;
}

}  // namespace

void mc_scratch_destroy(McScratch *m)
{
    if (!m) return;
    DevBuf *bufs[] = {&m->T, &m->acc, &m->sweep, &m->part, &m->cnt, &m->cosc};
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    if (m->gexec) cudaGraphExecDestroy(m->gexec);
    if (m->gs) cudaStreamDestroy(m->gs);
    if (m->e0) cudaEventDestroy(m->e0);
    if (m->e1) cudaEventDestroy(m->e1);
    delete m;
}

extern "C" {

int sp_mc_colours(sp_ctx *c, int *n_colours)
{
    if (!c || !n_colours) return SP_ERR_ARG;
    if (!c->have_geom || !c->have_ham) return mfail(c, SP_ERR_STATE, "context not configured");
    *n_colours = (int)(c->prec == SP_F64 ? mc_colours(c->Sd).size() : mc_colours(c->Sf).size());
    return SP_OK;
}

int sp_mc_sweeps(sp_ctx *c, void *spins_dev, int n_rep, const double *T, const sp_mc_params *p, int n_sweeps,
                 double *cone_dev, double *stats_dev, void *stream)
{
    if (!c) return SP_ERR_ARG;
    if (!c->have_geom || !c->have_ham) return mfail(c, SP_ERR_STATE, "context not configured");
    if (!spins_dev || !T || !p || !cone_dev || !stats_dev) return mfail(c, SP_ERR_ARG, "NULL argument");
    if (n_rep < 1 || n_sweeps < 0) return mfail(c, SP_ERR_ARG, "n_rep >= 1 and n_sweeps >= 0 required");
    if ((long long)n_rep * c->N >= (1LL << 31)) return mfail(c, SP_ERR_ARG, "more than 2^31 spins");
    if (!(p->target_accept >= 0 && p->target_accept < 1)) return mfail(c, SP_ERR_ARG, "target_accept in [0, 1) required");
    for (int r = 0; r < n_rep; ++r)
        if (!(T[r] >= 0)) return mfail(c, SP_ERR_ARG, "temperatures must be >= 0");
    if (c->h.dipole != SP_DIPOLE_NONE) return mfail(c, SP_ERR_UNSUPPORTED, "Monte Carlo with the dipole term");
    int e = c->prec == SP_F64
                ? mc_run<double>(c, c->Sd, spins_dev, n_rep, T, p, n_sweeps, cone_dev, stats_dev, (cudaStream_t)stream)
                : mc_run<float>(c, c->Sf, spins_dev, n_rep, T, p, n_sweeps, cone_dev, stats_dev, (cudaStream_t)stream);
    if (e == SP_ERR_UNSUPPORTED)
        return mfail(c, e, "lattice has no colouring (a neighbour beyond the next cell, or an odd periodic size not "
                           "divisible by 3)");
    if (e) return mfail(c, e, "Monte Carlo launch failed");
    return SP_OK;
}

int sp_sample(sp_ctx *c, const void *spins_dev, int n_rep, double *stats_dev, void *stream)
{
    if (!c) return SP_ERR_ARG;
    if (!c->have_geom || !c->have_ham) return mfail(c, SP_ERR_STATE, "context not configured");
    if (!spins_dev || !stats_dev) return mfail(c, SP_ERR_ARG, "NULL argument");
    if ((uintptr_t)spins_dev % (c->prec == SP_F64 ? 32 : 16)) return mfail(c, SP_ERR_ARG, "spins misaligned");
    if (n_rep < 1) return mfail(c, SP_ERR_ARG, "n_rep must be >= 1");
    if ((long long)n_rep * c->N >= (1LL << 31)) return mfail(c, SP_ERR_ARG, "more than 2^31 spins");
    if (c->h.dipole != SP_DIPOLE_NONE) return mfail(c, SP_ERR_UNSUPPORTED, "observables with the dipole term");
    if (c->N == 0) return SP_OK;
    int e = c->prec == SP_F64 ? sample_run<double>(c, c->Sd, spins_dev, n_rep, stats_dev, (cudaStream_t)stream)
                              : sample_run<float>(c, c->Sf, spins_dev, n_rep, stats_dev, (cudaStream_t)stream);
    if (e) return mfail(c, e, "observable sampling launch failed");
    return SP_OK;
}

}  // extern "C"
