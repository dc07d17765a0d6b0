// mc.cu -- Metropolis Monte Carlo with cone trial moves (Sec. Monte Carlo):
// sp_mc_sweeps and sp_mc_colours of include/spirit_gb.h.
//
// A sweep visits the colours of a lattice colouring in order: the sum
// colouring (c0 + c1 + c2) mod k where it exists (one basis atom, no bond
// with d0 + d1 + d2 divisible by k, k dividing n0 and the periodic extents
// the bonds cross), else the product colouring (basis atom and, per
// direction, the cell index modulo 2, or modulo 3 for a periodic direction
// of odd size divisible by 3).  Spins of one colour never interact, so all
// spins of a colour of all replicas update in parallel; each update is a
// Metropolis step with the rest fixed, so the chain samples the Boltzmann
// distribution (the paper visits the spins in a random sequential order
// instead).  Trial: a direction uniform on the cap of half-angle theta_cone
// around the spin; acceptance min(1, exp(-dE/kT)).  The three uniforms come
// from Philox4x32-10 with counter (spin, sweep lo, sweep hi, 8 replica + 1)
// -- the thermal field of the LLG uses word 3 = 8 replica, so the streams
// never overlap.
//
// Two launch shapes give the same spins, cones and counts:
//  - resident: one CTA per replica keeps the replica in shared memory for all
//    sweeps of a call (colours separated by block barriers, the cone and the
//    observables updated in the kernel) -- replicas of at most 2048 spins;
//  - one launch per colour over all replicas, then one for the cone feedback
//    (adaptive sweeps) or one for the observables that ends with the cone
//    step (sampled sweeps); the sweep index lives in device memory and is
//    advanced by that last launch, so runs of sweeps replay from a CUDA
//    graph.
#include <cmath>
#include <vector>

#include "ctx.h"

struct McScratch {
    // T: the replicas' temperature factors and cosc the cosines of their
    // cones, both in the compute type; acc: accepted trials of the sweep
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
    int k, res;            // sum colouring: (c0 + c1 + c2) mod k == res; k = 0: the product colouring
    int nk;                // sum colouring: sites of the colour per row (c1, c2), n0 / k
    FastDiv fk;            // division by nk
    FastDiv fkk;           // division by k
    int m0, m1, m2;        // product colouring: moduli per direction
    int off0, off1, off2;  // this colour's residues
    int s0, s1, s2;        // cells of this colour per direction
    int b;                 // basis atom
    long long per;         // spins of this colour per replica
    FastDiv fper;          // division by per (per * replicas < 2^31)
};

// threads of the resident kernel's CTA (FP64: fewer, for the registers)
#ifndef SPGB_MC_RES_BLOCK_F32
#define SPGB_MC_RES_BLOCK_F32 512
#endif
template <typename T> constexpr int kMcResBlock = sizeof(T) == 8 ? 256 : SPGB_MC_RES_BLOCK_F32;
constexpr int kMcMaxResColours = 32;   // colours the resident kernel takes
constexpr int kMcResMaxSweeps = 4096;  // sweeps per resident launch
constexpr int kMcResMaxSpins = 2048;   // largest replica the resident kernel takes
struct McColourSet {
    int n;
    McColour c[kMcMaxResColours];
};

// Philox round keys of the trial stream: key (seed lo, seed hi) advanced by
// the Weyl constants, round r at 2r, 2r + 1 (philox4x32_10_keyed).
struct McKeys {
    uint32_t rk[20];
};
inline McKeys mc_keys(uint64_t seed)
{
    McKeys k;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (uint32_t r = 0; r < 10; ++r) {
        k.rk[2 * r] = k0 + r * 0x9E3779B9u;
        k.rk[2 * r + 1] = k1 + r * 0xBB67AE85u;
    }
    return k;
}

// Spin index of the q-th site of colour col (q < col.per), and its basis
// atom and cell.
template <typename T>
__device__ __forceinline__ int mc_site(const Stencil<T> &S, const McColour &col, int q, int &b, int &c0, int &c1,
                                       int &c2)
{
    if (col.k) {
        const int row = fdiv(q, col.fk);
        c2 = fdiv(row, S.fn1);
        c1 = row - c2 * S.n1;
        const int s = c1 + c2;
        int first = col.res - (s - col.k * fdiv(s, col.fkk));
        first += first < 0 ? col.k : 0;
        c0 = first + col.k * (q - row * col.nk);
        b = 0;
    } else {
        c0 = col.off0 + col.m0 * (q % col.s0);
        q /= col.s0;
        c1 = col.off1 + col.m1 * (q % col.s1);
        q /= col.s1;
        c2 = col.off2 + col.m2 * q;
        b = col.b;
    }
    return b + S.nb * (c0 + S.n0 * (c1 + S.n1 * c2));
}

// The six face bonds of a one-atom lattice whose stencil is exactly the
// faces (+-1 along each direction), in the order +0, -0, +1, -1, +2, -2.
template <typename T> struct McFaces {
    T J[6], D[6][3];
};

// B0 + sum_j [J_ij n_j + n_j x D_ij] over the stencil entries of basis atom
// b at cell (c0, c1, c2) = spin i, neighbours wrapped (periodic) or skipped
// (open).  DMI = false when every D_ij of the stencil vanishes; FACES: the
// stencil is the six faces of F, whose neighbour indices follow from i and
// the strides without the per-entry offsets.
template <bool DMI, bool FACES, typename T, typename R>
__device__ __forceinline__ v3<T> mc_field(const Stencil<T> &S, const McFaces<T> &F, const R *n, int i, int b, int c0,
                                          int c1, int c2, v3<T> B)
{
    if constexpr (FACES) {
        const int s1 = S.n0, s2 = S.n0 * S.n1;
        const int j[6] = {c0 + 1 < S.n0 ? i + 1 : (S.per0 ? i - (S.n0 - 1) : -1),
                          c0 > 0 ? i - 1 : (S.per0 ? i + (S.n0 - 1) : -1),
                          c1 + 1 < S.n1 ? i + s1 : (S.per1 ? i - (S.n1 - 1) * s1 : -1),
                          c1 > 0 ? i - s1 : (S.per1 ? i + (S.n1 - 1) * s1 : -1),
                          c2 + 1 < S.n2 ? i + s2 : (S.per2 ? i - (S.n2 - 1) * s2 : -1),
                          c2 > 0 ? i - s2 : (S.per2 ? i + (S.n2 - 1) * s2 : -1)};
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            if (j[f] < 0) continue;
            const v3<T> nj = ld(n, j[f]);
            if (DMI) B = B + cross(nj, mk(F.D[f][0], F.D[f][1], F.D[f][2]));
            B = axpy(F.J[f], nj, B);
        }
    } else {
        for (int q = S.off[b]; q < S.off[b + 1]; ++q) {
            const NbrEntry<T> &E = S.e[q];
            const int x0 = wrap(c0 + E.d0, S.n0, S.per0), x1 = wrap(c1 + E.d1, S.n1, S.per1),
                      x2 = wrap(c2 + E.d2, S.n2, S.per2);
            if ((x0 | x1 | x2) < 0) continue;
            const v3<T> nj = ld(n, E.jb + S.nb * (x0 + S.n0 * (x1 + S.n1 * x2)));
            if (DMI) B = B + cross(nj, mk(E.Dx, E.Dy, E.Dz));
            B = axpy(E.J, nj, B);
        }
    }
    return B;
}

// The temperature as the trial uses it, 0 for T = 0 (accept only moves that
// lower the energy): FP64 takes kT = k_B T and exp(-dE / kT); FP32 takes
// log2(e) / kT and exp2(-dE log2(e) / kT), the same probability without a
// division.  FP32 draws its azimuth with sincospi(2 u0), FP64 with sin and
// cos of 2 pi u0.
template <typename T> __host__ __device__ __forceinline__ T mc_temp(double Tr);
template <> __host__ __device__ __forceinline__ double mc_temp<double>(double Tr)
{
    return Tr > 0 ? 0.08617333262 * Tr : 0.0;
}
template <> __host__ __device__ __forceinline__ float mc_temp<float>(double Tr)
{
    return Tr > 0 ? (float)(1.4426950408889634 / (0.08617333262 * Tr)) : 0.f;
}
__device__ __forceinline__ bool mc_accept(double u, double dE, double kT)
{
    return kT > 0 ? (u < exp(-dE / kT)) : (dE < 0);
}
__device__ __forceinline__ bool mc_accept(float u, float dE, float l2e_kT)
{
    return l2e_kT > 0.f ? (u < exp2f(-dE * l2e_kT)) : (dE < 0.f);
}
__device__ __forceinline__ void mc_azimuth(double u0, double *s, double *c)
{
    const double ph = 6.283185307179586 * u0;
    *s = sin(ph);
    *c = cos(ph);
}
__device__ __forceinline__ void mc_azimuth(float u0, float *s, float *c) { sincospif(2.f * u0, s, c); }

// One Metropolis trial of spin i = (b, c0, c1, c2) of replica rep (records
// xr: global or shared memory); stores the trial direction when accepted.
// The energy change takes the field's terms linear in n_i (Zeeman, exchange,
// DMI) and the anisotropy exactly.
template <bool DMI, bool FACES, typename T, typename R>
__device__ __forceinline__ bool mc_trial(const Stencil<T> &S, const McFaces<T> &F, R *xr, int i, int b, int c0, int c1,
                                         int c2, int rep, uint64_t sweep, const McKeys &keys, T ct, T temp)
{
    const v3<T> ni = ld(xr, i);
    const v3<T> Bl = mc_field<DMI, FACES>(S, F, xr, i, b, c0, c1, c2, mk(S.Bz[b][0], S.Bz[b][1], S.Bz[b][2]));
    const v3<T> kh = mk(S.Kh[b][0], S.Kh[b][1], S.Kh[b][2]);
    const T kn = dot(kh, ni);
    uint4 o = philox4x32_10_keyed(
        make_uint4((uint32_t)i, (uint32_t)sweep, (uint32_t)(sweep >> 32), 8u * (uint32_t)rep + 1u), keys.rk);
    const T scale = T(2.3283064365386963e-10);
    T u0 = ((T)o.x + T(0.5)) * scale, u1 = ((T)o.y + T(0.5)) * scale, u2 = ((T)o.z + T(0.5)) * scale;
    T cth = T(1) - u1 * (T(1) - ct);
    T sth = sqrt(fmax(T(0), T(1) - cth * cth));
    T sp, cp;
    mc_azimuth(u0, &sp, &cp);
    v3<T> a = fabs(ni.x) >= T(0.9) ? mk(T(0), T(1), T(0)) : mk(T(1), T(0), T(0));
    v3<T> e1 = normalised(a - dot(a, ni) * ni);
    v3<T> e2 = cross(ni, e1);
    v3<T> nt = normalised(cth * ni + sth * (cp * e1 + sp * e2));
    T knt = dot(kh, nt);
    T dE = -(dot(nt, Bl) - dot(ni, Bl)) - S.K[b] * (knt * knt - kn * kn);
    bool ok = mc_accept(u2, dE, temp);
    if (ok) st(xr, i, nt);
    return ok;
}

template <typename T, bool DMI, bool FACES>
__global__ void __launch_bounds__(kMcBlock) k_mc_colour(const __grid_constant__ Stencil<T> S,
                                                        const __grid_constant__ McFaces<T> F, rec_t<T> *__restrict__ x,
                                                        int n_rep, McColour col, const T *__restrict__ temps,
                                                        const T *__restrict__ cosc,
                                                        const unsigned long long *__restrict__ sweep_dev,
                                                        const __grid_constant__ McKeys keys,
                                                        unsigned long long *__restrict__ acc)
{
    __shared__ unsigned cnt[kMcBlock];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    // replicas x spins of a colour stay below 2^31 (checked on the host):
    // 32-bit indices, multiply-high divisions
    const int t0 = (int)blockIdx.x * kMcBlock;  // < total: the grid covers total exactly
    const unsigned t = (unsigned)t0 + threadIdx.x;
    const int rep0 = fdiv(t0, col.fper);
    if (t < (unsigned)col.per * (unsigned)n_rep) {
        const int rep = fdiv((int)t, col.fper);
        int b, c0, c1, c2;
        int i = mc_site(S, col, (int)t - rep * (int)col.per, b, c0, c1, c2);
        // per replica: the cone as its cosine (once per sweep, from FP64) and
        // the temperature factor (once per call): no FP64 work per trial
        if (mc_trial<DMI, FACES>(S, F, x + (long long)rep * S.N, i, b, c0, c1, c2, rep, *sweep_dev, keys, cosc[rep],
                          temps[rep]))
            atomicAdd(&cnt[rep - rep0], 1u);
    }
    __syncthreads();
    unsigned c = cnt[threadIdx.x];
    if (c) atomicAdd(&acc[rep0 + threadIdx.x], (unsigned long long)c);
}

// After a sweep: acceptance into the statistics, the cone's feedback
// (theta <- theta exp(ratio - target), kept in [1e-4, pi]) and the sweep
// counter -- a kernel of its own, or the end of k_mc_sample in sampled
// sweeps (one launch fewer per sweep).
template <typename T> struct McCone {
    unsigned long long *acc;  // accepted trials of the sweep per replica (reset here)
    double *cone;             // cone half-angles
    T *cosc;                  // their cosines in the compute type
    double target;            // target acceptance; 0: the cone stays
    unsigned long long *sweep;
};

template <typename T>
__device__ __forceinline__ void mc_cone_update(const McCone<T> &c, int r, long long N, double *stats)
{
    double a = (double)c.acc[r];
    stats[8 * r + 6] += a;
    stats[8 * r + 7] += (double)N;
    if (c.target > 0) c.cone[r] = fmin(3.141592653589793, fmax(1e-4, c.cone[r] * exp(a / (double)N - c.target)));
    c.cosc[r] = (T)cos(c.cone[r]);
    c.acc[r] = 0;
}

template <typename T>
__global__ void k_mc_cone(int n_rep, long long N, const McCone<T> c, double *stats)
{
    for (int r = threadIdx.x; r < n_rep; r += blockDim.x) mc_cone_update(c, r, N, stats);
    if (threadIdx.x == 0) *c.sweep += 1;
}

template <typename T>
__global__ void k_mc_cos(int n_rep, const double *cone, T *cosc)
{
    for (int r = threadIdx.x; r < n_rep; r += blockDim.x) cosc[r] = (T)cos(cone[r]);
}

// Per-spin observable sums: float-float in FP32 (TwoSum, FMA-exact
// products: the FP64 sum of the same terms to ~1e-14 without the FP64 pipe,
// a small fraction of the FP32 rate on this part), plain FP64 in FP64.
template <typename T> struct McAcc {
    using type = double;
};
template <> struct McAcc<float> {
    using type = f2sum;
};
__device__ __forceinline__ f2sum mc_term(float v) { return f2sum{v, 0.f}; }
__device__ __forceinline__ double mc_term(double v) { return v; }
// energy of spin i, -1/2 n_i.(B_i + mu_i B_ext)
__device__ __forceinline__ f2sum mc_energy(v3<float> n, v3<float> b)
{
    f2sum e = exact_dot(n, b);
    return f2sum{-0.5f * e.hi, -0.5f * e.lo};
}
__device__ __forceinline__ double mc_energy(v3<double> n, v3<double> b) { return -0.5 * dot(n, b); }

// Observables of spin i: sum of n (3 components) and its energy, B the
// local part of B_eff (Eq. 1 without the dipole term).
template <bool DMI, bool FACES, typename T, typename R, typename A>
__device__ __forceinline__ void mc_observe(const Stencil<T> &S, const McFaces<T> &F, const R *xr, int i, A v[4])
{
    const v3<T> ni = ld(xr, i);
    int b, c0, c1, c2;
    decode_site(S, i, b, c0, c1, c2);
    const v3<T> Bz = mk(S.Bz[b][0], S.Bz[b][1], S.Bz[b][2]);
    const T k2 = T(2) * S.K[b] * dot(mk(S.Kh[b][0], S.Kh[b][1], S.Kh[b][2]), ni);
    const v3<T> B = mc_field<DMI, FACES>(
        S, F, xr, i, b, c0, c1, c2,
        mk(fma(k2, S.Kh[b][0], Bz.x), fma(k2, S.Kh[b][1], Bz.y), fma(k2, S.Kh[b][2], Bz.z)));
    v[0] = v[0] + mc_term(ni.x);
    v[1] = v[1] + mc_term(ni.y);
    v[2] = v[2] + mc_term(ni.z);
    v[3] = v[3] + mc_energy(ni, B + Bz);
}

// Observables of every replica: bpr blocks per replica, each summing
// mc_observe over a strided share of its spins (a few per thread: the
// reductions are the cost otherwise); the last block of a replica reduces
// the partials (warp 0, a fixed order) and accumulates m, m^2, m^4, E, E^2
// and the sample count (FP64); with cone.acc set it then takes the sweep's
// cone step of that replica (k_mc_cone).
template <typename T, bool DMI, bool FACES>
__global__ void __launch_bounds__(kMcBlock) k_mc_sample(const __grid_constant__ Stencil<T> S,
                                                        const __grid_constant__ McFaces<T> F,
                                                        const rec_t<T> *__restrict__ x, int bpr, double *part,
                                                        unsigned *tickets, double *stats, const McCone<T> cone)
{
    using A = typename McAcc<T>::type;
    __shared__ double sh[kMcBlock / 32][4];
    __shared__ int last;
    int rep = blockIdx.x / bpr, blk = blockIdx.x - rep * bpr;
    const rec_t<T> *xr = x + (long long)rep * S.N;
    // block blk of the replica takes spins blk * kMcBlock + t + k bpr kMcBlock
    A v[4] = {};
    for (int i = blk * kMcBlock + threadIdx.x; i < S.N; i += bpr * kMcBlock)
        mc_observe<DMI, FACES>(S, F, xr, i, v);
#pragma unroll
    for (int k = 0; k < 4; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] = v[k] + shfl_down(v[k], o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) sh[w][k] = to_double(v[k]);
    }
    __syncthreads();
    if (w == 0) {
        double s[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            s[k] = l < kMcBlock / 32 ? sh[l][k] : 0.0;
            for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_down_sync(0xffffffffu, s[k], o);
        }
        if (l == 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k) part[4 * (size_t)blockIdx.x + k] = s[k];
            __threadfence();
            unsigned tk = atomicAdd(&tickets[rep], 1u);
            last = tk == (unsigned)(bpr - 1);
        }
    }
    __syncthreads();
    if (!last || w != 0) return;
    __threadfence();
    // warp 0 of the replica's last block: lane l sums partials l, l + 32, ...,
    // then the lanes combine (a fixed order)
    double M[4] = {0, 0, 0, 0};
    for (int p = l; p < bpr; p += 32)
#pragma unroll
        for (int k = 0; k < 4; ++k) M[k] += __ldcg(&part[4 * ((size_t)rep * bpr + p) + k]);
#pragma unroll
    for (int k = 0; k < 4; ++k)
        for (int o = 16; o > 0; o >>= 1) M[k] += __shfl_down_sync(0xffffffffu, M[k], o);
    if (l != 0) return;
    double m = sqrt(M[0] * M[0] + M[1] * M[1] + M[2] * M[2]) / (double)S.N;
    double *st = stats + 8 * (size_t)rep;
    st[0] += m;
    st[1] += m * m;
    st[2] += m * m * m * m;
    st[3] += M[3];
    st[4] += M[3] * M[3];
    st[5] += 1;
    tickets[rep] = 0;
    if (cone.acc) {  // the sweep's cone step for this replica
        mc_cone_update(cone, rep, (long long)S.N, stats);
        if (rep == 0) *cone.sweep += 1;
    }
}

// Resident sweeps: CTA r holds replica r in shared memory and runs n_sweeps
// sweeps.  Per sweep: the colours in order (a block barrier after each), then
// one block reduction of the accepted count and, when sampling, of
// mc_observe; warp 0 combines the warps' partials and its lane 0 applies the
// arithmetic of k_mc_cone and k_mc_sample to the replica's cone and
// statistics (FP64, kept in registers between sweeps).  With the cone fixed
// (target 0) the next sweep needs nothing from that update, so the other
// warps go on while lane 0 finishes it.
template <typename T, bool DMI, bool FACES>
__global__ void __launch_bounds__(kMcResBlock<T>) k_mc_resident(const __grid_constant__ Stencil<T> S,
                                                             const __grid_constant__ McFaces<T> F,
                                                             rec_t<T> *__restrict__ x,
                                                             const __grid_constant__ McColourSet cs,
                                                             const T *__restrict__ temps, double *__restrict__ cone,
                                                             double *__restrict__ stats,
                                                             const __grid_constant__ McKeys keys,
                                                             unsigned long long sweep0, int n_sweeps, double target,
                                                             int sample)
{
    using R = typename ShRec<T>::type;
    using A = typename McAcc<T>::type;
    constexpr int kB = kMcResBlock<T>, kW = kB / 32;
    extern __shared__ __align__(16) unsigned char mc_smem[];
    R *sh = reinterpret_cast<R *>(mc_smem);
    __shared__ A red[kW][4];
    __shared__ unsigned red_a[kW];
    __shared__ T ct_sh;
    const int rep = blockIdx.x;
    rec_t<T> *xr = x + (long long)rep * S.N;
    for (int i = threadIdx.x; i < S.N; i += kB) st(sh, i, ld(xr, i));
    const T temp = temps[rep];
    double cn = 0, acc6 = 0, acc7 = 0, st0 = 0, st1 = 0, st2 = 0, st3 = 0, st4 = 0, st5 = 0;
    if (threadIdx.x == 0) {
        const double *sr = stats + 8 * (size_t)rep;
        st0 = sr[0], st1 = sr[1], st2 = sr[2], st3 = sr[3], st4 = sr[4], st5 = sr[5], acc6 = sr[6], acc7 = sr[7];
        cn = cone[rep];
        ct_sh = (T)cos(cn);
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int sw = 0; sw < n_sweeps; ++sw) {
        const uint64_t sweep = sweep0 + (uint64_t)sw;
        const T ct = ct_sh;
        unsigned accepted = 0;
        for (int c = 0; c < cs.n; ++c) {
            const McColour &col = cs.c[c];
            const int per = (int)col.per;
            for (int q = threadIdx.x; q < per; q += kB) {
                int b, c0, c1, c2;
                const int i = mc_site(S, col, q, b, c0, c1, c2);
                accepted += mc_trial<DMI, FACES>(S, F, sh, i, b, c0, c1, c2, rep, sweep, keys, ct, temp) ? 1u : 0u;
            }
            __syncthreads();
        }
        A v[4] = {};
        if (sample)
            for (int i = threadIdx.x; i < S.N; i += kB) mc_observe<DMI, FACES>(S, F, sh, i, v);
        accepted = __reduce_add_sync(0xffffffffu, accepted);
        if (sample) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                for (int o = 16; o > 0; o >>= 1) v[k] = v[k] + shfl_down(v[k], o);
        }
        if (l == 0) {
            red_a[w] = accepted;
#pragma unroll
            for (int k = 0; k < 4; ++k) red[w][k] = v[k];
        }
        __syncthreads();
        if (w == 0) {
            unsigned a = __reduce_add_sync(0xffffffffu, l < kW ? red_a[l] : 0u);
            A M[4] = {};
            if (sample) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    M[k] = l < kW ? red[l][k] : A{};
                    for (int o = 16; o > 0; o >>= 1) M[k] = M[k] + shfl_down(M[k], o);
                }
            }
            if (l == 0) {
                acc6 += (double)a;
                acc7 += (double)S.N;
                if (target > 0) {
                    cn = fmin(3.141592653589793, fmax(1e-4, cn * exp((double)a / (double)S.N - target)));
                    ct_sh = (T)cos(cn);
                }
                if (sample) {
                    const double M0 = to_double(M[0]), M1 = to_double(M[1]), M2 = to_double(M[2]),
                                 M3 = to_double(M[3]);
                    double m = sqrt(M0 * M0 + M1 * M1 + M2 * M2) / (double)S.N;
                    st0 += m;
                    st1 += m * m;
                    st2 += m * m * m * m;
                    st3 += M3;
                    st4 += M3 * M3;
                    st5 += 1;
                }
            }
        }
        // red and red_a are next written after the next sweep's first
        // colour barrier, which warp 0 reaches only once it is done here
        if (target > 0) __syncthreads();
    }
    __syncthreads();
    for (int i = threadIdx.x; i < S.N; i += kB) st(xr, i, ld(sh, i));
    if (threadIdx.x == 0) {
        double *sr = stats + 8 * (size_t)rep;
        sr[0] = st0, sr[1] = st1, sr[2] = st2, sr[3] = st3, sr[4] = st4, sr[5] = st5, sr[6] = acc6, sr[7] = acc7;
        cone[rep] = cn;
    }
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

// The smallest k >= 2 for which (c0 + c1 + c2) mod k is a colouring with
// n0 / k sites of each colour in every row (c1, c2), 0 if there is none: one
// basis atom, k | n0, no bond with d0 + d1 + d2 divisible by k (a bond
// changes the sum by that much), and k dividing the extent of every periodic
// direction a bond crosses (the wrap changes the sum by a multiple of k).
template <typename T>
int mc_sum_modulus(const Stencil<T> &S)
{
    if (S.nb != 1) return 0;
    const int n[3] = {S.n0, S.n1, S.n2}, per[3] = {S.per0, S.per1, S.per2};
    for (int k = 2; k <= S.n0; ++k) {
        if (S.n0 % k) continue;
        bool ok = true;
        for (int q = 0; q < S.off[1] && ok; ++q) {
            const int d[3] = {S.e[q].d0, S.e[q].d1, S.e[q].d2};
            if ((d[0] + d[1] + d[2]) % k == 0) ok = false;
            for (int a = 0; a < 3; ++a)
                if (d[a] && per[a] && n[a] % k) ok = false;
        }
        if (ok) return k;
    }
    return 0;
}

// The sweep's colours in order: the sum colouring when it has no more
// colours than the product colouring (or that one does not exist).
template <typename T>
std::vector<McColour> mc_colours(const Stencil<T> &S)
{
    std::vector<McColour> out;
    int m[3];
    const int prod = mc_moduli(S, m) ? S.nb * m[0] * m[1] * m[2] : 0;
    const int k = mc_sum_modulus(S);
    if (k && (!prod || k <= prod)) {
        for (int r = 0; r < k; ++r) {
            McColour c{};
            c.k = k;
            c.res = r;
            c.nk = S.n0 / k;
            c.fk = make_fastdiv(c.nk);
            c.fkk = make_fastdiv(k);
            c.s0 = c.s1 = c.s2 = 1;
            c.per = (long long)S.N / k;
            c.fper = make_fastdiv((int)c.per);
            out.push_back(c);
        }
        return out;
    }
    if (!prod) return out;
    const int n[3] = {S.n0, S.n1, S.n2};
    // colour index = b + nb (r0 + m0 (r1 + m1 r2)), the oracle's order
    for (int r2 = 0; r2 < m[2]; ++r2)
        for (int r1 = 0; r1 < m[1]; ++r1)
            for (int r0 = 0; r0 < m[0]; ++r0)
                for (int b = 0; b < S.nb; ++b) {
                    McColour c{};
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
                    c.fper = make_fastdiv((int)c.per);
                    out.push_back(c);
                }
    return out;
}

// Shared memory of the resident kernel for one replica; 0 when it does not
// fit (or the colouring is too long for its parameter block).
// Blocks per replica of k_mc_sample: all blocks of all replicas resident at
// once (one wave, the SMs within one block of each other), at most one per
// kMcBlock spins.
template <typename T, bool DMI, bool FACES>
int mc_sample_blocks(int N, int n_rep)
{
    // resident blocks of the kernel on the device (computed once, thread-safe)
    static const int cap = [] {
        int dev = 0, sms = 0, per = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            sms = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mc_sample<T, DMI, FACES>, kMcBlock, 0) !=
                cudaSuccess ||
            per < 1)
            per = 1;
        return sms * per;
    }();
    const int want = cap / n_rep > 0 ? cap / n_rep : 1;
    const int most = (N + kMcBlock - 1) / kMcBlock;
    return want < most ? want : most;
}

template <typename T>
size_t mc_resident_bytes(const Stencil<T> &S, size_t n_colours)
{
    // opt-in shared memory per block (computed once, thread-safe)
    static const int optin = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            v = 0;
        return v;
    }();
    const size_t bytes = sizeof(typename ShRec<T>::type) * (size_t)S.N;
    const size_t reserve = 2048;  // the kernel's static shared memory
    if (n_colours > (size_t)kMcMaxResColours || bytes == 0 || bytes + reserve > (size_t)optin) return 0;
    // one SM per replica pays only while the per-colour launches are bound
    // by their fixed cost: measured on 29 replicas of 10^3 spins the
    // resident sweep takes 8-12 us against 13-21 us, of 15^3 (3 colours)
    // 25-39 us against 18-31 us
    if (S.N > kMcResMaxSpins) return 0;
    return bytes;
}

// True when some pair of the stencil carries a DMI vector.
template <typename T>
bool mc_has_dmi(const Stencil<T> &S)
{
    for (int q = 0; q < S.off[S.nb]; ++q)
        if (S.e[q].Dx != T(0) || S.e[q].Dy != T(0) || S.e[q].Dz != T(0)) return true;
    return false;
}

// The face bonds in the order of McFaces when the stencil is exactly the six
// faces of a one-atom lattice; false otherwise.
template <typename T>
bool mc_faces(const Stencil<T> &S, McFaces<T> &F)
{
    F = McFaces<T>{};
    if (S.nb != 1 || S.off[1] != 6) return false;
    bool seen[6] = {false, false, false, false, false, false};
    for (int q = 0; q < 6; ++q) {
        const NbrEntry<T> &E = S.e[q];
        const int d[3] = {E.d0, E.d1, E.d2};
        int f = -1, nz = 0;
        for (int a = 0; a < 3; ++a)
            if (d[a]) {
                ++nz;
                f = d[a] == 1 ? 2 * a : (d[a] == -1 ? 2 * a + 1 : -1);
            }
        if (E.jb != 0 || nz != 1 || f < 0 || seen[f]) return false;
        seen[f] = true;
        F.J[f] = E.J;
        F.D[f][0] = E.Dx;
        F.D[f][1] = E.Dy;
        F.D[f][2] = E.Dz;
    }
    return true;
}

template <typename T, bool DMI, bool FACES>
int mc_run(sp_ctx *c, const Stencil<T> &S, void *spins, int n_rep, const double *T_host, const sp_mc_params *p,
           int n_sweeps, double *cone, double *stats, cudaStream_t st)
{
    McScratch *&ms = c->mc;
    if (!ms) ms = new McScratch;
    std::vector<McColour> cols = mc_colours(S);
    if (cols.empty()) return SP_ERR_UNSUPPORTED;
    McFaces<T> F;
    mc_faces(S, F);
    const int bpr = mc_sample_blocks<T, DMI, FACES>(S.N, n_rep);
    if (grow_buf(ms->T, sizeof(T) * n_rep) || grow_buf(ms->acc, sizeof(unsigned long long) * (n_rep + kMcBlock)) ||
        grow_buf(ms->sweep, sizeof(unsigned long long)) || grow_buf(ms->part, 4 * sizeof(double) * (size_t)bpr * n_rep) ||
        grow_buf(ms->cnt, sizeof(unsigned) * n_rep) || grow_buf(ms->cosc, sizeof(T) * n_rep))
        return SP_ERR_CUDA;
    unsigned long long s0 = p->sweep0;
    // the trial's temperature factors, once per call on the host
    std::vector<T> temps_host(n_rep);
    for (int r = 0; r < n_rep; ++r) temps_host[r] = mc_temp<T>(T_host[r]);
    if (cudaMemcpyAsync(ms->T.p, temps_host.data(), sizeof(T) * n_rep, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(ms->sweep.p, &s0, sizeof s0, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(ms->acc.p, 0, sizeof(unsigned long long) * (n_rep + kMcBlock), st) != cudaSuccess ||
        cudaMemsetAsync(ms->cnt.p, 0, sizeof(unsigned) * n_rep, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)  // the host values above must outlive the copies
        return SP_ERR_CUDA;
    rec_t<T> *x = (rec_t<T> *)spins;
    const T *temps = (const T *)ms->T.p;
    const McKeys keys = mc_keys(p->seed);
    const size_t res_bytes = c->use_mc_resident ? mc_resident_bytes(S, cols.size()) : 0;
    if (res_bytes && n_sweeps > 0) {
        McColourSet set{};
        set.n = (int)cols.size();
        for (int k = 0; k < set.n; ++k) set.c[k] = cols[k];
        if (cudaFuncSetAttribute(k_mc_resident<T, DMI, FACES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)res_bytes) != cudaSuccess)
            return SP_ERR_CUDA;
        for (int k = 0; k < n_sweeps; k += kMcResMaxSweeps) {
            const int ns = n_sweeps - k < kMcResMaxSweeps ? n_sweeps - k : kMcResMaxSweeps;
            k_mc_resident<T, DMI, FACES><<<(unsigned)n_rep, kMcResBlock<T>, res_bytes, st>>>(S, F, x, set, temps, cone,
                                                                                     stats, keys,
                                                                              s0 + (unsigned long long)k, ns,
                                                                              p->target_accept, p->sample);
        }
        return cudaGetLastError() == cudaSuccess ? 0 : SP_ERR_CUDA;
    }
    T *cosc = (T *)ms->cosc.p;
    k_mc_cos<T><<<1, 256, 0, st>>>(n_rep, cone, cosc);
    unsigned long long *acc = (unsigned long long *)ms->acc.p, *sw = (unsigned long long *)ms->sweep.p;
    double *part = (double *)ms->part.p;
    unsigned *tk = (unsigned *)ms->cnt.p;
    auto sweep = [&](cudaStream_t ss) {
        for (const McColour &col : cols) {
            long long work = col.per * n_rep;
            k_mc_colour<T, DMI, FACES><<<(unsigned)((work + kMcBlock - 1) / kMcBlock), kMcBlock, 0, ss>>>(
                S, F, x, n_rep, col, temps, cosc, sw, keys, acc);
        }
        const McCone<T> cc{acc, cone, cosc, p->target_accept, sw};
        if (p->sample)
            k_mc_sample<T, DMI, FACES><<<(unsigned)(bpr * n_rep), kMcBlock, 0, ss>>>(S, F, x, bpr, part, tk, stats, cc);
        else
            k_mc_cone<T><<<1, 256, 0, ss>>>(n_rep, (long long)S.N, cc, stats);
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
        } key{x, cone, stats, temps, acc, sw, part, tk, cosc, p->seed, p->target_accept, p->sample, n_rep, (int)sizeof(T)};
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

// mc_run for the field variant the stencil allows.
template <typename T>
int mc_dispatch(sp_ctx *c, const Stencil<T> &S, void *spins, int n_rep, const double *T_host, const sp_mc_params *p,
                int n_sweeps, double *cone, double *stats, cudaStream_t st)
{
    McFaces<T> F;
    const bool dmi = mc_has_dmi(S), faces = mc_faces(S, F);
    auto run = dmi ? (faces ? mc_run<T, true, true> : mc_run<T, true, false>)
                   : (faces ? mc_run<T, false, true> : mc_run<T, false, false>);
    return run(c, S, spins, n_rep, T_host, p, n_sweeps, cone, stats, st);
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
    const bool dmi = mc_has_dmi(S);
    McFaces<T> F;
    const bool faces = mc_faces(S, F);
    const int bpr = dmi ? (faces ? mc_sample_blocks<T, true, true>(S.N, n_rep) : mc_sample_blocks<T, true, false>(S.N, n_rep))
                        : (faces ? mc_sample_blocks<T, false, true>(S.N, n_rep)
                                 : mc_sample_blocks<T, false, false>(S.N, n_rep));
    if (grow_buf(ms->part, 4 * sizeof(double) * (size_t)bpr * n_rep) || grow_buf(ms->cnt, sizeof(unsigned) * n_rep) ||
        cudaMemsetAsync(ms->cnt.p, 0, sizeof(unsigned) * n_rep, st) != cudaSuccess)
        return SP_ERR_CUDA;
    auto kern = dmi ? (faces ? k_mc_sample<T, true, true> : k_mc_sample<T, true, false>)
                    : (faces ? k_mc_sample<T, false, true> : k_mc_sample<T, false, false>);
    kern<<<(unsigned)(bpr * n_rep), kMcBlock, 0, st>>>(S, F, (const rec_t<T> *)spins, bpr, (double *)ms->part.p,
                                                       (unsigned *)ms->cnt.p, stats, McCone<T>{});
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
    if ((uintptr_t)spins_dev % (c->prec == SP_F64 ? 32 : 16)) return mfail(c, SP_ERR_ARG, "spins misaligned");
    if ((uintptr_t)cone_dev % 8 || (uintptr_t)stats_dev % 8) return mfail(c, SP_ERR_ARG, "cone or stats misaligned");
    if (n_rep < 1 || n_sweeps < 0) return mfail(c, SP_ERR_ARG, "n_rep >= 1 and n_sweeps >= 0 required");
    if ((long long)n_rep * c->N >= (1LL << 31)) return mfail(c, SP_ERR_ARG, "more than 2^31 spins");
    if (!(p->target_accept >= 0 && p->target_accept < 1)) return mfail(c, SP_ERR_ARG, "target_accept in [0, 1) required");
    for (int r = 0; r < n_rep; ++r)
        if (!(T[r] >= 0)) return mfail(c, SP_ERR_ARG, "temperatures must be >= 0");
    if (c->h.dipole != SP_DIPOLE_NONE) return mfail(c, SP_ERR_UNSUPPORTED, "Monte Carlo with the dipole term");
    if (int rc = status_enter(c)) return rc;
    int e = c->prec == SP_F64
                ? mc_dispatch<double>(c, c->Sd, spins_dev, n_rep, T, p, n_sweeps, cone_dev, stats_dev,
                                      (cudaStream_t)stream)
                : mc_dispatch<float>(c, c->Sf, spins_dev, n_rep, T, p, n_sweeps, cone_dev, stats_dev,
                                     (cudaStream_t)stream);
    if (e == SP_ERR_UNSUPPORTED)
        return mfail(c, e, "lattice has no colouring (neither (c0 + c1 + c2) mod k nor the product colouring "
                           "applies)");
    if (e) return mfail(c, e, "Monte Carlo launch failed");
    return status_check_records(c, spins_dev, (long)n_rep * c->N, SITE_STATE, (cudaStream_t)stream);
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
    if (int rc = status_enter(c)) return rc;
    int e = c->prec == SP_F64 ? sample_run<double>(c, c->Sd, spins_dev, n_rep, stats_dev, (cudaStream_t)stream)
                              : sample_run<float>(c, c->Sf, spins_dev, n_rep, stats_dev, (cudaStream_t)stream);
    if (e) return mfail(c, e, "observable sampling launch failed");
    return status_check_doubles(c, stats_dev, 8L * n_rep, SITE_SAMPLE, (cudaStream_t)stream);
}

}  // extern "C"
