// common.cuh -- device-side building blocks of the GB300 spin library:
// storage types, small-vector arithmetic, the neighbour-stencil parameter
// block and the Philox4x32-10 thermal-noise generator.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <stdint.h>

#include "spirit_gb.h"

namespace spgb {

// CODATA 2018 constants in the library's units (meV, T, ps, Angstrom).
constexpr double kMuB = 0.05788381806;            // Bohr magneton, meV/T
constexpr double kBoltzmann = 0.08617333262;      // meV/K
constexpr double kGamma = 0.176085963023;         // electron gyromagnetic ratio, rad/(ps T)
constexpr double kDipole = 0.05368151123574179;   // mu0/(4 pi) mu_B^2 / Angstrom^3, meV

// 4-wide spin records: float4 (16 B) for FP32, a 32-byte aligned double
// quadruple for FP64 (loaded as two 16-byte halves).
struct __align__(32) dq4 {
    double x, y, z, w;
};
template <typename T> struct Rec;
template <> struct Rec<float> { using type = float4; };
template <> struct Rec<double> { using type = dq4; };
template <typename T> using rec_t = typename Rec<T>::type;

template <typename T> struct v3 {
    T x, y, z;
};

template <typename T> __host__ __device__ __forceinline__ v3<T> mk(T x, T y, T z) { return v3<T>{x, y, z}; }
template <typename T> __device__ __forceinline__ v3<T> operator+(v3<T> a, v3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <typename T> __device__ __forceinline__ v3<T> operator-(v3<T> a, v3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename T> __device__ __forceinline__ v3<T> operator*(T s, v3<T> a) { return {s * a.x, s * a.y, s * a.z}; }
template <typename T> __device__ __forceinline__ v3<T> operator-(v3<T> a) { return {-a.x, -a.y, -a.z}; }
template <typename T> __device__ __forceinline__ T dot(v3<T> a, v3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
// dot product accumulated in FP64 (energies of FP32 states)
template <typename T> __device__ __forceinline__ double ddot(v3<T> a, v3<T> b)
{
    return fma((double)a.x, (double)b.x, fma((double)a.y, (double)b.y, (double)a.z * (double)b.z));
}
template <typename T> __device__ __forceinline__ v3<T> cross(v3<T> a, v3<T> b)
{
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
// s*a + b with fused multiply-adds
template <typename T> __device__ __forceinline__ v3<T> axpy(T s, v3<T> a, v3<T> b)
{
    return {fma(s, a.x, b.x), fma(s, a.y, b.y), fma(s, a.z, b.z)};
}
// Maximum that keeps a NaN (fmax drops it): reductions of max torque and
// max force must carry a non-finite value through to the status check.
template <typename T> __device__ __forceinline__ T nan_max(T a, T b) { return (a > b || a != a) ? a : b; }

__device__ __forceinline__ float rnorm(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rnorm(double x) { return rsqrt(x); }
template <typename T> __device__ __forceinline__ v3<T> normalised(v3<T> a)
{
    T r = rnorm(dot(a, a));
    return r * a;
}

__device__ __forceinline__ v3<float> ld(const float4 *p, long i)
{
    float4 v = __ldg(p + i);
    return {v.x, v.y, v.z};
}
__device__ __forceinline__ v3<double> ld(const dq4 *p, long i)
{
    const double2 *q = reinterpret_cast<const double2 *>(p + i);
    double2 a = __ldg(q), b = __ldg(q + 1);
    return {a.x, a.y, b.x};
}
// plain (coherent) loads for buffers written earlier in the same kernel
__device__ __forceinline__ v3<float> ldc(const float4 *p, long i)
{
    float4 v = p[i];
    return {v.x, v.y, v.z};
}
__device__ __forceinline__ v3<double> ldc(const dq4 *p, long i)
{
    const double2 *q = reinterpret_cast<const double2 *>(p + i);
    double2 a = q[0], b = q[1];
    return {a.x, a.y, b.x};
}
// Records held in shared memory: distinct types so that ld/ldc/st resolve to
// plain loads (never the read-only global path of ld above).
struct sh4f {
    float4 v;
};
struct sh4d {
    double2 a, b;
};
template <typename T> struct ShRec;
template <> struct ShRec<float> {
    typedef sh4f type;
};
template <> struct ShRec<double> {
    typedef sh4d type;
};
__device__ __forceinline__ v3<float> ld(const sh4f *p, long i)
{
    float4 v = p[i].v;
    return {v.x, v.y, v.z};
}
__device__ __forceinline__ v3<double> ld(const sh4d *p, long i)
{
    double2 a = p[i].a, b = p[i].b;
    return {a.x, a.y, b.x};
}
__device__ __forceinline__ v3<float> ldc(const sh4f *p, long i) { return ld(p, i); }
__device__ __forceinline__ v3<double> ldc(const sh4d *p, long i) { return ld(p, i); }
__device__ __forceinline__ void st(sh4f *p, long i, v3<float> v) { p[i].v = make_float4(v.x, v.y, v.z, 0.f); }
__device__ __forceinline__ void st(sh4d *p, long i, v3<double> v)
{
    p[i].a = make_double2(v.x, v.y);
    p[i].b = make_double2(v.z, 0.0);
}
__device__ __forceinline__ void st(float4 *p, long i, v3<float> v) { p[i] = make_float4(v.x, v.y, v.z, 0.f); }
__device__ __forceinline__ void st(dq4 *p, long i, v3<double> v)
{
    double2 *q = reinterpret_cast<double2 *>(p + i);
    q[0] = make_double2(v.x, v.y);
    q[1] = make_double2(v.z, 0.0);
}

// ---------------------------------------------------------------- float-float
// An unevaluated sum hi + lo of two floats (about 48 significant bits):
// FP32 sums whose result must match an FP64 sum without the FP64 pipe, which
// is a small fraction of the FP32 rate on this part.  Knuth's TwoSum and
// the FMA-exact product.
struct f2sum {
    float hi, lo;
};
__device__ __forceinline__ f2sum two_sum(float a, float b)
{
    float s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ f2sum operator+(f2sum a, f2sum b)
{
    f2sum s = two_sum(a.hi, b.hi);
    float lo = s.lo + (a.lo + b.lo), hi = s.hi + lo;
    return {hi, lo - (hi - s.hi)};
}
__device__ __forceinline__ bool operator>(f2sum a, f2sum b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ f2sum nan_max(f2sum a, f2sum b) { return (a > b || a.hi != a.hi) ? a : b; }
__device__ __forceinline__ f2sum exact_square(float a) { return {a * a, fmaf(a, a, -(a * a))}; }
__device__ __forceinline__ f2sum exact_dot(v3<float> a, v3<float> b)
{
    float p0 = a.x * b.x, p1 = a.y * b.y, p2 = a.z * b.z;
    return f2sum{p0, fmaf(a.x, b.x, -p0)} + f2sum{p1, fmaf(a.y, b.y, -p1)} + f2sum{p2, fmaf(a.z, b.z, -p2)};
}
__device__ __forceinline__ float shfl_down(float v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_down(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ f2sum shfl_down(f2sum v, int o)
{
    return {__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ double to_double(float v) { return v; }
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(f2sum v) { return (double)v.hi + (double)v.lo; }

// ---------------------------------------------------------------- stencil
// One directed neighbour entry: basis atom jb in cell c + d, exchange J and
// DMI vector D_ij as seen from the centre atom.
template <typename T> struct NbrEntry {
    int jb, d0, d1, d2;
    int lin;  // j - i for a site whose neighbours need no wrap (see Stencil::r0)
    T J, Dx, Dy, Dz;
};

// Division of a non-negative int below 2^31 by a fixed positive divisor d
// as q = (umulhi(n, m) + n) >> s with s = ceil(log2 d) and
// m = floor(2^32 (2^s - d) / d) + 1 (Granlund and Montgomery, PLDI 1994):
// a multiply-high, an add and a shift instead of a full integer division.
struct FastDiv {
    uint32_t m;
    int s, d;
};

inline FastDiv make_fastdiv(int d)
{
    FastDiv f;
    f.d = d;
    f.s = 0;
    while ((1LL << f.s) < (long long)d) ++f.s;
    unsigned long long one = 1;
    f.m = (uint32_t)(((one << 32) * ((one << f.s) - (unsigned long long)d)) / (unsigned long long)d + 1);
    return f;
}

__device__ __forceinline__ int fdiv(int n, const FastDiv &f)
{
    uint32_t t = __umulhi((uint32_t)n, f.m);
    return (int)((t + (uint32_t)n) >> f.s);
}

// Everything a kernel needs to evaluate the local part of Eq. 1 at a spin:
// lattice extents, per-basis on-site terms and the neighbour stencil.  Passed
// by value as a __grid_constant__ kernel parameter (about 3-5 KB).
template <typename T> struct alignas(16) Stencil {
    int nb, n0, n1, n2, per0, per1, per2, N;
    int r0, r1, r2;             // largest |d| of the entries along each direction
    FastDiv fnb, fn0, fn1;      // division by nb, n0, n1
    int off[SP_MAX_BASIS + 1];  // entries of basis b: [off[b], off[b+1])
    T mu[SP_MAX_BASIS];         // mu_b mu_B, meV/T
    T Bz[SP_MAX_BASIS][3];      // Zeeman field mu_b mu_B B, meV
    T K[SP_MAX_BASIS];          // anisotropy K_b, meV
    T Kh[SP_MAX_BASIS][3];      // anisotropy axis
    NbrEntry<T> e[SP_MAX_NBR];
};

static_assert(sizeof(Stencil<float>) % 16 == 0 && sizeof(Stencil<double>) % 16 == 0, "16-byte copies of a stencil");

// Copy of the part of a stencil in global memory that is in use (header and
// the entries of every basis atom) into shared memory, by the whole block;
// the block's later per-neighbour reads then come from shared memory.
template <typename T>
__device__ __forceinline__ void stage_stencil(const Stencil<T> *__restrict__ g, Stencil<T> *s)
{
    const int ne = g->off[g->nb];
    const size_t bytes = offsetof(Stencil<T>, e) + (size_t)ne * sizeof(NbrEntry<T>);
    const int n16 = (int)((bytes + 15) / 16);
    const uint4 *src = reinterpret_cast<const uint4 *>(g);
    uint4 *dst = reinterpret_cast<uint4 *>(s);
    for (int k = threadIdx.x; k < n16; k += blockDim.x) dst[k] = src[k];
    __syncthreads();
}

// Periodic wrap for |d| <= n (checked on the host); -1 across an open edge.
__device__ __forceinline__ int wrap(int x, int n, int per)
{
    if (per) {
        x += (x < 0) ? n : 0;
        x -= (x >= n) ? n : 0;
        return x;
    }
    return (x < 0 || x >= n) ? -1 : x;
}

// Spin index i = b + nb (c0 + n0 (c1 + n1 c2)) -> (b, c0, c1, c2).
template <typename T>
__device__ __forceinline__ void decode_site(const Stencil<T> &S, int i, int &b, int &c0, int &c1, int &c2)
{
    int r = fdiv(i, S.fnb);
    b = i - r * S.nb;
    int r1 = fdiv(r, S.fn0);
    c0 = r - r1 * S.n0;
    c2 = fdiv(r1, S.fn1);
    c1 = r1 - c2 * S.n1;
}

// Local part of B_eff = -dH/dn at spin i (Eq. 1 without the dipole term):
// mu_i B + 2 K (Khat.n_i) Khat + sum_j [J_ij n_j + n_j x D_ij].
// Sites at least r0, r1, r2 cells from every edge take their neighbours at
// the fixed offsets i + lin (the same indices the wrap gives).
// The decision is taken per warp (all active lanes interior), so that a warp
// never runs both index paths: on small lattices most warps touch an edge.
template <typename T>
__device__ __forceinline__ bool interior_site(const Stencil<T> &S, int c0, int c1, int c2)
{
    const bool in = c0 >= S.r0 && c0 < S.n0 - S.r0 && c1 >= S.r1 && c1 < S.n1 - S.r1 && c2 >= S.r2 &&
                    c2 < S.n2 - S.r2;
    return __all_sync(__activemask(), in);
}

// Index of the neighbour of entry E of site i = (b, c0, c1, c2), or -1
// across an open edge.
template <typename T>
__device__ __forceinline__ int nbr_index(const Stencil<T> &S, const NbrEntry<T> &E, int i, bool inner, int c0, int c1,
                                         int c2)
{
    if (inner) return i + E.lin;
    int x0 = wrap(c0 + E.d0, S.n0, S.per0);
    int x1 = wrap(c1 + E.d1, S.n1, S.per1);
    int x2 = wrap(c2 + E.d2, S.n2, S.per2);
    if ((x0 | x1 | x2) < 0) return -1;
    return E.jb + S.nb * (x0 + S.n0 * (x1 + S.n1 * x2));
}

template <typename T, typename R>
__device__ __forceinline__ v3<T> local_field(const Stencil<T> &S, const R *n, int i, v3<T> ni, int &b)
{
    int c0, c1, c2;
    decode_site(S, i, b, c0, c1, c2);
    T kn = dot(mk(S.Kh[b][0], S.Kh[b][1], S.Kh[b][2]), ni);
    T k2 = T(2) * S.K[b] * kn;
    v3<T> B = mk(fma(k2, S.Kh[b][0], S.Bz[b][0]), fma(k2, S.Kh[b][1], S.Bz[b][1]), fma(k2, S.Kh[b][2], S.Bz[b][2]));
    const bool inner = interior_site(S, c0, c1, c2);
    for (int q = S.off[b]; q < S.off[b + 1]; ++q) {
        const NbrEntry<T> &E = S.e[q];
        int j = nbr_index(S, E, i, inner, c0, c1, c2);
        if (j < 0) continue;
        v3<T> nj = ld(n, j);
        v3<T> c = cross(nj, mk(E.Dx, E.Dy, E.Dz));
        B = axpy(E.J, nj, B + c);
    }
    return B;
}

// ---------------------------------------------------------------- launches
// Programmatic dependent launch: a kernel lets the next one on its stream be
// scheduled while it runs (the next kernel's blocks take SMs as they free up
// and do their independent prologue), and a kernel waits for the previous
// one's completion and memory before it reads what that one wrote.  Without
// the launch attribute both are no-ops.
__device__ __forceinline__ void allow_dependents() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
__device__ __forceinline__ void wait_prerequisite() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// Launch a kernel that calls wait_prerequisite() before it reads anything
// written earlier on the stream, with programmatic stream serialisation --
// except into a CUDA graph being captured, where kernel-to-kernel edges are
// already short and programmatic ones measured slower.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return e;
    if (cap != cudaStreamCaptureStatusNone) {
        kern<<<grid, block, smem, st>>>(args...);
        return cudaGetLastError();
    }
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = grid;
    lc.blockDim = block;
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    lc.attrs = at;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, kern, args...);
}

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplications with the published multipliers and Weyl key
// increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// The same with the ten round keys given: rk[2r], rk[2r+1] = key after r
// Weyl steps.
__device__ __forceinline__ uint4 philox4x32_10_keyed(uint4 c, const uint32_t *rk)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 thermal_bits(uint64_t seed, uint64_t step, uint32_t replica, uint32_t i)
{
    return philox4x32_10(make_uint4(i, (uint32_t)step, (uint32_t)(step >> 32), replica * 8u),
                         make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// Three standard normals by Box-Muller: (u0,u1) -> eta_x, eta_y; (u2,u3) ->
// eta_z; u = (x + 1/2) 2^-32.
__device__ __forceinline__ v3<float> box_muller(uint4 x, float)
{
    const float s = 2.3283064365386963e-10f;  // 2^-32
    float u0 = fmaf((float)x.x, s, 0.5f * s), u1 = fmaf((float)x.y, s, 0.5f * s);
    float u2 = fmaf((float)x.z, s, 0.5f * s), u3 = fmaf((float)x.w, s, 0.5f * s);
    float r0 = sqrtf(fmaxf(0.f, -2.f * __logf(u0))), r1 = sqrtf(fmaxf(0.f, -2.f * __logf(u2)));
    float s1, c1;
    sincospif(2.f * u1, &s1, &c1);
    return {r0 * c1, r0 * s1, r1 * cospif(2.f * u3)};
}
__device__ __forceinline__ v3<double> box_muller(uint4 x, double)
{
    const double s = 2.3283064365386963e-10;
    double u0 = ((double)x.x + 0.5) * s, u1 = ((double)x.y + 0.5) * s;
    double u2 = ((double)x.z + 0.5) * s, u3 = ((double)x.w + 0.5) * s;
    double r0 = sqrt(-2.0 * log(u0)), r1 = sqrt(-2.0 * log(u2));
    double s1, c1;
    sincospi(2.0 * u1, &s1, &c1);
    return {r0 * c1, r0 * s1, r1 * cospi(2.0 * u3)};
}

// ---------------------------------------------------------------- LLG
// A(n, B) = c (B + alpha n x B), c = -gamma / ((1 + alpha^2) mu)  (Eq. 3 as dn/dt = n x A)
template <typename T> __device__ __forceinline__ v3<T> llg_A(T c, T alpha, v3<T> n, v3<T> B)
{
    return c * axpy(alpha, cross(n, B), B);
}

// Depondt step: rotate n about -Ahat by |A| dt (Rodrigues' formula).
__device__ __forceinline__ void sincos_(float x, float *s, float *c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_(double x, double *s, double *c) { sincos(x, s, c); }
template <typename T> __device__ __forceinline__ v3<T> rotate(v3<T> n, v3<T> A, T dt)
{
    T w2 = dot(A, A);
    if (w2 == T(0)) return n;
    T iw = rnorm(w2);
    T th = w2 * iw * dt;
    v3<T> ax = (-iw) * A;
    T s, c;
    sincos_(th, &s, &c);
    v3<T> axn = cross(ax, n);
    T an = dot(ax, n);
    // 1 - cos without cancellation for small angles: sin^2 / (1 + cos)
    T omc = c > T(0) ? s * s / (T(1) + c) : T(1) - c;
    // n cos + (ax x n) sin + ax (ax.n)(1 - cos)
    return axpy(an * omc, ax, axpy(s, axn, c * n));
}

// SIB step (Appendix C): the solution of M x = M^T n with M = I + skew(a),
// a = dt A / 2, which Cramer's rule gives in closed form as the Cayley
// rotation x = [(1 - a.a) n + 2 (a.n) a + 2 n x a] / (1 + a.a).
template <typename T> __device__ __forceinline__ v3<T> sib_solve(v3<T> n, v3<T> A, T dt)
{
    v3<T> a = (T(0.5) * dt) * A;
    T aa = dot(a, a), an = dot(a, n);
    v3<T> x = axpy(T(2) * an, a, axpy(T(2), cross(n, a), (T(1) - aa) * n));
    return (T(1) / (T(1) + aa)) * x;
}

}  // namespace spgb
