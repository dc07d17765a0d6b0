// dipole.cu -- dipole-dipole field by zero-padded FFT convolution on a 2D
// lattice with one basis atom (Sec. "Dipolar interactions").
//
//   B_i = C mu_i sum_{j != i} mu_j (3 rhat (rhat.n_j) - n_j) / r^3
//       = IFFT( Khat . FFT(n) )_i,  Khat = FFT(N) C mu^2 / (P0 P1),
// with N(r) = (3 rhat rhat^T - I) / r^3 tabulated on a grid padded to
// P_k = next power of two >= 2 n_k - 1 per direction, so the circular
// convolution equals the open-boundary sum.  N is even in r, hence Khat is
// real and symmetric (6 components) and only kx <= P0/2 is stored.
//
// Three kernels per field evaluation:
//   rows    real FFT of each non-zero row (x and y components packed into one
//           complex transform, z in a second), half spectrum to S[c][y][kx];
//   columns complex FFT over y of a few columns, multiply by Khat, inverse
//           FFT, only rows y < n1 written back (the padding is never read);
//   irows   complex-to-real inverse of each row, cropped to x < n0.
// Transforms are radix-2 in shared memory: decimation in time for forward
// transforms (bit-reversed load, natural output) and in frequency for
// inverse ones (natural input, bit-reversed output), so no reordering pass.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "dipole.h"
#include "dipole_fast.h"

namespace spgb {

template <typename T> struct CxT;
template <> struct CxT<float> { using type = float2; };
template <> struct CxT<double> { using type = double2; };
template <typename T> using cx_t = typename CxT<T>::type;

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) { return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
template <typename C> __device__ __forceinline__ C cconj(C a) { return C{a.x, -a.y}; }

__device__ __forceinline__ int bitrev(int i, int logP) { return logP ? (int)(__brev((unsigned)i) >> (32 - logP)) : 0; }

// nf transforms of length P stored back to back; input bit-reversed.
template <typename C>
__device__ void fft_dit(C *a, int nf, int P, int logP, const C *__restrict__ tw, bool inv)
{
    int hp = P >> 1;
    for (int s = 1; s <= logP; ++s) {
        int half = 1 << (s - 1), stride = P >> s;
        for (int t = threadIdx.x; t < nf * hp; t += blockDim.x) {
            int f = t >> (logP - 1), u = t & (hp - 1);
            int j = u & (half - 1);
            int i0 = ((u >> (s - 1)) << s) + j;
            C w = tw[j * stride];
            if (inv) w.y = -w.y;
            C *b = a + f * P;
            C x0 = b[i0], x1 = cmul(b[i0 + half], w);
            b[i0] = cadd(x0, x1);
            b[i0 + half] = csub(x0, x1);
        }
        __syncthreads();
    }
}

// nf transforms of length P; natural input, bit-reversed output.
template <typename C>
__device__ void fft_dif(C *a, int nf, int P, int logP, const C *__restrict__ tw, bool inv)
{
    int hp = P >> 1;
    for (int s = logP; s >= 1; --s) {
        int half = 1 << (s - 1), stride = P >> s;
        for (int t = threadIdx.x; t < nf * hp; t += blockDim.x) {
            int f = t >> (logP - 1), u = t & (hp - 1);
            int j = u & (half - 1);
            int i0 = ((u >> (s - 1)) << s) + j;
            C w = tw[j * stride];
            if (inv) w.y = -w.y;
            C *b = a + f * P;
            C x0 = b[i0], x1 = b[i0 + half];
            b[i0] = cadd(x0, x1);
            b[i0 + half] = cmul(csub(x0, x1), w);
        }
        __syncthreads();
    }
}

struct Dims {
    int n0, n1, P0, P1, L0, L1, ncols, sst, cw;
};

// rows y < n1: half spectra of the x, y, z moment components
template <typename T>
__global__ void __launch_bounds__(256) k_dip_rows(Dims d, const rec_t<T> *__restrict__ n, cx_t<T> *__restrict__ S,
                                                  const cx_t<T> *__restrict__ tw0)
{
    using C = cx_t<T>;
    extern __shared__ unsigned char smem_raw[];
    C *c1 = reinterpret_cast<C *>(smem_raw), *c2 = c1 + d.P0;
    int y = blockIdx.x;
    for (int x = threadIdx.x; x < d.P0; x += blockDim.x) {
        int r = bitrev(x, d.L0);
        if (x < d.n0) {
            v3<T> m = ld(n, (long)y * d.n0 + x);
            c1[r] = C{m.x, m.y};
            c2[r] = C{m.z, T(0)};
        } else {
            c1[r] = C{T(0), T(0)};
            c2[r] = C{T(0), T(0)};
        }
    }
    __syncthreads();
    fft_dit(c1, 2, d.P0, d.L0, tw0, false);
    long plane = (long)d.n1 * d.sst;
    for (int k = threadIdx.x; k <= d.P0 / 2; k += blockDim.x) {
        C a = c1[k], b = cconj(c1[(d.P0 - k) & (d.P0 - 1)]);
        C X = C{T(0.5) * (a.x + b.x), T(0.5) * (a.y + b.y)};
        C Dd = csub(a, b);
        C Y = C{T(0.5) * Dd.y, T(-0.5) * Dd.x};
        long o = (long)y * d.sst + k;
        S[o] = X;
        S[plane + o] = Y;
        S[2 * plane + o] = c2[k];
    }
}

// columns kx0 .. kx0+cw-1: FFT over y (padded), multiply by Khat, inverse FFT
template <typename T>
__global__ void __launch_bounds__(256) k_dip_cols(Dims d, cx_t<T> *__restrict__ S, const T *__restrict__ K,
                                                  const cx_t<T> *__restrict__ tw1)
{
    using C = cx_t<T>;
    extern __shared__ unsigned char smem_raw[];
    C *a = reinterpret_cast<C *>(smem_raw);  // [3][cw][P1]
    int kx0 = blockIdx.x * d.cw;
    long plane = (long)d.n1 * d.sst;
    int tot = 3 * d.cw * d.P1;
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
        int y = t % d.P1, w = (t / d.P1) % d.cw, c = t / (d.P1 * d.cw);
        int kx = kx0 + w;
        C v = C{T(0), T(0)};
        if (y < d.n1 && kx < d.ncols) v = S[c * plane + (long)y * d.sst + kx];
        a[(c * d.cw + w) * d.P1 + bitrev(y, d.L1)] = v;
    }
    __syncthreads();
    fft_dit(a, 3 * d.cw, d.P1, d.L1, tw1, false);
    for (int t = threadIdx.x; t < d.cw * d.P1; t += blockDim.x) {
        int ky = t % d.P1, w = t / d.P1;
        int kx = kx0 + w;
        if (kx >= d.ncols) continue;
        const T *k6 = K + ((long)ky * d.ncols + kx) * 6;
        T xx = k6[0], xy = k6[1], xz = k6[2], yy = k6[3], yz = k6[4], zz = k6[5];
        C X = a[(0 * d.cw + w) * d.P1 + ky], Y = a[(1 * d.cw + w) * d.P1 + ky], Z = a[(2 * d.cw + w) * d.P1 + ky];
        a[(0 * d.cw + w) * d.P1 + ky] = C{xx * X.x + xy * Y.x + xz * Z.x, xx * X.y + xy * Y.y + xz * Z.y};
        a[(1 * d.cw + w) * d.P1 + ky] = C{xy * X.x + yy * Y.x + yz * Z.x, xy * X.y + yy * Y.y + yz * Z.y};
        a[(2 * d.cw + w) * d.P1 + ky] = C{xz * X.x + yz * Y.x + zz * Z.x, xz * X.y + yz * Y.y + zz * Z.y};
    }
    __syncthreads();
    fft_dif(a, 3 * d.cw, d.P1, d.L1, tw1, true);
    for (int t = threadIdx.x; t < 3 * d.cw * d.n1; t += blockDim.x) {
        int y = t % d.n1, w = (t / d.n1) % d.cw, c = t / (d.n1 * d.cw);
        int kx = kx0 + w;
        if (kx >= d.ncols) continue;
        S[c * plane + (long)y * d.sst + kx] = a[(c * d.cw + w) * d.P1 + bitrev(y, d.L1)];
    }
}

// rows y < n1: complex-to-real inverse, cropped to x < n0
template <typename T>
__global__ void __launch_bounds__(256) k_dip_irows(Dims d, const cx_t<T> *__restrict__ S, rec_t<T> *__restrict__ out,
                                                   const cx_t<T> *__restrict__ tw0)
{
    using C = cx_t<T>;
    extern __shared__ unsigned char smem_raw[];
    C *c1 = reinterpret_cast<C *>(smem_raw), *c2 = c1 + d.P0;
    int y = blockIdx.x;
    long plane = (long)d.n1 * d.sst;
    const C *s0 = S + (long)y * d.sst, *s1 = s0 + plane, *s2 = s0 + 2 * plane;
    for (int k = threadIdx.x; k < d.P0; k += blockDim.x) {
        C X, Y, Z;
        if (k <= d.P0 / 2) {
            X = s0[k];
            Y = s1[k];
            Z = s2[k];
        } else {
            X = cconj(s0[d.P0 - k]);
            Y = cconj(s1[d.P0 - k]);
            Z = cconj(s2[d.P0 - k]);
        }
        c1[k] = C{X.x - Y.y, X.y + Y.x};  // X + i Y
        c2[k] = Z;
    }
    __syncthreads();
    fft_dif(c1, 2, d.P0, d.L0, tw0, true);
    for (int x = threadIdx.x; x < d.n0; x += blockDim.x) {
        int r = bitrev(x, d.L0);
        st(out, (long)y * d.n0 + x, mk(c1[r].x, c1[r].y, c2[r].x));
    }
}

// ---------------------------------------------------------------- host side
struct DipolePlan {
    DipoleGeom g;
    Dims d;
    void *K[2] = {nullptr, nullptr}, *S[2] = {nullptr, nullptr}, *tw0[2] = {nullptr, nullptr},
         *tw1[2] = {nullptr, nullptr};
    bool ready[2] = {false, false};
    // FP32 warp-FFT path on a 1024 x 1024 grid
    bool fast = false, force_generic = false;
    void *Kt = nullptr, *ST = nullptr;
};

namespace {

int p2(int x)
{
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}
int lg(int p)
{
    int l = 0;
    while ((1 << l) < p) ++l;
    return l;
}

// In-place iterative radix-2 FFT of a power-of-two complex sequence with
// stride (forward, exp(-i)), double precision, host side.
void host_fft(std::complex<double> *a, int P, long stride)
{
    for (int i = 1, j = 0; i < P; ++i) {
        int bit = P >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i * stride], a[j * stride]);
    }
    for (int len = 2; len <= P; len <<= 1) {
        double ang = -2.0 * M_PI / len;
        for (int k = 0; k < len / 2; ++k) {
            std::complex<double> w(std::cos(ang * k), std::sin(ang * k));
            for (int i0 = 0; i0 < P; i0 += len) {
                std::complex<double> &u = a[(i0 + k) * stride], &v = a[(i0 + k + len / 2) * stride];
                std::complex<double> t = v * w;
                v = u - t;
                u = u + t;
            }
        }
    }
}

template <typename T> cudaError_t prepare(DipolePlan *p, cudaStream_t st)
{
    int ix = sizeof(T) == 8 ? 1 : 0;
    if (p->ready[ix]) return cudaSuccess;
    const Dims &d = p->d;
    using C = cx_t<T>;
    // interaction tensor on the padded grid, transformed in double precision
    long M = (long)d.P0 * d.P1;
    std::vector<std::complex<double>> grid(6 * M);
    for (int g1 = 0; g1 < d.P1; ++g1)
        for (int g0 = 0; g0 < d.P0; ++g0) {
            int s0 = g0 <= d.P0 / 2 ? g0 : g0 - d.P0, s1 = g1 <= d.P1 / 2 ? g1 : g1 - d.P1;
            if (std::abs(s0) > d.n0 - 1 || std::abs(s1) > d.n1 - 1 || (s0 == 0 && s1 == 0)) continue;
            double r[3];
            for (int l = 0; l < 3; ++l) r[l] = s0 * p->g.A[0][l] + s1 * p->g.A[1][l];
            double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2], rl = std::sqrt(r2), i3 = 1.0 / (r2 * rl);
            double u[3] = {r[0] / rl, r[1] / rl, r[2] / rl};
            long o = (long)g1 * d.P0 + g0;
            grid[0 * M + o] = (3 * u[0] * u[0] - 1) * i3;
            grid[1 * M + o] = 3 * u[0] * u[1] * i3;
            grid[2 * M + o] = 3 * u[0] * u[2] * i3;
            grid[3 * M + o] = (3 * u[1] * u[1] - 1) * i3;
            grid[4 * M + o] = 3 * u[1] * u[2] * i3;
            grid[5 * M + o] = (3 * u[2] * u[2] - 1) * i3;
        }
    for (int c = 0; c < 6; ++c) {
        std::complex<double> *a = grid.data() + c * M;
        for (int g1 = 0; g1 < d.P1; ++g1) host_fft(a + (long)g1 * d.P0, d.P0, 1);
        if (d.P1 > 1)
            for (int g0 = 0; g0 < d.P0; ++g0) host_fft(a + g0, d.P1, d.P0);
    }
    double scale = kDipole * p->g.mu[0] * p->g.mu[0] / (double)M;
    std::vector<T> K(6 * (size_t)d.ncols * d.P1);
    for (int ky = 0; ky < d.P1; ++ky)
        for (int kx = 0; kx < d.ncols; ++kx)
            for (int c = 0; c < 6; ++c) K[((size_t)ky * d.ncols + kx) * 6 + c] = (T)(grid[c * M + (long)ky * d.P0 + kx].real() * scale);
    if (sizeof(T) == 4 && d.P0 == 1024 && d.P1 == 1024) {
        // per-column structure of arrays for the warp-FFT path: Kt[kx][6][ky]
        std::vector<float> Kt((size_t)513 * 1024 * 6);
        for (int kx = 0; kx < 513; ++kx)
            for (int c = 0; c < 6; ++c)
                for (int ky = 0; ky < 1024; ++ky)
                    Kt[((size_t)kx * 6 + c) * 1024 + ky] = (float)(grid[c * M + (long)ky * d.P0 + kx].real() * scale);
        cudaError_t e;
        if ((e = cudaMalloc(&p->Kt, sizeof(float) * Kt.size())) != cudaSuccess) return e;
        if ((e = cudaMalloc(&p->ST, sizeof(float2) * 3 * 513 * (size_t)d.n1)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(p->Kt, Kt.data(), sizeof(float) * Kt.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        if ((e = dipole_fast_setup()) != cudaSuccess) return e;
        p->fast = true;
    }
    std::vector<C> t0(std::max(1, d.P0 / 2)), t1(std::max(1, d.P1 / 2));
    for (int k = 0; k < d.P0 / 2; ++k) t0[k] = C{(T)std::cos(2 * M_PI * k / d.P0), (T)-std::sin(2 * M_PI * k / d.P0)};
    for (int k = 0; k < d.P1 / 2; ++k) t1[k] = C{(T)std::cos(2 * M_PI * k / d.P1), (T)-std::sin(2 * M_PI * k / d.P1)};
    if (d.P1 / 2 == 0) t1[0] = C{T(1), T(0)};
    cudaError_t e;
    if ((e = cudaMalloc(&p->K[ix], sizeof(T) * K.size())) != cudaSuccess) return e;
    if ((e = cudaMalloc(&p->S[ix], sizeof(C) * 3 * (size_t)d.n1 * d.sst)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&p->tw0[ix], sizeof(C) * t0.size())) != cudaSuccess) return e;
    if ((e = cudaMalloc(&p->tw1[ix], sizeof(C) * t1.size())) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(p->K[ix], K.data(), sizeof(T) * K.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(p->tw0[ix], t0.data(), sizeof(C) * t0.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(p->tw1[ix], t1.data(), sizeof(C) * t1.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;  // host vectors go out of scope
    size_t row_smem = 2 * sizeof(C) * d.P0, col_smem = 3 * sizeof(C) * (size_t)d.cw * d.P1;
    if ((e = cudaFuncSetAttribute(k_dip_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_dip_irows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_dip_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)col_smem)) != cudaSuccess) return e;
    p->ready[ix] = true;
    return cudaSuccess;
}

template <typename T> cudaError_t run(DipolePlan *p, const void *n, void *out, cudaStream_t st)
{
    cudaError_t e = prepare<T>(p, st);
    if (e != cudaSuccess) return e;
    int ix = sizeof(T) == 8 ? 1 : 0;
    using C = cx_t<T>;
    const Dims &d = p->d;
    if (sizeof(T) == 4 && p->fast && !p->force_generic)
        return dipole_fast_run(d.n0, d.n1, (const float4 *)n, (float2 *)p->ST, (const float *)p->Kt, (float4 *)out, st);
    size_t row_smem = 2 * sizeof(C) * d.P0, col_smem = 3 * sizeof(C) * (size_t)d.cw * d.P1;
    C *S = (C *)p->S[ix];
    k_dip_rows<T><<<d.n1, 256, row_smem, st>>>(d, (const rec_t<T> *)n, S, (const C *)p->tw0[ix]);
    k_dip_cols<T><<<(d.ncols + d.cw - 1) / d.cw, 256, col_smem, st>>>(d, S, (const T *)p->K[ix], (const C *)p->tw1[ix]);
    k_dip_irows<T><<<d.n1, 256, row_smem, st>>>(d, S, (rec_t<T> *)out, (const C *)p->tw0[ix]);
    return cudaGetLastError();
}

}  // namespace

int dipole_create(DipolePlan **out, const DipoleGeom &g)
{
    *out = nullptr;
    if (g.nb != 1 || g.nc[2] != 1) return SP_ERR_UNSUPPORTED;
    Dims d;
    d.n0 = g.nc[0];
    d.n1 = g.nc[1];
    d.P0 = std::max(2, p2(2 * d.n0 - 1));
    d.P1 = d.n1 > 1 ? p2(2 * d.n1 - 1) : 1;
    if (d.P0 > 4096 || d.P1 > 4096) return SP_ERR_UNSUPPORTED;
    d.L0 = lg(d.P0);
    d.L1 = lg(d.P1);
    d.ncols = d.P0 / 2 + 1;
    d.sst = (d.ncols + 3) & ~3;
    // columns per block: keep the double-precision tile within 96 KB
    d.cw = 1;
    while (d.cw < 8 && 3L * 2 * d.cw * d.P1 * 16 <= 96 * 1024) d.cw *= 2;
    DipolePlan *p = new (std::nothrow) DipolePlan();
    if (!p) return SP_ERR_STATE;
    p->g = g;
    p->d = d;
    *out = p;
    return SP_OK;
}

void dipole_destroy(DipolePlan *p)
{
    if (!p) return;
    for (int k = 0; k < 2; ++k) {
        if (p->K[k]) cudaFree(p->K[k]);
        if (p->S[k]) cudaFree(p->S[k]);
        if (p->tw0[k]) cudaFree(p->tw0[k]);
        if (p->tw1[k]) cudaFree(p->tw1[k]);
    }
    if (p->Kt) cudaFree(p->Kt);
    if (p->ST) cudaFree(p->ST);
    delete p;
}

void dipole_force_generic(DipolePlan *p, bool on)
{
    if (p) p->force_generic = on;
}

cudaError_t dipole_field(DipolePlan *p, int prec, const void *n, void *out, cudaStream_t st)
{
    if (!p) return cudaErrorInvalidValue;
    return prec == SP_F64 ? run<double>(p, n, out, st) : run<float>(p, n, out, st);
}

}  // namespace spgb
