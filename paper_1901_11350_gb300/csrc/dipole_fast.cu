// dipole_fast.cu -- FP32 dipole convolution on a 1024 x 1024 padded grid
// (one-atom 2D lattices with 257..512 cells per side), same mathematics as
// dipole.cu with transforms laid out for the GPU:
//
// * every 1024-point transform is done by one warp as a four-step FFT,
//   1024 = 32 x 32: lane l holds x[32 n2 + l]; a 32-point FFT over n2 in
//   registers; twiddle W_1024^(l k2); transpose through shared memory; a
//   32-point FFT over n1 in registers -> lane m holds X[m + 32 k1];
// * row spectra are stored column-contiguous, ST[c][kx][y], so the column
//   pass reads and writes coalesced runs, and the row passes move runs of
//   two rows;
// * the column pass multiplies by Khat in the strided register layout the
//   inverse transform takes as input, so no reordering is needed.
#include <cmath>

#include "dipole.h"
#include "dipole_fast.h"

namespace spgb {

namespace {

constexpr int kRows = 2;         // rows per block in the row passes (two warps each)
constexpr int kTr = 32 * 33;     // transpose tile per warp (padded rows)

// W_32^j = exp(-2 pi i j / 32), j = 0..15
__constant__ float2 c_w32[16] = {
    {1.000000000e+00f, 0.000000000e+00f},   {9.807852804e-01f, -1.950903220e-01f},
    {9.238795325e-01f, -3.826834324e-01f},  {8.314696123e-01f, -5.555702330e-01f},
    {7.071067812e-01f, -7.071067812e-01f},  {5.555702330e-01f, -8.314696123e-01f},
    {3.826834324e-01f, -9.238795325e-01f},  {1.950903220e-01f, -9.807852804e-01f},
    {0.000000000e+00f, -1.000000000e+00f},  {-1.950903220e-01f, -9.807852804e-01f},
    {-3.826834324e-01f, -9.238795325e-01f}, {-5.555702330e-01f, -8.314696123e-01f},
    {-7.071067812e-01f, -7.071067812e-01f}, {-8.314696123e-01f, -5.555702330e-01f},
    {-9.238795325e-01f, -3.826834324e-01f}, {-9.807852804e-01f, -1.950903220e-01f}};

__device__ __forceinline__ float2 cm(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 ca(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cs(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cj(float2 a) { return make_float2(a.x, -a.y); }


constexpr int rev5(int i)
{
    return ((i & 1) << 4) | ((i & 2) << 2) | (i & 4) | ((i & 8) >> 2) | ((i & 16) >> 4);
}

// In-register radix-2 DIT FFT of 32 points (natural order in and out);
// INV: conjugate twiddles (unnormalised inverse).  The twiddles W^0 = 1 and
// W^8 = -i (+i inverse) are applied exactly, without multiplications.
// ZIN: the upper half of the input (a[16..31]) is zero, so the first
// stage's butterflies reduce to copies (a zero-padded transform).
template <bool INV, bool ZIN = false> __device__ __forceinline__ void fft32(float2 (&a)[32])
{
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const int j = rev5(i);
        if (i < j) {
            float2 t = a[i];
            a[i] = a[j];
            a[j] = t;
        }
    }
#pragma unroll
    for (int s = 1; s <= 5; ++s) {
        const int half = 1 << (s - 1), span = 1 << s;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int j = k % half, i0 = (k / half) * span + j, i1 = i0 + half;
            if (ZIN && s == 1) {  // a[i1] came from an input index >= 16
                a[i1] = a[i0];
                continue;
            }
            const int w = j * (32 / span);
            float2 t;
            if (w == 0) {
                t = a[i1];
            } else if (w == 8) {
                t = INV ? make_float2(-a[i1].y, a[i1].x) : make_float2(a[i1].y, -a[i1].x);
            } else {
                float2 tw = c_w32[w];
                if (INV) tw.y = -tw.y;
                t = cm(a[i1], tw);
            }
            a[i1] = cs(a[i0], t);
            a[i0] = ca(a[i0], t);
        }
    }
}

// Twiddles of the four-step transform, W_1024^(l k2) = exp(-2 pi i l k2 /
// 1024) for k2 = 0..31 (rows) and lane l (contiguous), rounded from FP64 on
// the host; the inverse uses their conjugates.
__device__ float2 g_tw1024[32 * 32];

// Four-step 1024-point FFT by one warp: on entry a[n2] = x[32 n2 + lane], on
// exit a[k1] = X[lane + 32 k1].  tr: this warp's 32 x 33 transpose tile.
// ZIN: x[512..1023] = 0 (a[16..31] are not read).
template <bool INV, bool ZIN = false> __device__ __forceinline__ void fft1024(float2 (&a)[32], float2 *tr, int lane)
{
    fft32<INV, ZIN>(a);
#pragma unroll
    for (int k2 = 1; k2 < 32; ++k2) {
        const float2 w = __ldg(&g_tw1024[k2 * 32 + lane]);
        a[k2] = cm(a[k2], INV ? cj(w) : w);
    }
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) tr[k2 * 33 + lane] = a[k2];
    __syncwarp();
#pragma unroll
    for (int n1 = 0; n1 < 32; ++n1) a[n1] = tr[lane * 33 + n1];
    __syncwarp();
    fft32<INV>(a);
}

// ------------------------------------------------------------ row pass
// Block: kRows rows, two warps per row (z, and x + i y).  Writes ST[c][k][y]
// for k = 0..512: half spectra of the x and y moment components (packed into
// one complex transform) and of z.
__global__ void __launch_bounds__(64 * kRows) k_rows(int n0, int n1, const float4 *__restrict__ n, float2 *__restrict__ ST)
{
    extern __shared__ float2 sm[];
    float2 *stage = sm;                                             // [3][513][kRows]
    float2 *tr = sm + 3 * 513 * kRows + (threadIdx.x / 32) * kTr;  // per warp
    int wid = threadIdx.x / 32, lane = threadIdx.x % 32;
    int w = wid >> 1, part = wid & 1;  // row in block; 0: z, 1: x + i y
    int y0 = blockIdx.x * kRows, y = y0 + w;
    bool row = y < n1;
    allow_dependents();
    wait_prerequisite();  // the spins may come from the pass just before
    float2 a[32];
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) {  // x < 512: the upper half is padding
        int x = 32 * n2 + lane;
        float4 v = (row && x < n0) ? __ldg(&n[(long)y * n0 + x]) : make_float4(0.f, 0.f, 0.f, 0.f);
        a[n2] = part ? make_float2(v.x, v.y) : make_float2(v.z, 0.f);
        a[n2 + 16] = make_float2(0.f, 0.f);
    }
    fft1024<false, true>(a, tr, lane);
    if (part == 0) {
#pragma unroll
        for (int k1 = 0; k1 <= 16; ++k1) {
            int k = lane + 32 * k1;
            if (k <= 512) stage[(2 * 513 + k) * kRows + w] = a[k1];
        }
    } else {
        // separate X and Y: X = (C[k] + conj C[-k]) / 2, Y = (C[k] - conj C[-k]) / 2i
#pragma unroll
        for (int k1 = 0; k1 < 32; ++k1) tr[lane + 32 * k1] = a[k1];  // spectrum, natural order
        __syncwarp();
#pragma unroll
        for (int k1 = 0; k1 <= 16; ++k1) {
            int k = lane + 32 * k1;
            if (k <= 512) {
                float2 A = tr[k], Bc = cj(tr[(1024 - k) & 1023]);
                float2 d = cs(A, Bc);
                stage[(0 * 513 + k) * kRows + w] = make_float2(0.5f * (A.x + Bc.x), 0.5f * (A.y + Bc.y));
                stage[(1 * 513 + k) * kRows + w] = make_float2(0.5f * d.y, -0.5f * d.x);
            }
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * 513 * kRows; t += blockDim.x) {
        int r = t % kRows, ck = t / kRows;
        if (y0 + r < n1) ST[(long)ck * n1 + y0 + r] = stage[t];
    }
}

// ------------------------------------------------------------ column pass
// Block: one column kx, warp c = component.  Khat of the column (6 x 1024
// reals, structure of arrays) is copied to shared memory with cp.async while
// the forward transform over y runs (zero rows y >= n1); product with Khat
// in the strided layout of the inverse transform's input; rows y < n1
// written back in place.
__device__ __forceinline__ void cp16(void *smem, const void *gmem)
{
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp8(void *smem, const void *gmem)
{
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}

__global__ void __launch_bounds__(96) k_cols(int n1, float2 *__restrict__ ST, const float *__restrict__ Kt)
{
    // The transpose tiles are live only inside the transforms and the spectra
    // only between them, so they share memory (barriers between the phases):
    // 49 KB per block, four blocks per SM, all 513 columns in one wave.
    extern __shared__ float2 sm[];
    float2 *spec = sm;                                  // [3][1024], between the transforms
    float2 *tr = sm + (threadIdx.x / 32) * kTr;         // [3][kTr], inside the transforms
    float *ks = reinterpret_cast<float *>(sm + 3 * kTr);  // [6][1024]
    int c = threadIdx.x / 32, lane = threadIdx.x % 32;
    int kx = blockIdx.x;
    const float *K = Kt + (long)kx * 6 * 1024;
    allow_dependents();
    for (int t = threadIdx.x; t < 6 * 1024 / 4; t += blockDim.x) cp16(ks + 4 * t, K + 4 * t);
    asm volatile("cp.async.commit_group;\n" ::);
    wait_prerequisite();  // the row spectra
    float2 *col = ST + ((long)c * 513 + kx) * n1;
    float2 a[32];
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) {  // y < 512: the upper half is padding
        int y = 32 * n2 + lane;
        a[n2] = y < n1 ? col[y] : make_float2(0.f, 0.f);
        a[n2 + 16] = make_float2(0.f, 0.f);
    }
    fft1024<false, true>(a, tr, lane);
    __syncthreads();  // every warp is done with its transpose tile
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) spec[c * 1024 + lane + 32 * k1] = a[k1];
    asm volatile("cp.async.wait_group 0;\n" ::);
    __syncthreads();
    // row c of the symmetric tensor (xx xy xz yy yz zz)
    const int i0 = c == 0 ? 0 : (c == 1 ? 1 : 2);
    const int i1 = c == 0 ? 1 : (c == 1 ? 3 : 4);
    const int i2 = c == 0 ? 2 : (c == 1 ? 4 : 5);
#pragma unroll
    for (int n2 = 0; n2 < 32; ++n2) {
        int ky = 32 * n2 + lane;
        float r0 = ks[i0 * 1024 + ky], r1 = ks[i1 * 1024 + ky], r2 = ks[i2 * 1024 + ky];
        float2 X = spec[ky], Y = spec[1024 + ky], Z = spec[2048 + ky];
        a[n2] = make_float2(r0 * X.x + r1 * Y.x + r2 * Z.x, r0 * X.y + r1 * Y.y + r2 * Z.y);
    }
    __syncthreads();  // every warp has read the spectra before the tiles reuse them
    fft1024<true>(a, tr, lane);
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) {
        int y = lane + 32 * k1;
        if (y < n1) col[y] = a[k1];
    }
}

// ------------------------------------------------------------ inverse rows
// Block: kRows rows, two warps per row: complex-to-real inverse of z, and of
// X + i Y; cropped to x < n0 and written as 4-wide records.
__global__ void __launch_bounds__(64 * kRows) k_irows(int n0, int n1, const float2 *__restrict__ ST, float4 *__restrict__ out)
{
    extern __shared__ float2 sm[];
    float2 *stage = sm;
    float2 *tr = sm + 3 * 513 * kRows + (threadIdx.x / 32) * kTr;
    float *zs = reinterpret_cast<float *>(sm + 3 * 513 * kRows + 2 * kRows * kTr);  // [kRows][512]
    int wid = threadIdx.x / 32, lane = threadIdx.x % 32;
    int w = wid >> 1, part = wid & 1;
    int y0 = blockIdx.x * kRows, y = y0 + w;
    allow_dependents();
    wait_prerequisite();  // the column pass's spectra
    for (int t = threadIdx.x; t < 3 * 513 * kRows; t += blockDim.x) {
        int r = t % kRows, ck = t / kRows;
        if (y0 + r < n1)
            cp8(stage + t, ST + (long)ck * n1 + y0 + r);
        else
            stage[t] = make_float2(0.f, 0.f);
    }
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    float2 a[32];
#pragma unroll
    for (int n2 = 0; n2 < 32; ++n2) {
        int k = 32 * n2 + lane;
        if (part == 0) {
            a[n2] = k <= 512 ? stage[(2 * 513 + k) * kRows + w] : cj(stage[(2 * 513 + 1024 - k) * kRows + w]);
        } else {
            float2 X, Y;
            if (k <= 512) {
                X = stage[(0 * 513 + k) * kRows + w];
                Y = stage[(1 * 513 + k) * kRows + w];
            } else {
                X = cj(stage[(0 * 513 + 1024 - k) * kRows + w]);
                Y = cj(stage[(1 * 513 + 1024 - k) * kRows + w]);
            }
            a[n2] = make_float2(X.x - Y.y, X.y + Y.x);  // X + i Y
        }
    }
    fft1024<true>(a, tr, lane);
    if (part == 0) {
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) zs[w * 512 + lane + 32 * k1] = a[k1].x;
    }
    __syncthreads();
    if (part == 1 && y < n1) {
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) {
            int x = lane + 32 * k1;
            if (x < n0) out[(long)y * n0 + x] = make_float4(a[k1].x, a[k1].y, zs[w * 512 + x], 0.f);
        }
    }
}

constexpr size_t kRowSmem = sizeof(float2) * (3 * 513 * kRows + 2 * kRows * kTr) + sizeof(float) * kRows * 512;
constexpr size_t kColSmem = sizeof(float2) * (3 * kTr) + sizeof(float) * 6 * 1024;
static_assert(3 * kTr >= 3 * 1024, "the transpose tiles must cover the spectra they alias");

}  // namespace

cudaError_t dipole_fast_setup()
{
    static bool table = false;  // per process
    if (!table) {
        float2 tw[32 * 32];
        for (int k2 = 0; k2 < 32; ++k2)
            for (int l = 0; l < 32; ++l) {
                const double ph = -2.0 * M_PI * (double)(k2 * l) / 1024.0;
                tw[k2 * 32 + l] = make_float2((float)std::cos(ph), (float)std::sin(ph));
            }
        cudaError_t e = cudaMemcpyToSymbol(g_tw1024, tw, sizeof tw);
        if (e != cudaSuccess) return e;
        table = true;
    }
    cudaError_t e = cudaFuncSetAttribute(k_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRowSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_irows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRowSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kColSmem);
    return e;
}

cudaError_t dipole_fast_run(int n0, int n1, const float4 *n, float2 *ST, const float *Kt, float4 *out, cudaStream_t st)
{
    int rb = (n1 + kRows - 1) / kRows;
    cudaError_t e = launch_pdl(k_rows, dim3(rb), dim3(64 * kRows), kRowSmem, st, n0, n1, n, ST);
    if (e == cudaSuccess) e = launch_pdl(k_cols, dim3(513), dim3(96), kColSmem, st, n1, ST, Kt);
    if (e == cudaSuccess) e = launch_pdl(k_irows, dim3(rb), dim3(64 * kRows), kRowSmem, st, n0, n1, (const float2 *)ST, out);
    return e;
}

}  // namespace spgb
