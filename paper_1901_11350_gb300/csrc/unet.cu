// unet.cu -- BF16 U-Net that warm-starts energy minimisation (the C ABI of
// include/spirit_gb_unet.h): periodic 3x3 implicit-GEMM convolutions on the
// tensor cores (forward, data gradient, weight gradient), the pointwise
// kernels around them, the FP32 head with its loss, and Adam.
//
// Convolution as a GEMM: M = pixels, N = output channels, K = 9 taps x input
// channels.  A CTA owns 128 pixels x BN channels; each K step stages one tap
// x 32 input channels of the (virtual) input -- periodic wrap, nearest
// upsampling and channel concatenation are resolved in the address
// computation -- and the matching weight slice in shared memory with
// cp.async, three stages deep, and feeds m16n8k16 BF16 MMAs with FP32
// accumulators.  Shared-memory rows are 64 bytes with the 16-byte chunks
// XOR-swizzled so ldmatrix reads are free of bank conflicts.
#include <cuda_bf16.h>
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "spirit_gb.h"
#include "spirit_gb_unet.h"

namespace {

typedef __nv_bfloat16 bf16;

constexpr int kBM = 128;     // pixels per convolution CTA
constexpr int kBK = 32;      // input channels per K step
constexpr int kStages = 3;   // cp.async pipeline depth
constexpr int kThreads = 256;

struct ConvSrc {
    const bf16 *s0;
    int C0, up0;
    const bf16 *s1;
    int C1;
};

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16(unsigned dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
}
// the same through L1 (the weight gradient's taps re-read shifted copies of
// the same input rows; measured slower for the forward convolution)
__device__ __forceinline__ void cp16_ca(unsigned dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm4(unsigned addr, unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm4t(unsigned addr, unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Byte offset of 16-byte chunk c of row r in a tile of 64-byte rows, and in a
// tile of 128-byte rows.  Eight consecutive rows at one logical chunk land on
// eight distinct bank groups.
__device__ __forceinline__ unsigned swz64(int r, int c) { return (unsigned)(r * 64 + ((c ^ ((r >> 1) & 3)) << 4)); }
__device__ __forceinline__ unsigned swz128(int r, int c) { return (unsigned)(r * 128 + ((c ^ (r & 7)) << 4)); }

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Address of channels [c, c+8) of the virtual input at pixel (b, y, x).
__device__ __forceinline__ const bf16 *src_at(const ConvSrc &S, int b, int y, int x, int H, int W, int c)
{
    if (c < S.C0) {
        if (S.up0) return S.s0 + ((size_t)(b * (H >> 1) + (y >> 1)) * (W >> 1) + (x >> 1)) * S.C0 + c;
        return S.s0 + ((size_t)(b * H + y) * W + x) * S.C0 + c;
    }
    return S.s1 + ((size_t)(b * H + y) * W + x) * S.C1 + (c - S.C0);
}

// ------------------------------------------------------------------ conv
// out[p][co] = act(bias[co] + sum_{t,ci} Wk[co][t][ci] in[p + off(t)][ci]),
// zeroed where mask[p][co] is not > 0.  Grid (P/128, Cout/BN), 256 threads as
// 4 (pixels) x 2 (channels) warps of 32 x BN/2.
template <int BN>
__global__ void __launch_bounds__(kThreads) k_conv(ConvSrc S, const bf16 *__restrict__ Wk, const float *__restrict__ bias,
                                                   int relu, const bf16 *__restrict__ mask, int H, int W, int Cout,
                                                   bf16 *__restrict__ out)
{
    constexpr int A_BYTES = kBM * 64, STAGE = A_BYTES + BN * 64;
    constexpr int WN = BN / 2, NT = WN / 8;
    extern __shared__ __align__(128) unsigned char smem[];
    const int Cin = S.C0 + S.C1, nkc = Cin / kBK, nk = 9 * nkc;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 3, wn = warp >> 2;
    const int HW = H * W;
    const int ar = tid >> 2, ac = tid & 3;
    int pb[2], py[2], px[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        int p = m0 + ar + 64 * j;
        pb[j] = p / HW;
        int q = p - pb[j] * HW;
        py[j] = q / W;
        px[j] = q - py[j] * W;
    }
    const unsigned sbase = smem_u32(smem);
    auto load = [&](int k, int stage) {
        int t = k / nkc, cc = (k - t * nkc) * kBK;
        int dy = t / 3 - 1, dx = t % 3 - 1;
        unsigned sa = sbase + stage * STAGE;
#pragma unroll
        for (int j = 0; j < 2; ++j)
            cp16(sa + swz64(ar + 64 * j, ac),
                 src_at(S, pb[j], wrap(py[j] + dy, H), wrap(px[j] + dx, W), H, W, cc + ac * 8));
        unsigned sb = sa + A_BYTES;
        for (int idx = tid; idx < BN * 4; idx += kThreads) {
            int r = idx >> 2, c = idx & 3;
            cp16(sb + swz64(r, c), Wk + (size_t)(n0 + r) * 9 * Cin + t * Cin + cc + c * 8);
        }
    };
    float acc[2][NT][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
#pragma unroll
    for (int s = 0; s < kStages - 1; ++s) {
        if (s < nk) load(s, s);
        cp_commit();
    }
    const int lj = lane >> 3, lr = lane & 7;
    for (int k = 0; k < nk; ++k) {
        cp_wait<kStages - 2>();
        __syncthreads();
        int kn = k + kStages - 1;
        if (kn < nk) load(kn, kn % kStages);
        cp_commit();
        unsigned sa = sbase + (k % kStages) * STAGE, sb = sa + A_BYTES;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            unsigned a[2][4];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
                ldsm4(sa + swz64(wm * 32 + mi * 16 + lr + (lj & 1) * 8, kk * 2 + (lj >> 1)), a[mi][0], a[mi][1],
                      a[mi][2], a[mi][3]);
#pragma unroll
            for (int ni = 0; ni < NT; ni += 2) {
                unsigned b0, b1, b2, b3;
                ldsm4(sb + swz64(wn * WN + ni * 8 + lr + (lj >> 1) * 8, kk * 2 + (lj & 1)), b0, b1, b2, b3);
#pragma unroll
                for (int mi = 0; mi < 2; ++mi) {
                    mma16816(acc[mi][ni], a[mi], b0, b1);
                    mma16816(acc[mi][ni + 1], a[mi], b2, b3);
                }
            }
        }
    }
    cp_wait<0>();
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < NT; ++ni) {
            int co = n0 + wn * WN + ni * 8 + 2 * t4;
            float c0 = bias ? bias[co] : 0.f, c1 = bias ? bias[co + 1] : 0.f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                int p = m0 + wm * 32 + mi * 16 + g + h * 8;
                float v0 = acc[mi][ni][2 * h] + c0, v1 = acc[mi][ni][2 * h + 1] + c1;
                if (relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                size_t o = (size_t)p * Cout + co;
                if (mask) {
                    __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162 *>(mask + o);
                    if (!(__low2float(mk) > 0.f)) v0 = 0.f;
                    if (!(__high2float(mk) > 0.f)) v1 = 0.f;
                }
                *reinterpret_cast<__nv_bfloat162 *>(out + o) = __floats2bfloat162_rn(v0, v1);
            }
        }
}

// ------------------------------------------------------------------ conv, tcgen05
// The same convolution on the 5th-generation tensor cores: one thread issues
// 128 x BN x 16 MMAs (kind::f16, BF16 in, FP32 out) whose accumulator lives
// in tensor memory; operands are the shared-memory stages above, read through
// K-major SWIZZLE_64B descriptors (the 64-byte XOR layout of swz64 is that
// swizzle).  Each stage is released by a tcgen05.commit on its own mbarrier.
// Every wait is bounded: on a timeout the CTA records an error, stops
// issuing work, waits (bounded) for the MMAs it issued, frees its tensor
// memory and returns.
constexpr int kTcStages = 4;

__device__ int g_tc_error;  // set when a bounded wait ran out

__device__ __forceinline__ uint64_t desc_sw64(unsigned addr)
{
    // start >> 4 | leading byte offset 16 B (unused for swizzled K-major) |
    // stride byte offset 512 B (8 rows of 64 B) | descriptor version 1 |
    // layout 4 = 64-byte swizzle
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Wait for completion of the phase with this parity, for at most `limit`
// cycles (2^32 is about two seconds); false when the limit ran out.  A limit
// of 0 gives up at once, without polling.
constexpr long long kWaitCycles = 1LL << 32;
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, long long limit = kWaitCycles)
{
    if (limit <= 0) return false;
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// Cycles k_conv_tc's pipeline waits (a stage's MMAs releasing its buffers)
// poll before they give up; sp_conv3x3_set_wait_limit.  The final wait for
// the accumulator always keeps kWaitCycles, so that every MMA a CTA issued
// has finished before it frees its tensor memory.
__device__ long long g_tc_wait_limit = kWaitCycles;

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void tc_mma(unsigned tmem_d, uint64_t adesc, uint64_t bdesc, unsigned idesc, unsigned acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
                 "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
                 : "memory");
}

__device__ __forceinline__ void tc_commit(unsigned bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's tensor-memory lane
__device__ __forceinline__ void tc_ld16(unsigned taddr, float (&v)[16])
{
    unsigned r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                 "[%16];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// + the CTA's tap table: for each of the 9 taps and 128 pixels the source
// pixel index in src0's grid and in the full-resolution grid (2 x 4.5 KB)
constexpr int kTapTable = 2 * 9 * kBM * 4;
template <int BN>
constexpr size_t conv_tc_smem()
{
    return 1024 + (size_t)kTcStages * (kBM * 64 + BN * 64) + 8 * kTcStages + 16 + 16 + kTapTable;
}

template <int BN>
__global__ void __launch_bounds__(kThreads) k_conv_tc(ConvSrc S, const bf16 *__restrict__ Wk,
                                                      const float *__restrict__ bias, int relu,
                                                      const bf16 *__restrict__ mask, int H, int W, int Cout,
                                                      bf16 *__restrict__ out)
{
    constexpr int A_BYTES = kBM * 64, STAGE = A_BYTES + BN * 64;
    constexpr unsigned TCOLS = BN;  // 32, 64 or 128: a power of two >= 32
    constexpr unsigned IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(BN >> 3) << 17) |
                               ((unsigned)(kBM >> 4) << 24);
    extern __shared__ unsigned char smem_raw[];
    const unsigned raw = smem_u32(smem_raw);
    const unsigned base = (raw + 1023u) & ~1023u;  // swizzle atoms need 1024-byte alignment here
    const unsigned bar0 = base + kTcStages * STAGE;
    const unsigned slot = bar0 + 8 * kTcStages;
    volatile unsigned *slot_ptr = reinterpret_cast<volatile unsigned *>(smem_raw + (slot - raw));
    int *tq = reinterpret_cast<int *>(smem_raw + (slot + 16 - raw));  // [2][9][kBM]

    const int Cin = S.C0 + S.C1, nkc = Cin / kBK, nk = 9 * nkc;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int HW = H * W;
    const long long wait_limit = g_tc_wait_limit;
    const int ar = tid >> 2, ac = tid & 3;
    // the tap table, once per CTA: pixel indices of every (tap, pixel) with
    // the periodic wrap applied, so that a stage's copies only add offsets
    for (int e = tid; e < 9 * kBM; e += kThreads) {
        const int t = e / kBM, p = m0 + (e - t * kBM);
        const int b = p / HW, q = p - b * HW, y = q / W, x = q - y * W;
        const int yy = wrap(y + t / 3 - 1, H), xx = wrap(x + t % 3 - 1, W);
        const int full = (b * H + yy) * W + xx;
        tq[e] = S.up0 ? (b * (H >> 1) + (yy >> 1)) * (W >> 1) + (xx >> 1) : full;
        tq[9 * kBM + e] = full;
    }
    // this thread's weight rows: chunk idx = tid + 256 i of the BN x 4 chunks
    constexpr int BW = (BN * 4 + kThreads - 1) / kThreads;
    const bf16 *wrow[BW];
    unsigned woff[BW];
#pragma unroll
    for (int i = 0; i < BW; ++i) {
        const int idx = tid + kThreads * i, r = idx >> 2, c = idx & 3;
        wrow[i] = Wk + (size_t)(n0 + (idx < BN * 4 ? r : 0)) * 9 * Cin + c * 8;
        woff[i] = swz64(r, c);
    }
    const unsigned aoff0 = swz64(ar, ac), aoff1 = swz64(ar + 64, ac);
    // the next stage to load: K step k_ld = tap t_ld, channels [cc_ld, cc_ld + 32)
    int k_ld = 0, t_ld = 0, cc_ld = 0;
    auto load = [&](int stage) {
        const unsigned sa = base + stage * STAGE;
        const int *q = tq + (cc_ld < S.C0 ? 0 : 9 * kBM) + t_ld * kBM + ar;
        const bf16 *src = cc_ld < S.C0 ? S.s0 + cc_ld + ac * 8 : S.s1 + (cc_ld - S.C0) + ac * 8;
        const int cs = cc_ld < S.C0 ? S.C0 : S.C1;
        cp16(sa + aoff0, src + (size_t)q[0] * cs);
        cp16(sa + aoff1, src + (size_t)q[64] * cs);
        const unsigned sb = sa + A_BYTES;
#pragma unroll
        for (int i = 0; i < BW; ++i)
            if (tid + kThreads * i < BN * 4) cp16(sb + woff[i], wrow[i] + k_ld * kBK);
        ++k_ld;
        cc_ld += kBK;
        if (cc_ld == Cin) {
            cc_ld = 0;
            ++t_ld;
        }
    };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot), "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < kTcStages; ++s) mbar_init(bar0 + 8 * s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();  // also publishes the tap table
    tc_fence_after();
    const unsigned tmem = *slot_ptr;

#pragma unroll
    for (int s = 0; s < kTcStages - 1; ++s) {
        if (s < nk) load(s);
        cp_commit();
    }
    int failed = 0, issued = 0;
    for (int k = 0; k < nk; ++k) {
        const int s = k % kTcStages;
        cp_wait<kTcStages - 2>();
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        if (__syncthreads_or(failed)) {
            failed = 1;
            break;
        }
        if (tid == 0) {
            tc_fence_after();
            const unsigned sa = base + s * STAGE, sb = sa + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < 2; ++kk)
                tc_mma(tmem, desc_sw64(sa + kk * 32), desc_sw64(sb + kk * 32), IDESC, (k > 0 || kk > 0) ? 1u : 0u);
            tc_commit(bar0 + 8 * s);
        }
        issued = k + 1;
        const int kn = k + kTcStages - 1;
        if (kn < nk) {
            const int sn = kn % kTcStages;  // the stage the MMAs of iteration k-1 read
            if (k >= 1 && !mbar_wait(bar0 + 8 * sn, ((k - 1) / kTcStages) & 1, wait_limit)) failed = 1;
            if (!failed) load(sn);
        }
        cp_commit();
    }
    cp_wait<0>();
    // the last commit tracks every MMA issued before it
    if (issued > 0 && !mbar_wait(bar0 + 8 * ((issued - 1) % kTcStages), ((issued - 1) / kTcStages) & 1)) failed = 1;
    failed = __syncthreads_or(failed) || issued < nk;
    tc_fence_after();
    const int q = warp & 3, half = warp >> 2;
    const int p = m0 + q * 32 + lane;
#pragma unroll
    for (int c0 = half * (BN / 2); c0 < (half + 1) * (BN / 2); c0 += 16) {
        float v[16];
        tc_ld16(tmem + ((unsigned)(q * 32) << 16) + (unsigned)c0, v);
        if (failed) continue;
        const int co = n0 + c0;
        size_t o = (size_t)p * Cout + co;
        __align__(16) bf16 mk[16];
        if (mask) {
            *reinterpret_cast<uint4 *>(mk) = *reinterpret_cast<const uint4 *>(mask + o);
            *reinterpret_cast<uint4 *>(mk + 8) = *reinterpret_cast<const uint4 *>(mask + o + 8);
        }
        __align__(16) bf16 r[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            float x = v[e] + (bias ? bias[co + e] : 0.f);
            if (relu) x = fmaxf(x, 0.f);
            if (mask && !(__bfloat162float(mk[e]) > 0.f)) x = 0.f;
            r[e] = __float2bfloat16(x);
        }
        *reinterpret_cast<uint4 *>(out + o) = *reinterpret_cast<const uint4 *>(r);
        *reinterpret_cast<uint4 *>(out + o + 8) = *reinterpret_cast<const uint4 *>(r + 8);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TCOLS) : "memory");
    if (failed && tid == 0) atomicExch(&g_tc_error, 1);
}

// ------------------------------------------------------------------ conv, tcgen05, warp-specialised
// The same convolution with the loads and the MMAs decoupled: warps 0-6 load
// stages with cp.async and signal each stage's "full" mbarrier when their
// copies land (cp.async.mbarrier.arrive.noinc), one lane of warp 7 waits for
// a full stage, makes the copies visible to the tensor cores' proxy, issues
// the stage's MMAs and commits them to the stage's "empty" mbarrier, which
// the loaders wait for before refilling it.  No CTA-wide barrier in the main
// loop.  Input rows are read through L1 (cp.async.ca): the nine taps read
// shifted copies of the same rows.  Every wait is bounded as in k_conv_tc.
constexpr int kWsStages = 6;
constexpr int kWsLoaders = 224;  // warps 0-6
constexpr int kWsRows = (kBM * 4 + kWsLoaders - 1) / kWsLoaders;  // A chunks per loader (3)

__device__ __forceinline__ void cp_arrive_noinc(unsigned bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(bar) : "memory");
}

template <int BN>
constexpr size_t conv_ws_smem()
{
    return 1024 + (size_t)kWsStages * (kBM * 64 + BN * 64) + 16 * kWsStages + 16 + 16;
}

template <int BN>
__global__ void __launch_bounds__(kThreads) k_conv_ws(ConvSrc S, const bf16 *__restrict__ Wk,
                                                      const float *__restrict__ bias, int relu,
                                                      const bf16 *__restrict__ mask, int H, int W, int Cout,
                                                      bf16 *__restrict__ out)
{
    constexpr int A_BYTES = kBM * 64, STAGE = A_BYTES + BN * 64;
    constexpr unsigned TCOLS = BN;
    constexpr unsigned IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(BN >> 3) << 17) |
                               ((unsigned)(kBM >> 4) << 24);
    extern __shared__ unsigned char smem_raw[];
    const unsigned raw = smem_u32(smem_raw);
    const unsigned base = (raw + 1023u) & ~1023u;
    const unsigned full0 = base + kWsStages * STAGE;  // kWsStages "full" barriers
    const unsigned empty0 = full0 + 8 * kWsStages;    // kWsStages "empty" barriers
    const unsigned done = empty0 + 8 * kWsStages;     // last MMA finished
    const unsigned slot = done + 8;
    volatile unsigned *slot_ptr = reinterpret_cast<volatile unsigned *>(smem_raw + (slot - raw));
    __shared__ int s_fail;

    const int Cin = S.C0 + S.C1, nkc = Cin / kBK, nk = 9 * nkc;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int HW = H * W;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot), "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < kWsStages; ++s) {
            mbar_init(full0 + 8 * s, kWsLoaders);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(done, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *slot_ptr;
    int failed = 0;

    if (warp < 7) {
        // loaders: A chunks idx = tid + 224 j (512 of them), B chunks likewise;
        // the pixel of each A chunk is decoded once
        int pb[kWsRows], py[kWsRows], px[kWsRows];
#pragma unroll
        for (int j = 0; j < kWsRows; ++j) {
            int idx = tid + kWsLoaders * j;
            int p = m0 + (idx >> 2);
            pb[j] = p / HW;
            int q = p - pb[j] * HW;
            py[j] = q / W;
            px[j] = q - py[j] * W;
        }
        for (int k = 0; k < nk && !failed; ++k) {
            const int s = k % kWsStages, u = k / kWsStages;
            if (u > 0 && !mbar_wait(empty0 + 8 * s, (u - 1) & 1)) {
                failed = 1;
                break;
            }
            const int t = k / nkc, cc = (k - t * nkc) * kBK;
            const int dy = t / 3 - 1, dx = t % 3 - 1;
            const unsigned sa = base + s * STAGE, sb = sa + A_BYTES;
#pragma unroll
            for (int j = 0; j < kWsRows; ++j) {
                int idx = tid + kWsLoaders * j;
                if (idx < kBM * 4) {
                    int r = idx >> 2, c = idx & 3;
                    cp16_ca(sa + swz64(r, c),
                            src_at(S, pb[j], wrap(py[j] + dy, H), wrap(px[j] + dx, W), H, W, cc + c * 8));
                }
            }
            for (int idx = tid; idx < BN * 4; idx += kWsLoaders) {
                int r = idx >> 2, c = idx & 3;
                cp16(sb + swz64(r, c), Wk + (size_t)(n0 + r) * 9 * Cin + t * Cin + cc + c * 8);
            }
            cp_arrive_noinc(full0 + 8 * s);
        }
        // the copies above belong to no commit group: wait for all of them
        asm volatile("cp.async.wait_all;\n" ::: "memory");
    } else if (lane == 0) {
        // MMA issuer
        int k = 0;
        for (; k < nk; ++k) {
            const int s = k % kWsStages, u = k / kWsStages;
            if (!mbar_wait(full0 + 8 * s, u & 1)) {
                failed = 1;
                break;
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            tc_fence_after();
            const unsigned sa = base + s * STAGE, sb = sa + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < 2; ++kk)
                tc_mma(tmem, desc_sw64(sa + kk * 32), desc_sw64(sb + kk * 32), IDESC, (k > 0 || kk > 0) ? 1u : 0u);
            tc_commit(empty0 + 8 * s);
        }
        // completion of every MMA issued (possibly none)
        tc_commit(done);
        if (k < nk) failed = 1;
    }
    if (failed) s_fail = 1;
    // wait for the accumulator (bounded), then every warp reads its lanes
    if (!mbar_wait(done, 0)) failed = 1;
    failed = __syncthreads_or(failed || s_fail);
    tc_fence_after();
    const int q = warp & 3, half = warp >> 2;
    const int p = m0 + q * 32 + lane;
#pragma unroll
    for (int c0 = half * (BN / 2); c0 < (half + 1) * (BN / 2); c0 += 16) {
        float v[16];
        tc_ld16(tmem + ((unsigned)(q * 32) << 16) + (unsigned)c0, v);
        if (failed) continue;
        const int co = n0 + c0;
        size_t o = (size_t)p * Cout + co;
        __align__(16) bf16 mk[16];
        if (mask) {
            *reinterpret_cast<uint4 *>(mk) = *reinterpret_cast<const uint4 *>(mask + o);
            *reinterpret_cast<uint4 *>(mk + 8) = *reinterpret_cast<const uint4 *>(mask + o + 8);
        }
        __align__(16) bf16 r[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            float x = v[e] + (bias ? bias[co + e] : 0.f);
            if (relu) x = fmaxf(x, 0.f);
            if (mask && !(__bfloat162float(mk[e]) > 0.f)) x = 0.f;
            r[e] = __float2bfloat16(x);
        }
        *reinterpret_cast<uint4 *>(out + o) = *reinterpret_cast<const uint4 *>(r);
        *reinterpret_cast<uint4 *>(out + o + 8) = *reinterpret_cast<const uint4 *>(r + 8);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TCOLS) : "memory");
    if (failed && tid == 0) atomicExch(&g_tc_error, 1);
}

// ------------------------------------------------------------------ conv, tcgen05, halo tiles
// The same convolution with the input of a band of whole image rows loaded
// once per chunk of 32 input channels.  A CTA computes R rows of one image
// for BN output channels.  Per chunk it stages the band's halo tile -- R + 2
// rows of W + 2 pixels, the periodic wrap, the upsampling and the channel
// concatenation resolved through a per-CTA pixel table -- in the no-swizzle
// K-major layout (four planes of 8 channels, 16 bytes per pixel, pixels
// consecutive) and the chunk's weights of all nine taps.  Outputs are
// numbered in "slots" with the tile's row pitch W + 2, so that a tap is a
// fixed pixel offset: the MMA of tap (dy, dx) over slots [s, s + 128) reads
// A from tile pixel s + (1 + dy)(W + 2) + 1 + dx -- a 16-byte aligned start
// address -- and the nine taps re-read nothing from memory.  Slots in the two
// halo columns, and past the band, compute values that are not stored.  The
// accumulators of all slots (MT tiles of 128 slots x BN columns) stay in
// tensor memory across the chunks.  One stage: the chunk's copies, a CTA
// barrier, the MMAs (one thread issues and commits them), and the next
// chunk's copies wait for that commit; two CTAs per SM overlap one's copies
// with the other's MMAs.  Waits are bounded as in k_conv_tc.
struct HaloGeom {
    int R, Wp, npix, slots, MT, apix;
    unsigned a_bytes, b_bytes, tbl_bytes, smem, tcols;
};

constexpr unsigned kHaloSmemMax = 113 * 1024;  // two CTAs per SM
constexpr unsigned kHaloTmemMax = 256;         // tensor-memory columns per CTA (two per SM)

__host__ __device__ inline HaloGeom halo_geom(int R, int W, int BN)
{
    HaloGeom g;
    g.R = R;
    g.Wp = W + 2;
    g.npix = (R + 2) * g.Wp;
    g.slots = R * g.Wp;
    g.MT = (g.slots + kBM - 1) / kBM;
    g.apix = g.MT * kBM + 2 * g.Wp + 2;  // the last tile's reads of tap (+1, +1) stay inside
    g.a_bytes = 64u * g.apix;
    g.b_bytes = 9u * 64u * BN;
    g.tbl_bytes = 8u * g.npix;
    g.smem = 128 + g.a_bytes + g.b_bytes + g.tbl_bytes + 16;
    unsigned cols = 32;
    while (cols < (unsigned)(g.MT * BN)) cols *= 2;
    g.tcols = cols;
    return g;
}

__device__ __forceinline__ uint64_t desc_ns(unsigned addr, unsigned lbo, unsigned sbo)
{
    // start >> 4 | leading byte offset (between core matrices along K) |
    // stride byte offset (between 8-row groups) | descriptor version 1 |
    // no swizzle
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           ((uint64_t)1 << 46);
}

template <int BN>
__global__ void __launch_bounds__(kThreads) k_conv_halo(ConvSrc S, const bf16 *__restrict__ Wk,
                                                        const float *__restrict__ bias, int relu,
                                                        const bf16 *__restrict__ mask, int H, int W, int Cout, int R,
                                                        bf16 *__restrict__ out)
{
    constexpr unsigned IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(BN >> 3) << 17) |
                               ((unsigned)(kBM >> 4) << 24);
    const HaloGeom G = halo_geom(R, W, BN);
    extern __shared__ unsigned char smem_raw[];
    const unsigned raw = smem_u32(smem_raw);
    const unsigned base = (raw + 127u) & ~127u;
    const unsigned sa = base, sb = base + G.a_bytes;
    int *tbl = reinterpret_cast<int *>(smem_raw + (sb + G.b_bytes - raw));  // [2][npix]
    const unsigned bar = sb + G.b_bytes + G.tbl_bytes, slot = bar + 8;
    volatile unsigned *slot_ptr = reinterpret_cast<volatile unsigned *>(smem_raw + (slot - raw));

    const int Cin = S.C0 + S.C1, nch = Cin / kBK;
    const int bands = H / R, b = blockIdx.x / bands, y0 = (blockIdx.x - b * bands) * R;
    const int n0 = blockIdx.y * BN;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long wait_limit = g_tc_wait_limit;
    // pixel table: source pixel of every tile pixel in src0's grid and in the
    // full-resolution grid
    for (int hp = tid; hp < G.npix; hp += kThreads) {
        const int hy = hp / G.Wp, hx = hp - hy * G.Wp;
        const int y = wrap(y0 - 1 + hy, H), x = wrap(hx - 1, W);
        const int full = (b * H + y) * W + x;
        tbl[hp] = S.up0 ? (b * (H >> 1) + (y >> 1)) * (W >> 1) + (x >> 1) : full;
        tbl[G.npix + hp] = full;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot), "r"(G.tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();  // also publishes the pixel table
    tc_fence_after();
    const unsigned tmem = *slot_ptr;
    const unsigned lbo_a = 16u * G.apix, lbo_b = 16u * BN;

    int failed = 0, issued = 0;
    for (int c = 0; c < nch; ++c) {
        // the MMAs of the previous chunk read the buffers this one refills
        if (c > 0 && !mbar_wait(bar, (c - 1) & 1, wait_limit)) failed = 1;
        if (__syncthreads_or(failed)) {
            failed = 1;
            break;
        }
        const int cc = c * kBK;
        const bool first = cc < S.C0;
        const bf16 *src = first ? S.s0 + cc : S.s1 + (cc - S.C0);
        const int cs = first ? S.C0 : S.C1;
        const int *tp = tbl + (first ? 0 : G.npix);
        for (int e = tid; e < 4 * G.npix; e += kThreads) {
            const int hp = e >> 2, g = e & 3;
            cp16(sa + g * lbo_a + 16u * hp, src + (size_t)tp[hp] * cs + g * 8);
        }
        for (int e = tid; e < 36 * BN; e += kThreads) {
            const int g = e & 3, nt = e >> 2, n = nt / 9, t = nt - n * 9;
            cp16(sb + (unsigned)(t * 4 + g) * lbo_b + 16u * n, Wk + ((size_t)(n0 + n) * 9 + t) * Cin + cc + g * 8);
        }
        cp_commit();
        cp_wait<0>();
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            for (int mt = 0; mt < G.MT; ++mt)
                for (int t = 0; t < 9; ++t) {
                    const unsigned a0 = sa + 16u * (unsigned)(mt * kBM + (t / 3) * G.Wp + t % 3);
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk)
                        tc_mma(tmem + (unsigned)(mt * BN), desc_ns(a0 + kk * 2 * lbo_a, lbo_a, 128),
                               desc_ns(sb + (unsigned)(t * 4 + kk * 2) * lbo_b, lbo_b, 128), IDESC,
                               (c > 0 || t > 0 || kk > 0) ? 1u : 0u);
                }
            tc_commit(bar);
        }
        issued = c + 1;
    }
    // the last commit tracks every MMA issued before it
    if (issued > 0 && !mbar_wait(bar, (issued - 1) & 1)) failed = 1;
    failed = __syncthreads_or(failed) || issued < nch;
    tc_fence_after();
    const int q = warp & 3, half = warp >> 2;
    for (int mt = 0; mt < G.MT; ++mt) {
        const int s = mt * kBM + q * 32 + lane, y = s / G.Wp, x = s - y * G.Wp;
        const bool valid = !failed && y < R && x < W;
        const size_t pix = (size_t)(b * H + y0 + y) * W + x;
#pragma unroll
        for (int c0 = half * (BN / 2); c0 < (half + 1) * (BN / 2); c0 += 16) {
            float v[16];
            tc_ld16(tmem + ((unsigned)(q * 32) << 16) + (unsigned)(mt * BN + c0), v);
            if (!valid) continue;
            const int co = n0 + c0;
            const size_t o = pix * Cout + co;
            __align__(16) bf16 mk[16];
            if (mask) {
                *reinterpret_cast<uint4 *>(mk) = *reinterpret_cast<const uint4 *>(mask + o);
                *reinterpret_cast<uint4 *>(mk + 8) = *reinterpret_cast<const uint4 *>(mask + o + 8);
            }
            __align__(16) bf16 r[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                float xv = v[e] + (bias ? bias[co + e] : 0.f);
                if (relu) xv = fmaxf(xv, 0.f);
                if (mask && !(__bfloat162float(mk[e]) > 0.f)) xv = 0.f;
                r[e] = __float2bfloat16(xv);
            }
            *reinterpret_cast<uint4 *>(out + o) = *reinterpret_cast<const uint4 *>(r);
            *reinterpret_cast<uint4 *>(out + o + 8) = *reinterpret_cast<const uint4 *>(r + 8);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(G.tcols) : "memory");
    if (failed && tid == 0) atomicExch(&g_tc_error, 1);
}

// ------------------------------------------------------------------ wgrad
// part[z][co][t][ci] = sum over pixels p of split z of dz[p][co] in[p+off(t)][ci].
// Grid (Cout/BMC, 9 * Cin/32, splits), 128 threads as 2 x 2 warps of
// BMC/2 x 16; K steps of 32 pixels.  Both operands are stored pixel-major and
// read with transposing ldmatrix.
template <int BMC>
__global__ void __launch_bounds__(128) k_wgrad(ConvSrc S, const bf16 *__restrict__ dz, int H, int W, int Cout, int P,
                                               int pix_per_split, float *__restrict__ part)
{
    constexpr int A_BYTES = 32 * BMC * 2, STAGE = A_BYTES + 32 * 64;
    constexpr int MT = BMC / 32;  // m16 tiles per warp
    __shared__ __align__(128) unsigned char smem[kStages * STAGE];
    const int Cin = S.C0 + S.C1, nkc = Cin / kBK;
    const int co0 = blockIdx.x * BMC;
    const int t = blockIdx.y / nkc, ci0 = (blockIdx.y - t * nkc) * kBK;
    const int dy = t / 3 - 1, dx = t % 3 - 1;
    const int p_begin = blockIdx.z * pix_per_split;
    const int p_end = min(P, p_begin + pix_per_split);
    const int nk = (p_end - p_begin) / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;
    const int HW = H * W;
    const unsigned sbase = smem_u32(smem);
    // B rows: thread tid loads chunk (tid & 3) of pixel row (tid >> 2)
    const int br = tid >> 2, bc = tid & 3;
    auto load = [&](int k, int stage) {
        int pk = p_begin + k * 32;
        unsigned sa = sbase + stage * STAGE;
        for (int idx = tid; idx < 32 * (BMC / 8); idx += 128) {
            int r = idx / (BMC / 8), c = idx % (BMC / 8);
            unsigned off = BMC == 64 ? swz128(r, c) : swz64(r, c);
            cp16(sa + off, dz + (size_t)(pk + r) * Cout + co0 + c * 8);
        }
        int p = pk + br;
        int b = p / HW, q = p - b * HW, y = q / W, x = q - y * W;
        cp16(sa + A_BYTES + swz64(br, bc), src_at(S, b, wrap(y + dy, H), wrap(x + dx, W), H, W, ci0 + bc * 8));
    };
    float acc[MT][2][4];
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
#pragma unroll
    for (int s = 0; s < kStages - 1; ++s) {
        if (s < nk) load(s, s);
        cp_commit();
    }
    const int lj = lane >> 3, lr = lane & 7;
    for (int k = 0; k < nk; ++k) {
        cp_wait<kStages - 2>();
        __syncthreads();
        int kn = k + kStages - 1;
        if (kn < nk) load(kn, kn % kStages);
        cp_commit();
        unsigned sa = sbase + (k % kStages) * STAGE, sb = sa + A_BYTES;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            unsigned a[MT][4];
#pragma unroll
            for (int mi = 0; mi < MT; ++mi) {
                int row = kk * 16 + lr + (lj >> 1) * 8;
                int ch = (wm * (BMC / 2) + mi * 16 + (lj & 1) * 8) >> 3;
                unsigned off = BMC == 64 ? swz128(row, ch) : swz64(row, ch);
                ldsm4t(sa + off, a[mi][0], a[mi][1], a[mi][2], a[mi][3]);
            }
            unsigned b0, b1, b2, b3;
            {
                int row = kk * 16 + lr + (lj & 1) * 8;
                int ch = (wn * 16 + (lj >> 1) * 8) >> 3;
                ldsm4t(sb + swz64(row, ch), b0, b1, b2, b3);
            }
#pragma unroll
            for (int mi = 0; mi < MT; ++mi) {
                mma16816(acc[mi][0], a[mi], b0, b1);
                mma16816(acc[mi][1], a[mi], b2, b3);
            }
        }
    }
    cp_wait<0>();
    const int g = lane >> 2, t4 = lane & 3;
    float *pz = part + (size_t)blockIdx.z * Cout * 9 * Cin;
#pragma unroll
    for (int mi = 0; mi < MT; ++mi)
#pragma unroll
        for (int ni = 0; ni < 2; ++ni) {
            int ci = ci0 + wn * 16 + ni * 8 + 2 * t4;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                int co = co0 + wm * (BMC / 2) + mi * 16 + g + h * 8;
                *reinterpret_cast<float2 *>(pz + ((size_t)co * 9 + t) * Cin + ci) =
                    make_float2(acc[mi][ni][2 * h], acc[mi][ni][2 * h + 1]);
            }
        }
}

// ------------------------------------------------------------------ wgrad, tcgen05
// The weight gradient on the 5th-generation tensor cores, one GEMM per
// (row tile, output-channel tile, pixel split):
//     D[r][co] = sum_p in[p + off(t)][ci] dz[p][co],   r = t Cin + ci,
// M = 128 rows r (four runs of 32 channels of one tap each), N = BN output
// channels, K = the split's pixels, 32 per pipeline stage (two 128 x BN x 16
// MMAs).  Both operands are copied straight from their pixel-major tensors,
// so they enter the MMA MN-major: 64-byte swizzle atoms of 32 consecutive
// channels x 8 pixels, stored with the four pixel groups of a stage next to
// each other (SBO = 512 B between pixel groups, LBO = 2048 B between channel
// runs).  The FP32 accumulator (128 lanes x BN columns of tensor memory) is
// this split's partial sum part[z][co][t][ci]; k_sum_parts adds the splits
// in a fixed order.  Waits are bounded as in k_conv_tc.
constexpr int kWgPix = 32;  // pixels per stage

template <int BN>
constexpr size_t wgrad_tc_smem()
{
    // + 2 KB: the descriptors of the last stage never reach past the end
    return 1024 + (size_t)kTcStages * (4 * 4 * 512 + (BN / 32) * 4 * 512) + 8 * kTcStages + 16 + 2048;
}

// MN-major SWIZZLE_64B descriptor: start >> 4 | LBO >> 4 (between atoms
// along M or N) | SBO >> 4 (between groups of 8 along K) | version 1 |
// layout 4 = 64-byte swizzle
__device__ __forceinline__ uint64_t desc_mn64(unsigned addr, unsigned lbo, unsigned sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

template <int BN>
__global__ void __launch_bounds__(kThreads) k_wgrad_tc(ConvSrc S, const bf16 *__restrict__ dz, int H, int W, int Cout,
                                                       int P, int pix_per_split, float *__restrict__ part)
{
    constexpr int NA = BN / 32;                 // channel runs (atoms) of the B tile
    constexpr int A_BYTES = 4 * 4 * 512;        // 4 runs x 4 pixel groups
    constexpr int STAGE = A_BYTES + NA * 4 * 512;
    constexpr int BG = BN / 8;                  // 16-byte chunks of dz per pixel
    constexpr int BJ = (kWgPix * BG + kThreads - 1) / kThreads;  // B chunks per thread
    constexpr unsigned TCOLS = BN;
    constexpr unsigned IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                               ((unsigned)(BN >> 3) << 17) | ((unsigned)(128 >> 4) << 24);
    extern __shared__ unsigned char smem_raw[];
    const unsigned raw = smem_u32(smem_raw);
    const unsigned base = (raw + 1023u) & ~1023u;
    const unsigned bar0 = base + kTcStages * STAGE;
    const unsigned slot = bar0 + 8 * kTcStages;
    volatile unsigned *slot_ptr = reinterpret_cast<volatile unsigned *>(smem_raw + (slot - raw));

    const int Cin = S.C0 + S.C1, R = 9 * Cin;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * BN;
    const int p_begin = blockIdx.z * pix_per_split;
    const int nk = (min(P, p_begin + pix_per_split) - p_begin) / kWgPix;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int HW = H * W;
    const long long wait_limit = g_tc_wait_limit;
    // A: this thread copies chunk ag of run ar at pixels apx and apx + 16
    const int ar = (tid >> 2) & 3, ag = tid & 3, apx = tid >> 4;
    const int r_run = m0 + 32 * ar;
    const bool a_on = r_run < R;
    const int a_t = a_on ? r_run / Cin : 0;
    const int a_ci = (a_on ? r_run - a_t * Cin : 0) + 8 * ag;
    const int a_dy = a_t / 3 - 1, a_dx = a_t % 3 - 1;
    // this thread's two pixels of the stage to load next, (b, y, x), advanced
    // by kWgPix pixels per stage
    int lb[2], ly[2], lx[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int p = p_begin + apx + 16 * j;
        lb[j] = p / HW;
        const int q = p - lb[j] * HW;
        ly[j] = q / W;
        lx[j] = q - ly[j] * W;
    }
    auto load = [&](int k, int stage) {
        const int pk = p_begin + k * kWgPix;
        const unsigned sa = base + stage * STAGE, sb = sa + A_BYTES;
        if (a_on) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int px = apx + 16 * j;
                cp16_ca(sa + (ar * 4 + (px >> 3)) * 512 + swz64(px & 7, ag),
                        src_at(S, lb[j], wrap(ly[j] + a_dy, H), wrap(lx[j] + a_dx, W), H, W, a_ci));
                lx[j] += kWgPix;
                while (lx[j] >= W) {
                    lx[j] -= W;
                    if (++ly[j] == H) {
                        ly[j] = 0;
                        ++lb[j];
                    }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < BJ; ++j) {
            const int idx = tid + kThreads * j;
            if (idx < kWgPix * BG) {
                const int px = idx / BG, c = idx % BG;
                cp16(sb + ((c >> 2) * 4 + (px >> 3)) * 512 + swz64(px & 7, c & 3),
                     dz + (size_t)(pk + px) * Cout + n0 + 8 * c);
            }
        }
    };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot), "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < kTcStages; ++s) mbar_init(bar0 + 8 * s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    // runs past the last row (9 Cin not a multiple of 128) stay zero
    for (int s = 0; s < kTcStages; ++s)
        for (int i = tid; i < 4 * 128; i += kThreads) {
            const int run = i >> 7;
            if (m0 + 32 * run >= R)
                *reinterpret_cast<uint4 *>(smem_raw + (base - raw) + s * STAGE + run * 2048 + (i & 127) * 16) =
                    make_uint4(0u, 0u, 0u, 0u);
        }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *slot_ptr;

#pragma unroll
    for (int s = 0; s < kTcStages - 1; ++s) {
        if (s < nk) load(s, s);
        cp_commit();
    }
    int failed = 0, issued = 0;
    for (int k = 0; k < nk; ++k) {
        const int s = k % kTcStages;
        cp_wait<kTcStages - 2>();
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        if (__syncthreads_or(failed)) {
            failed = 1;
            break;
        }
        if (tid == 0) {
            tc_fence_after();
            const unsigned sa = base + s * STAGE, sb = sa + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < 2; ++kk)
                tc_mma(tmem, desc_mn64(sa + kk * 1024, 2048, 512), desc_mn64(sb + kk * 1024, 2048, 512), IDESC,
                       (k > 0 || kk > 0) ? 1u : 0u);
            tc_commit(bar0 + 8 * s);
        }
        issued = k + 1;
        const int kn = k + kTcStages - 1;
        if (kn < nk) {
            const int sn = kn % kTcStages;  // the stage the MMAs of iteration k-1 read
            if (k >= 1 && !mbar_wait(bar0 + 8 * sn, ((k - 1) / kTcStages) & 1, wait_limit)) failed = 1;
            if (!failed) load(kn, sn);
        }
        cp_commit();
    }
    cp_wait<0>();
    if (issued > 0 && !mbar_wait(bar0 + 8 * ((issued - 1) % kTcStages), ((issued - 1) / kTcStages) & 1)) failed = 1;
    failed = __syncthreads_or(failed) || issued < nk;
    tc_fence_after();
    const int q = warp & 3, half = warp >> 2;
    const int r = m0 + q * 32 + lane;
    const int t = r / Cin, ci = r - t * Cin;
    float *pz = part + (size_t)blockIdx.z * Cout * R;
#pragma unroll
    for (int c0 = half * (BN / 2); c0 < (half + 1) * (BN / 2); c0 += 16) {
        float v[16];
        tc_ld16(tmem + ((unsigned)(q * 32) << 16) + (unsigned)c0, v);
        if (failed || r >= R) continue;
        if (nk == 0) {
#pragma unroll
            for (int e = 0; e < 16; ++e) v[e] = 0.f;
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) pz[((size_t)(n0 + c0 + e) * 9 + t) * Cin + ci] = v[e];
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TCOLS) : "memory");
    if (failed && tid == 0) atomicExch(&g_tc_error, 1);
}

// out[i] = sum_{z < nz} part[z * n + i], in order of z.
__global__ void k_sum_parts(const float *__restrict__ part, int nz, long long n, float *__restrict__ out)
{
    // four running sums over z = 4k + j (four loads in flight), added as
    // (s0 + s1) + (s2 + s3): a fixed order
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float s[4] = {0.f, 0.f, 0.f, 0.f};
        int z = 0;
        for (; z + 3 < nz; z += 4) {
#pragma unroll
            for (int j = 0; j < 4; ++j) s[j] += __ldg(part + (size_t)(z + j) * n + i);
        }
        for (int j = 0; z < nz; ++z, ++j) s[j] += __ldg(part + (size_t)z * n + i);
        out[i] = (s[0] + s[1]) + (s[2] + s[3]);
    }
}

// part[blk][c] = sum over the block's pixels of dz[p][c]; C a multiple of 32
// (blockIdx.y takes channels in slices of 256).
__global__ void __launch_bounds__(256) k_colsum(const bf16 *__restrict__ dz, int P, int C, int pix_per_blk,
                                                float *__restrict__ part)
{
    // block (x, y): pixels [x pix_per_blk, (x + 1) pix_per_blk), channels
    // [256 y, 256 y + Cs).  Each thread sums 8 channels (one 16-byte vector)
    // of every G-th pixel of the run, four vectors in flight; the block's G
    // partial sums of a channel are then added in a fixed order.
    __shared__ float sh[256][8];
    const int c0 = 256 * blockIdx.y, Cs = min(256, C - c0);
    const int ng = Cs >> 3, G = 256 / ng;  // channel groups per pixel, pixels per pass
    const int cg = threadIdx.x % ng, r = threadIdx.x / ng;
    dz += c0;
    const int p0 = blockIdx.x * pix_per_blk, p1 = min(P, p0 + pix_per_blk);
    float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const bool in = r < G;
    int p = p0 + r;
    for (; in && p + 3 * G < p1; p += 4 * G) {
        uint4 u[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) u[k] = __ldg(reinterpret_cast<const uint4 *>(dz + (size_t)(p + k * G) * C) + cg);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u[k]);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2 f = __bfloat1622float2(h[e]);
                a[2 * e] += f.x;
                a[2 * e + 1] += f.y;
            }
        }
    }
    for (; in && p < p1; p += G) {
        const uint4 u = __ldg(reinterpret_cast<const uint4 *>(dz + (size_t)p * C) + cg);
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 f = __bfloat1622float2(h[e]);
            a[2 * e] += f.x;
            a[2 * e + 1] += f.y;
        }
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) sh[threadIdx.x][e] = a[e];
    __syncthreads();
    if ((int)threadIdx.x < Cs) {
        const int c = threadIdx.x;
        float t = 0.f;
        for (int k = 0; k < G; ++k) t += sh[k * ng + (c >> 3)][c & 7];
        part[(size_t)blockIdx.x * C + c0 + c] = t;
    }
}

// ------------------------------------------------------------------ pointwise
// x[p][0..31] = (n_x, n_y, n_z, f0..f3, 0...), one thread per 8 channels.
__global__ void k_build_input(const float4 *__restrict__ spins, const float *__restrict__ feat, int HW, long long P,
                              bf16 *__restrict__ x)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= P * 4) return;
    long long p = i >> 2;
    int part = (int)(i & 3);
    __align__(16) bf16 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __float2bfloat16(0.f);
    if (part == 0) {
        float4 n = spins[p];
        const float *f = feat + (p / HW) * SP_UNET_FEATURES;
        v[0] = __float2bfloat16(n.x);
        v[1] = __float2bfloat16(n.y);
        v[2] = __float2bfloat16(n.z);
        v[3] = __float2bfloat16(f[0]);
        v[4] = __float2bfloat16(f[1]);
        v[5] = __float2bfloat16(f[2]);
        v[6] = __float2bfloat16(f[3]);
    }
    *reinterpret_cast<uint4 *>(x + p * SP_UNET_IN_CH + part * 8) = *reinterpret_cast<uint4 *>(v);
}

// 2x2 mean pooling of a [B][H][W][C] tensor, one thread per 8 channels of an
// output pixel.
__global__ void k_pool(const bf16 *__restrict__ a, int B, int H, int W, int C, bf16 *__restrict__ out)
{
    int Ho = H / 2, Wo = W / 2, G = C / 8;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)B * Ho * Wo * G) return;
    int g = (int)(i % G);
    long long q = i / G;
    int xo = (int)(q % Wo), yo = (int)((q / Wo) % Ho), b = (int)(q / ((long long)Wo * Ho));
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        size_t src = ((size_t)(b * H + 2 * yo + (d >> 1)) * W + 2 * xo + (d & 1)) * C + g * 8;
        uint4 u = *reinterpret_cast<const uint4 *>(a + src);
        const bf16 *e = reinterpret_cast<const bf16 *>(&u);
#pragma unroll
        for (int k = 0; k < 8; ++k) s[k] += __bfloat162float(e[k]);
    }
    __align__(16) bf16 o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) o[k] = __float2bfloat16(0.25f * s[k]);
    *reinterpret_cast<uint4 *>(out + (size_t)q * C + g * 8) = *reinterpret_cast<uint4 *>(o);
}

// Backward of a concatenation [up(coarse) C0 | skip C1] at H x W:
// dcoarse[q][c] = (sum of the 2x2 fine gradients of channel c) where
// coarse[q][c] > 0 (ReLU), else 0.  One thread per 8 channels of a coarse pixel.
__global__ void k_cat_coarse(const bf16 *__restrict__ dcat, int C0, int C1, const bf16 *__restrict__ coarse, int B,
                             int H, int W, bf16 *__restrict__ dcoarse)
{
    int Ho = H / 2, Wo = W / 2, G = C0 / 8, Ct = C0 + C1;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)B * Ho * Wo * G) return;
    int g = (int)(i % G);
    long long q = i / G;
    int xo = (int)(q % Wo), yo = (int)((q / Wo) % Ho), b = (int)(q / ((long long)Wo * Ho));
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        size_t src = ((size_t)(b * H + 2 * yo + (d >> 1)) * W + 2 * xo + (d & 1)) * Ct + g * 8;
        uint4 u = *reinterpret_cast<const uint4 *>(dcat + src);
        const bf16 *e = reinterpret_cast<const bf16 *>(&u);
#pragma unroll
        for (int k = 0; k < 8; ++k) s[k] += __bfloat162float(e[k]);
    }
    uint4 um = *reinterpret_cast<const uint4 *>(coarse + (size_t)q * C0 + g * 8);
    const bf16 *m = reinterpret_cast<const bf16 *>(&um);
    __align__(16) bf16 o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) o[k] = __float2bfloat16(__bfloat162float(m[k]) > 0.f ? s[k] : 0.f);
    *reinterpret_cast<uint4 *>(dcoarse + (size_t)q * C0 + g * 8) = *reinterpret_cast<uint4 *>(o);
}

// dz[p][c] = (dcat[p][C0 + c] + dpool[p/2][c] / 4) where a[p][c] > 0, else 0:
// the skip tensor a feeds both the concatenation and the 2x2 mean pool.
__global__ void k_skip_grad(const bf16 *__restrict__ dcat, int C0, int C1, const bf16 *__restrict__ dpool,
                            const bf16 *__restrict__ a, int B, int H, int W, bf16 *__restrict__ dz)
{
    int G = C1 / 8, Ct = C0 + C1;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)B * H * W * G) return;
    int g = (int)(i % G);
    long long p = i / G;
    int x = (int)(p % W), y = (int)((p / W) % H), b = (int)(p / ((long long)W * H));
    uint4 u0 = *reinterpret_cast<const uint4 *>(dcat + (size_t)p * Ct + C0 + g * 8);
    uint4 u1 = *reinterpret_cast<const uint4 *>(dpool + ((size_t)(b * (H / 2) + y / 2) * (W / 2) + x / 2) * C1 + g * 8);
    uint4 u2 = *reinterpret_cast<const uint4 *>(a + (size_t)p * C1 + g * 8);
    const bf16 *e0 = reinterpret_cast<const bf16 *>(&u0), *e1 = reinterpret_cast<const bf16 *>(&u1),
               *e2 = reinterpret_cast<const bf16 *>(&u2);
    __align__(16) bf16 o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        float v = __bfloat162float(e0[k]) + 0.25f * __bfloat162float(e1[k]);
        o[k] = __float2bfloat16(__bfloat162float(e2[k]) > 0.f ? v : 0.f);
    }
    *reinterpret_cast<uint4 *>(dz + (size_t)p * C1 + g * 8) = *reinterpret_cast<uint4 *>(o);
}

// ------------------------------------------------------------------ head
constexpr int kHeadVals = 3 * 32 + 3 + 1;  // dWh, dbh, loss
constexpr int kHeadRow = 37;                 // floats per pixel row of k_head's block sums

// Per pixel: y = Wh a + bh, m = y/|y|.  predict: out[p] = (m, 0).  train:
// loss 1 - m.m_t, dy = -(m_t - (m.m_t) m) / (|y| P), dz[p][c] = (Wh^T dy)_c
// where a[p][c] > 0, and per-block sums of dy a^T, dy and the loss.
template <bool TRAIN>
__global__ void __launch_bounds__(256) k_head(const bf16 *__restrict__ a, const float *__restrict__ Wh,
                                              const float *__restrict__ target, long long P, float inv_P,
                                              float4 *__restrict__ out, bf16 *__restrict__ dz, float *__restrict__ part)
{
    __shared__ float w[3 * 32 + 3];
    // per-pixel values for the block sums (row of 36 floats, padded to 37
    // against bank conflicts of the column reads)
    __shared__ float hv[256 * kHeadRow];
    for (int k = threadIdx.x; k < 3 * 32 + 3; k += blockDim.x) w[k] = Wh[k];
    __syncthreads();
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float av[32];
    float y[3] = {0.f, 0.f, 0.f};
    bool live = p < P;
    if (live) {
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            uint4 u = *reinterpret_cast<const uint4 *>(a + p * 32 + g * 8);
            const bf16 *e = reinterpret_cast<const bf16 *>(&u);
#pragma unroll
            for (int k = 0; k < 8; ++k) av[g * 8 + k] = __bfloat162float(e[k]);
        }
#pragma unroll
        for (int o = 0; o < 3; ++o) {
            float s = w[96 + o];
#pragma unroll
            for (int c = 0; c < 32; ++c) s = fmaf(w[o * 32 + c], av[c], s);
            y[o] = s;
        }
    } else {
#pragma unroll
        for (int c = 0; c < 32; ++c) av[c] = 0.f;
    }
    float ny = sqrtf(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
    float inv = ny > 0.f ? 1.f / ny : 0.f;
    float m[3] = {y[0] * inv, y[1] * inv, y[2] * inv};
    if (!TRAIN) {
        if (live) out[p] = make_float4(m[0], m[1], m[2], 0.f);
        return;
    }
    float dy[3] = {0.f, 0.f, 0.f}, loss = 0.f;
    if (live) {
        float4 tt = reinterpret_cast<const float4 *>(target)[p];
        float mt[3] = {tt.x, tt.y, tt.z};
        float c = m[0] * mt[0] + m[1] * mt[1] + m[2] * mt[2];
        loss = 1.f - c;
        float s = -inv * inv_P;
#pragma unroll
        for (int o = 0; o < 3; ++o) dy[o] = s * (mt[o] - c * m[o]);
        __align__(16) bf16 d[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            float v = w[k] * dy[0] + w[32 + k] * dy[1] + w[64 + k] * dy[2];
            d[k] = __float2bfloat16(av[k] > 0.f ? v : 0.f);
        }
#pragma unroll
        for (int g = 0; g < 4; ++g)
            *reinterpret_cast<uint4 *>(dz + p * 32 + g * 8) = reinterpret_cast<const uint4 *>(d)[g];
    }
    // block sums of value j of kHeadVals (dWh[o][c] = sum dy[o] av[c], dbh[o]
    // = sum dy[o], the loss): every thread leaves its pixel's 32 activations,
    // 3 output gradients and loss in shared memory, then thread j adds value
    // j over the block's pixels in pixel order
    float *row = hv + threadIdx.x * kHeadRow;
#pragma unroll
    for (int c = 0; c < 32; ++c) row[c] = av[c];
    row[32] = dy[0];
    row[33] = dy[1];
    row[34] = dy[2];
    row[35] = loss;
    __syncthreads();
    const int j = threadIdx.x;
    if (j < kHeadVals) {
        float s = 0.f;
        if (j < 96) {
            const int o = j >> 5, c = j & 31;
            for (int k = 0; k < (int)blockDim.x; ++k) s = fmaf(hv[k * kHeadRow + 32 + o], hv[k * kHeadRow + c], s);
        } else {
            const int col = j < 99 ? 32 + (j - 96) : 35;
            for (int k = 0; k < (int)blockDim.x; ++k) s += hv[k * kHeadRow + col];
        }
        part[(size_t)j * gridDim.x + blockIdx.x] = s;  // value-major: k_head_reduce reads a row
    }
}

// grad[0..98] = sum of the per-block head sums; *loss = their loss sum / P.
// Value j = blockIdx.x of the head's block partials (value-major rows of
// nblk): each thread adds a strided subset in FP64, then a fixed-order tree
// over the block.
__global__ void __launch_bounds__(256) k_head_reduce(const float *__restrict__ part, int nblk, double inv_P,
                                                     float *__restrict__ grad, double *__restrict__ loss)
{
    __shared__ double sh[256];
    const int j = blockIdx.x;
    const float *row = part + (size_t)j * nblk;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += row[b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (j < 99)
            grad[j] = (float)sh[0];
        else if (loss)
            *loss = sh[0] * inv_P;
    }
}

// ------------------------------------------------------------------ weights
struct LayerTab {
    int n;
    long long w_off[SP_UNET_LAYERS], bf_off[SP_UNET_LAYERS];
    int cout[SP_UNET_LAYERS], cin[SP_UNET_LAYERS];
};

// Wk[co][t][ci] = bf16(W) and Wt[ci][8-t][co] = bf16(W) for every layer.
__global__ void k_prep_weights(LayerTab L, const float *__restrict__ params, bf16 *__restrict__ wk, bf16 *__restrict__ wt)
{
    for (int l = 0; l < L.n; ++l) {
        int Co = L.cout[l], Ci = L.cin[l];
        long long n = (long long)Co * 9 * Ci;
        const float *W = params + L.w_off[l];
        bf16 *k = wk + L.bf_off[l], *tr = wt + L.bf_off[l];
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
            int ci = (int)(i % Ci);
            long long r = i / Ci;
            int t = (int)(r % 9), co = (int)(r / 9);
            bf16 v = __float2bfloat16(W[i]);
            k[i] = v;
            tr[((size_t)ci * 9 + (8 - t)) * Co + co] = v;
        }
    }
}

__global__ void k_transpose(const bf16 *__restrict__ W, int Co, int Ci, bf16 *__restrict__ Wt)
{
    long long n = (long long)Co * 9 * Ci;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int ci = (int)(i % Ci);
        long long r = i / Ci;
        int t = (int)(r % 9), co = (int)(r / 9);
        Wt[((size_t)ci * 9 + (8 - t)) * Co + co] = W[i];
    }
}

// Adam (Kingma & Ba): m, v moving averages of g and g^2, bias-corrected step.
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float gi = g[i];
        float mi = b1 * m[i] + (1.f - b1) * gi;
        float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

// ------------------------------------------------------------------ launchers
// exact grid for one thread per item
unsigned blocks(long long n, int threads = 256) { return (unsigned)((n + threads - 1) / threads); }

// capped grid for grid-stride loops
int grid_for(long long n, int threads = 256)
{
    long long b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > 152LL * 64 ? 152LL * 64 : b));
}

bool conv_shape_ok(int C0, int C1, int up0, int B, int H, int W, int Cout)
{
    long long P = (long long)B * H * W;
    if (B < 1 || H < 1 || W < 1 || P % kBM != 0) return false;
    if (C0 < 32 || C0 % 32 || C1 < 0 || C1 % 32 || Cout < 32 || Cout % 32) return false;
    if (up0 && (H % 2 || W % 2)) return false;
    return P < (1LL << 31) - 256;
}

int g_use_tc = 3;  // 0: mma.sync, 1: tcgen05, 2: tcgen05 warp-specialised, 3: tcgen05 halo tiles (default)

template <int BN>
cudaError_t conv_tc_launch(dim3 grid, const ConvSrc &S, const bf16 *W, const float *bias, int relu, const bf16 *mask,
                           int H, int Wd, int Cout, bf16 *out, cudaStream_t st)
{
    static bool attr = false;  // per process; the attribute is per function
    constexpr size_t sm = conv_tc_smem<BN>();
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_conv_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_conv_tc<BN><<<grid, kThreads, sm, st>>>(S, W, bias, relu, mask, H, Wd, Cout, out);
    return cudaGetLastError();
}

template <int BN>
cudaError_t conv_ws_launch(dim3 grid, const ConvSrc &S, const bf16 *W, const float *bias, int relu, const bf16 *mask,
                           int H, int Wd, int Cout, bf16 *out, cudaStream_t st)
{
    static bool attr = false;
    constexpr size_t sm = conv_ws_smem<BN>();
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_conv_ws<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_conv_ws<BN><<<grid, kThreads, sm, st>>>(S, W, bias, relu, mask, H, Wd, Cout, out);
    return cudaGetLastError();
}

// Kernel 3 takes the halo tiles for image rows of at least this many pixels
// and kernel 1 below.  Measured at batch 64 (forward, ms, kernel 1 -> halo):
// 128^2 32->32 0.109 -> 0.087, 96->32 0.245 -> 0.172, 64^2 64->64 0.065 ->
// 0.059; 32^2 128->128 0.048 -> 0.077, 384->128 0.115 -> 0.182, 16^2
// 256->256 0.046 -> 0.073: on short rows with many channel chunks the
// halo kernel's single stage (copies, then MMAs) loses to kernel 1's
// four-stage pipeline.
constexpr int kHaloMinWidth = 64;

// Rows per CTA of the halo-tile kernel: the most of 8, 4, 2, 1 that divide H
// with the accumulators and the stage inside a two-per-SM share; 0 if none.
int halo_rows(int H, int W, int BN)
{
    for (int R = 8; R >= 1; R /= 2) {
        if (H % R) continue;
        const HaloGeom g = halo_geom(R, W, BN);
        if ((unsigned)(g.MT * BN) <= kHaloTmemMax && g.smem <= kHaloSmemMax) return R;
    }
    return 0;
}

template <int BN>
cudaError_t conv_halo_launch(int R, const ConvSrc &S, const bf16 *W, const float *bias, int relu, const bf16 *mask,
                             int B, int H, int Wd, int Cout, bf16 *out, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(k_conv_halo<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHaloSmemMax);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const HaloGeom g = halo_geom(R, Wd, BN);
    dim3 grid((unsigned)(B * (H / R)), (unsigned)(Cout / BN));
    k_conv_halo<BN><<<grid, kThreads, g.smem, st>>>(S, W, bias, relu, mask, H, Wd, Cout, R, out);
    return cudaGetLastError();
}

cudaError_t conv_launch(const ConvSrc &S, const bf16 *W, const float *bias, int relu, const bf16 *mask, int B, int H,
                        int Wd, int Cout, bf16 *out, cudaStream_t st)
{
    long long P = (long long)B * H * Wd;
    int bn = Cout % 128 == 0 ? 128 : (Cout % 64 == 0 ? 64 : 32);
    dim3 grid((unsigned)(P / kBM), (unsigned)(Cout / bn));
    if (g_use_tc == 3 && Wd >= kHaloMinWidth) {
        const int R = halo_rows(H, Wd, bn);
        if (R > 0) {
            switch (bn) {
            case 128: return conv_halo_launch<128>(R, S, W, bias, relu, mask, B, H, Wd, Cout, out, st);
            case 64: return conv_halo_launch<64>(R, S, W, bias, relu, mask, B, H, Wd, Cout, out, st);
            default: return conv_halo_launch<32>(R, S, W, bias, relu, mask, B, H, Wd, Cout, out, st);
            }
        }
    }
    if (g_use_tc == 2) {
        switch (bn) {
        case 128: return conv_ws_launch<128>(grid, S, W, bias, relu, mask, H, Wd, Cout, out, st);
        case 64: return conv_ws_launch<64>(grid, S, W, bias, relu, mask, H, Wd, Cout, out, st);
        default: return conv_ws_launch<32>(grid, S, W, bias, relu, mask, H, Wd, Cout, out, st);
        }
    }
    if (g_use_tc) {  // 1, and 3 where the halo tiles do not fit
        switch (bn) {
        case 128: return conv_tc_launch<128>(grid, S, W, bias, relu, mask, H, Wd, Cout, out, st);
        case 64: return conv_tc_launch<64>(grid, S, W, bias, relu, mask, H, Wd, Cout, out, st);
        default: return conv_tc_launch<32>(grid, S, W, bias, relu, mask, H, Wd, Cout, out, st);
        }
    }
    size_t sm;
    switch (bn) {
    case 128:
        sm = kStages * (kBM * 64 + 128 * 64);
        k_conv<128><<<grid, kThreads, sm, st>>>(S, W, bias, relu, mask, H, Wd, Cout, out);
        break;
    case 64:
        sm = kStages * (kBM * 64 + 64 * 64);
        k_conv<64><<<grid, kThreads, sm, st>>>(S, W, bias, relu, mask, H, Wd, Cout, out);
        break;
    default:
        sm = kStages * (kBM * 64 + 32 * 64);
        k_conv<32><<<grid, kThreads, sm, st>>>(S, W, bias, relu, mask, H, Wd, Cout, out);
    }
    return cudaGetLastError();
}

struct WgradPlan {
    int bmc, splits, pix_per_split, bias_blocks, bias_pix;
    int tc_bn;              // > 0: k_wgrad_tc with this many output channels per CTA
    long long part_floats;  // partial weight sums
    long long bias_floats;  // partial bias sums
};

int wgrad_tc_bn(int Cout) { return Cout % 256 == 0 ? 256 : (Cout % 128 == 0 ? 128 : (Cout % 64 == 0 ? 64 : 32)); }

// Pixel splits: enough CTAs for a few per SM over the tiles; each split a
// whole number of 32-pixel steps.
WgradPlan wgrad_plan(long long P, int Cin, int Cout, bool tc)
{
    WgradPlan w;
    w.bmc = Cout % 64 == 0 ? 64 : 32;
    w.tc_bn = tc ? wgrad_tc_bn(Cout) : 0;
    long long base = tc ? ((9LL * Cin + 127) / 128) * (Cout / w.tc_bn) : (long long)(Cout / w.bmc) * 9 * (Cin / kBK);
    long long chunks = P / 32;
    // tcgen05: one wave of CTAs at the occupancy the stages' shared memory
    // allows (fewer splits also mean fewer partial sums to add up)
    const long long res = !tc ? 4 : (w.tc_bn == 256 ? 2 : (w.tc_bn == 128 ? 3 : (w.tc_bn == 64 ? 4 : 5)));
    long long s = tc ? std::max(1LL, 152 * res / base) : (4LL * 152 + base - 1) / base;
    if (s > chunks) s = chunks;
    if (s < 1) s = 1;
    long long per = (chunks + s - 1) / s;
    w.pix_per_split = (int)(per * 32);
    w.splits = (int)((chunks + per - 1) / per);
    w.part_floats = (long long)w.splits * Cout * 9 * Cin;
    // bias partial sums: one wave of two blocks per SM (at least 1024 pixels
    // each)
    w.bias_pix = (int)std::max(1024LL, ((P + 2 * 152 - 1) / (2 * 152) + 63) / 64 * 64);
    w.bias_blocks = (int)((P + w.bias_pix - 1) / w.bias_pix);
    w.bias_floats = (long long)w.bias_blocks * Cout;
    return w;
}

// workspace for either kernel, so that a workspace sized once stays valid
// when the kernel choice changes
long long wgrad_ws_bytes(long long P, int Cin, int Cout)
{
    long long b = 0;
    for (int tc = 0; tc < 2; ++tc) {
        WgradPlan w = wgrad_plan(P, Cin, Cout, tc != 0);
        b = std::max(b, (w.part_floats + w.bias_floats) * (long long)sizeof(float));
    }
    return b;
}

template <int BN>
cudaError_t wgrad_tc_launch(dim3 grid, const ConvSrc &S, const bf16 *dz, int H, int Wd, int Cout, int P, int pps,
                            float *part, cudaStream_t st)
{
    static bool attr = false;  // per process; the attribute is per function
    constexpr size_t sm = wgrad_tc_smem<BN>();
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_wgrad_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_wgrad_tc<BN><<<grid, kThreads, sm, st>>>(S, dz, H, Wd, Cout, P, pps, part);
    return cudaGetLastError();
}

cudaError_t wgrad_launch(const ConvSrc &S, const bf16 *dz, int B, int H, int Wd, int Cout, float *dW, float *db,
                         float *ws, cudaStream_t st)
{
    long long P = (long long)B * H * Wd;
    int Cin = S.C0 + S.C1;
    WgradPlan w = wgrad_plan(P, Cin, Cout, g_use_tc != 0);
    if (w.tc_bn) {
        dim3 grid((unsigned)((9 * Cin + 127) / 128), (unsigned)(Cout / w.tc_bn), (unsigned)w.splits);
        cudaError_t e;
        switch (w.tc_bn) {
        case 256: e = wgrad_tc_launch<256>(grid, S, dz, H, Wd, Cout, (int)P, w.pix_per_split, ws, st); break;
        case 128: e = wgrad_tc_launch<128>(grid, S, dz, H, Wd, Cout, (int)P, w.pix_per_split, ws, st); break;
        case 64: e = wgrad_tc_launch<64>(grid, S, dz, H, Wd, Cout, (int)P, w.pix_per_split, ws, st); break;
        default: e = wgrad_tc_launch<32>(grid, S, dz, H, Wd, Cout, (int)P, w.pix_per_split, ws, st); break;
        }
        if (e != cudaSuccess) return e;
    } else {
        dim3 grid((unsigned)(Cout / w.bmc), (unsigned)(9 * (Cin / kBK)), (unsigned)w.splits);
        if (w.bmc == 64)
            k_wgrad<64><<<grid, 128, 0, st>>>(S, dz, H, Wd, Cout, (int)P, w.pix_per_split, ws);
        else
            k_wgrad<32><<<grid, 128, 0, st>>>(S, dz, H, Wd, Cout, (int)P, w.pix_per_split, ws);
    }
    long long n = (long long)Cout * 9 * Cin;
    k_sum_parts<<<grid_for(n), 256, 0, st>>>(ws, w.splits, n, dW);
    if (db) {
        float *bp = ws + w.part_floats;
        k_colsum<<<dim3(w.bias_blocks, (Cout + 255) / 256), 256, 0, st>>>(dz, (int)P, Cout, w.bias_pix, bp);
        k_sum_parts<<<grid_for(Cout), 256, 0, st>>>(bp, w.bias_blocks, Cout, db);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ network
struct LayerDef {
    int cin0, up, cin1, cout, level;
};
// inputs: cin0 channels of the previous tensor (upsampled when up), cin1
// skip channels; level 0..3 = L, L/2, L/4, L/8
const LayerDef kLayers[SP_UNET_LAYERS] = {
    {32, 0, 0, 32, 0},   {32, 0, 0, 32, 0},     {32, 0, 0, 64, 1},   {64, 0, 0, 64, 1},   {64, 0, 0, 128, 2},
    {128, 0, 0, 128, 2}, {128, 0, 0, 256, 3},   {256, 0, 0, 256, 3}, {256, 1, 128, 128, 2}, {128, 0, 0, 128, 2},
    {128, 1, 64, 64, 1}, {64, 0, 0, 64, 1},     {64, 1, 32, 32, 0},  {32, 0, 0, 32, 0}};

struct Offsets {
    long long w[SP_UNET_LAYERS + 1], b[SP_UNET_LAYERS + 1], total;
};

Offsets param_offsets()
{
    Offsets o;
    long long k = 0;
    for (int l = 0; l < SP_UNET_LAYERS; ++l) {
        int cin = kLayers[l].cin0 + kLayers[l].cin1;
        o.w[l] = k;
        k += (long long)kLayers[l].cout * 9 * cin;
        o.b[l] = k;
        k += kLayers[l].cout;
    }
    o.w[SP_UNET_LAYERS] = k;
    k += 3 * 32;
    o.b[SP_UNET_LAYERS] = k;
    k += 3;
    o.total = k;
    return o;
}

}  // namespace

struct sp_unet {
    int L = 0, bmax = 0;
    std::string err;
    Offsets off;
    LayerTab tab;
    long long n_bf = 0;  // BF16 weight elements
    void *arena = nullptr;
    float *params = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    bf16 *wk = nullptr, *wt = nullptr;
    bf16 *x = nullptr, *act[SP_UNET_LAYERS] = {}, *pool[3] = {}, *dz[SP_UNET_LAYERS] = {}, *dpool[3] = {};
    bf16 *dcat[3] = {};  // level 0..2 concatenation gradients
    float *ws = nullptr, *head_part = nullptr;
    long long ws_floats = 0;
    int head_blocks = 0;
};

namespace {

int ufail(sp_unet *n, int code, const char *fmt, ...)
{
    if (n) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        n->err = buf;
    }
    return code;
}

int cfail(sp_unet *n, cudaError_t e, const char *what)
{
    return ufail(n, SP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

long long level_pixels(const sp_unet *n, int batch, int level)
{
    long long s = n->L >> level;
    return (long long)batch * s * s;
}

ConvSrc layer_src(const sp_unet *n, int l)
{
    ConvSrc S{nullptr, kLayers[l].cin0, kLayers[l].up, nullptr, kLayers[l].cin1};
    switch (l) {
    case 0: S.s0 = n->x; break;
    case 2: S.s0 = n->pool[0]; break;
    case 4: S.s0 = n->pool[1]; break;
    case 6: S.s0 = n->pool[2]; break;
    case 8: S.s0 = n->act[7]; S.s1 = n->act[5]; break;
    case 10: S.s0 = n->act[9]; S.s1 = n->act[3]; break;
    case 12: S.s0 = n->act[11]; S.s1 = n->act[1]; break;
    default: S.s0 = n->act[l - 1];
    }
    return S;
}

int check_batch(sp_unet *n, int batch)
{
    if (batch < 1 || batch > n->bmax) return ufail(n, SP_ERR_ARG, "batch %d outside 1..%d", batch, n->bmax);
    if (level_pixels(n, batch, 3) % kBM) return ufail(n, SP_ERR_ARG, "batch * (L/8)^2 must be a multiple of 128");
    return SP_OK;
}

cudaError_t forward(sp_unet *n, const float *spins, const float *feat, int batch, cudaStream_t st)
{
    int L = n->L;
    long long P0 = level_pixels(n, batch, 0);
    k_build_input<<<blocks(P0 * 4), 256, 0, st>>>((const float4 *)spins, feat, L * L, P0, n->x);
    for (int l = 0; l < SP_UNET_LAYERS; ++l) {
        int s = L >> kLayers[l].level;
        cudaError_t e = conv_launch(layer_src(n, l), n->wk + n->tab.bf_off[l], n->params + n->off.b[l], 1, nullptr,
                                    batch, s, s, kLayers[l].cout, n->act[l], st);
        if (e != cudaSuccess) return e;
        if (l == 1 || l == 3 || l == 5) {
            int k = l / 2, C = kLayers[l].cout;
            long long work = level_pixels(n, batch, k + 1) * (C / 8);
            k_pool<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(n->act[l], batch, s, s, C, n->pool[k]);
        }
    }
    return cudaGetLastError();
}

cudaError_t backward(sp_unet *n, int batch, cudaStream_t st)
{
    int L = n->L;
    for (int l = SP_UNET_LAYERS - 1; l >= 0; --l) {
        const LayerDef &d = kLayers[l];
        int s = L >> d.level;
        ConvSrc S = layer_src(n, l);
        cudaError_t e = wgrad_launch(S, n->dz[l], batch, s, s, d.cout, n->grad + n->off.w[l], n->grad + n->off.b[l],
                                     n->ws, st);
        if (e != cudaSuccess) return e;
        if (l == 0) break;
        int cin = d.cin0 + d.cin1;
        ConvSrc G{n->dz[l], d.cout, 0, nullptr, 0};
        const bf16 *wt = n->wt + n->tab.bf_off[l];
        if (d.cin1) {  // concatenation input: dcat, then split it
            int k = d.level;
            e = conv_launch(G, wt, nullptr, 0, nullptr, batch, s, s, cin, n->dcat[k], st);
            if (e != cudaSuccess) return e;
            long long work = level_pixels(n, batch, k + 1) * (d.cin0 / 8);
            k_cat_coarse<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(n->dcat[k], d.cin0, d.cin1, S.s0, batch, s, s,
                                                                        n->dz[l - 1]);
        } else if (l == 2 || l == 4 || l == 6) {  // pooled input: gradient of the pool, then the skip tensor
            int k = l / 2 - 1;
            e = conv_launch(G, wt, nullptr, 0, nullptr, batch, s, s, cin, n->dpool[k], st);
            if (e != cudaSuccess) return e;
            int sf = L >> k, Cs = kLayers[l - 1].cout;
            long long work = level_pixels(n, batch, k) * (Cs / 8);
            // the decoder layer that reads skip tensor act[l-1]
            int dec = 12 - 2 * k;
            k_skip_grad<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(n->dcat[k], kLayers[dec].cin0, Cs, n->dpool[k],
                                                                       n->act[l - 1], batch, sf, sf, n->dz[l - 1]);
        } else {  // plain input: mask with the input's ReLU
            e = conv_launch(G, wt, nullptr, 0, n->act[l - 1], batch, s, s, cin, n->dz[l - 1], st);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaGetLastError();
}

}  // namespace

extern "C" {

long long sp_unet_n_params(void) { return param_offsets().total; }

int sp_unet_layer(int layer, int *cout, int *cin, long long *w_offset, long long *b_offset)
{
    if (layer < 0 || layer > SP_UNET_LAYERS) return SP_ERR_ARG;
    Offsets o = param_offsets();
    if (layer == SP_UNET_LAYERS) {
        if (cout) *cout = 3;
        if (cin) *cin = 32;
    } else {
        if (cout) *cout = kLayers[layer].cout;
        if (cin) *cin = kLayers[layer].cin0 + kLayers[layer].cin1;
    }
    if (w_offset) *w_offset = o.w[layer];
    if (b_offset) *b_offset = o.b[layer];
    return SP_OK;
}

const char *sp_unet_last_error(const sp_unet *net) { return net ? net->err.c_str() : "NULL network"; }

void sp_unet_destroy(sp_unet *net)
{
    if (!net) return;
    if (net->arena) cudaFree(net->arena);
    delete net;
}

int sp_unet_create(sp_unet **out, int L, int batch_max)
{
    if (!out) return SP_ERR_ARG;
    *out = nullptr;
    if (L < 8 || L % 8 || L > 4096 || batch_max < 1) return SP_ERR_ARG;
    sp_unet *n = new sp_unet;
    n->L = L;
    n->bmax = batch_max;
    n->off = param_offsets();
    n->tab.n = SP_UNET_LAYERS;
    long long kb = 0;
    for (int l = 0; l < SP_UNET_LAYERS; ++l) {
        n->tab.cout[l] = kLayers[l].cout;
        n->tab.cin[l] = kLayers[l].cin0 + kLayers[l].cin1;
        n->tab.w_off[l] = n->off.w[l];
        n->tab.bf_off[l] = kb;
        kb += (long long)n->tab.cout[l] * 9 * n->tab.cin[l];
    }
    n->n_bf = kb;
    // workspace: largest wgrad plan over the layers at batch_max
    long long ws = 0;
    for (int l = 0; l < SP_UNET_LAYERS; ++l) {
        long long P = level_pixels(n, batch_max, kLayers[l].level);
        long long b = wgrad_ws_bytes(P, n->tab.cin[l], kLayers[l].cout) / (long long)sizeof(float);
        if (b > ws) ws = b;
    }
    n->ws_floats = ws;
    long long P0 = level_pixels(n, batch_max, 0);
    n->head_blocks = (int)((P0 + 255) / 256);
    // carve one allocation, 256-byte aligned pieces
    std::vector<std::pair<void **, size_t>> pieces;
    auto add = [&](void **p, size_t bytes) { pieces.push_back({p, bytes}); };
    size_t np = (size_t)n->off.total;
    add((void **)&n->params, np * 4);
    add((void **)&n->grad, np * 4);
    add((void **)&n->m, np * 4);
    add((void **)&n->v, np * 4);
    add((void **)&n->wk, (size_t)kb * 2);
    add((void **)&n->wt, (size_t)kb * 2);
    add((void **)&n->x, (size_t)P0 * SP_UNET_IN_CH * 2);
    for (int l = 0; l < SP_UNET_LAYERS; ++l) {
        size_t b = (size_t)level_pixels(n, batch_max, kLayers[l].level) * kLayers[l].cout * 2;
        add((void **)&n->act[l], b);
        add((void **)&n->dz[l], b);
    }
    for (int k = 0; k < 3; ++k) {
        int C = kLayers[2 * k + 1].cout;
        size_t b = (size_t)level_pixels(n, batch_max, k + 1) * C * 2;
        add((void **)&n->pool[k], b);
        add((void **)&n->dpool[k], b);
        int dec = 12 - 2 * k;
        add((void **)&n->dcat[k], (size_t)level_pixels(n, batch_max, k) * (kLayers[dec].cin0 + kLayers[dec].cin1) * 2);
    }
    add((void **)&n->ws, (size_t)ws * 4);
    add((void **)&n->head_part, (size_t)n->head_blocks * kHeadVals * 4);
    size_t total = 0;
    for (auto &pc : pieces) total += (pc.second + 255) / 256 * 256;
    cudaError_t e = cudaMalloc(&n->arena, total);
    if (e != cudaSuccess) {
        delete n;
        return SP_ERR_CUDA;
    }
    size_t o = 0;
    for (auto &pc : pieces) {
        *pc.first = (char *)n->arena + o;
        o += (pc.second + 255) / 256 * 256;
    }
    e = cudaMemset(n->arena, 0, total);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        sp_unet_destroy(n);
        return SP_ERR_CUDA;
    }
    *out = n;
    return SP_OK;
}

int sp_unet_set_params(sp_unet *net, const float *host, long long n)
{
    if (!net) return SP_ERR_ARG;
    if (!host || n != net->off.total) return ufail(net, SP_ERR_ARG, "expected %lld parameters", net->off.total);
    size_t b = (size_t)n * 4;
    cudaError_t e = cudaMemcpy(net->params, host, b, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(net->m, 0, b);
    if (e == cudaSuccess) e = cudaMemset(net->v, 0, b);
    if (e != cudaSuccess) return cfail(net, e, "set_params");
    k_prep_weights<<<grid_for(net->n_bf), 256>>>(net->tab, net->params, net->wk, net->wt);
    e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? SP_OK : cfail(net, e, "prepare weights");
}

int sp_unet_get_params(sp_unet *net, float *host, long long n)
{
    if (!net) return SP_ERR_ARG;
    if (!host || n != net->off.total) return ufail(net, SP_ERR_ARG, "expected %lld parameters", net->off.total);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(host, net->params, (size_t)n * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? SP_OK : cfail(net, e, "get_params");
}

int sp_unet_predict(sp_unet *net, const float *spins_dev, const float *features_dev, int batch, float *out_dev,
                    void *stream)
{
    if (!net) return SP_ERR_ARG;
    if (!spins_dev || !features_dev || !out_dev) return ufail(net, SP_ERR_ARG, "NULL device pointer");
    int rc = check_batch(net, batch);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = forward(net, spins_dev, features_dev, batch, st);
    if (e != cudaSuccess) return cfail(net, e, "forward");
    long long P = level_pixels(net, batch, 0);
    k_head<false><<<(unsigned)((P + 255) / 256), 256, 0, st>>>(net->act[SP_UNET_LAYERS - 1], net->params + net->off.w[SP_UNET_LAYERS],
                                                               nullptr, P, 0.f, (float4 *)out_dev, nullptr, nullptr);
    e = cudaGetLastError();
    return e == cudaSuccess ? SP_OK : cfail(net, e, "head");
}

int sp_unet_loss_grad(sp_unet *net, const float *spins_dev, const float *features_dev, const float *target_dev,
                      int batch, double *loss_dev, float *grad_dev, void *stream)
{
    if (!net) return SP_ERR_ARG;
    if (!spins_dev || !features_dev || !target_dev || !loss_dev) return ufail(net, SP_ERR_ARG, "NULL device pointer");
    int rc = check_batch(net, batch);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = forward(net, spins_dev, features_dev, batch, st);
    if (e != cudaSuccess) return cfail(net, e, "forward");
    long long P = level_pixels(net, batch, 0);
    int nb = (int)((P + 255) / 256);
    k_head<true><<<nb, 256, 0, st>>>(net->act[SP_UNET_LAYERS - 1], net->params + net->off.w[SP_UNET_LAYERS], target_dev,
                                     P, (float)(1.0 / (double)P), nullptr, net->dz[SP_UNET_LAYERS - 1], net->head_part);
    k_head_reduce<<<kHeadVals, 256, 0, st>>>(net->head_part, nb, 1.0 / (double)P,
                                             net->grad + net->off.w[SP_UNET_LAYERS], loss_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cfail(net, e, "head");
    e = backward(net, batch, st);
    if (e != cudaSuccess) return cfail(net, e, "backward");
    if (grad_dev) {
        e = cudaMemcpyAsync(grad_dev, net->grad, (size_t)net->off.total * 4, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cfail(net, e, "copy gradient");
    }
    return SP_OK;
}

int sp_unet_adam(sp_unet *net, double lr, double beta1, double beta2, double eps, int step, void *stream)
{
    if (!net) return SP_ERR_ARG;
    if (!(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0) || step < 1)
        return ufail(net, SP_ERR_ARG, "bad Adam parameters");
    cudaStream_t st = (cudaStream_t)stream;
    double c1 = 1.0 / (1.0 - pow(beta1, step)), c2 = 1.0 / (1.0 - pow(beta2, step));
    k_adam<<<grid_for(net->off.total), 256, 0, st>>>(net->params, net->grad, net->m, net->v, net->off.total, (float)lr,
                                                      (float)beta1, (float)beta2, (float)eps, (float)c1, (float)c2);
    k_prep_weights<<<grid_for(net->n_bf), 256, 0, st>>>(net->tab, net->params, net->wk, net->wt);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SP_OK : cfail(net, e, "adam");
}

int sp_conv3x3_forward(const uint16_t *src0, int C0, int up0, const uint16_t *src1, int C1, const uint16_t *W,
                       const float *bias, int relu, const uint16_t *mask, int B, int H, int Wd, int Cout,
                       uint16_t *out, void *stream)
{
    if (!src0 || !W || !out || (C1 && !src1)) return SP_ERR_ARG;
    if (!conv_shape_ok(C0, C1, up0, B, H, Wd, Cout)) return SP_ERR_ARG;
    ConvSrc S{(const bf16 *)src0, C0, up0 ? 1 : 0, (const bf16 *)src1, C1};
    cudaError_t e = conv_launch(S, (const bf16 *)W, bias, relu, (const bf16 *)mask, B, H, Wd, Cout, (bf16 *)out,
                                (cudaStream_t)stream);
    return e == cudaSuccess ? SP_OK : SP_ERR_CUDA;
}

int sp_conv3x3_transpose(const uint16_t *W, int Cout, int Cin, uint16_t *Wt, void *stream)
{
    if (!W || !Wt || Cout < 1 || Cin < 1) return SP_ERR_ARG;
    k_transpose<<<grid_for((long long)Cout * 9 * Cin), 256, 0, (cudaStream_t)stream>>>((const bf16 *)W, Cout, Cin,
                                                                                        (bf16 *)Wt);
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ERR_CUDA;
}

int sp_conv3x3_set_kernel(int tcgen05)
{
    if (tcgen05 < 0 || tcgen05 > 3) return SP_ERR_ARG;
    g_use_tc = tcgen05;
    return SP_OK;
}

int sp_conv3x3_get_kernel(void) { return g_use_tc; }

int sp_conv3x3_set_wait_limit(long long cycles)
{
    if (cycles < 0) return SP_ERR_ARG;
    if (cudaMemcpyToSymbol(g_tc_wait_limit, &cycles, sizeof cycles) != cudaSuccess) return SP_ERR_CUDA;
    return SP_OK;
}

int sp_unet_device_error(void)
{
    int v = 0, zero = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return SP_ERR_CUDA;
    if (cudaMemcpyFromSymbol(&v, g_tc_error, sizeof v) != cudaSuccess) return SP_ERR_CUDA;
    if (v && cudaMemcpyToSymbol(g_tc_error, &zero, sizeof zero) != cudaSuccess) return SP_ERR_CUDA;
    return v ? SP_ERR_TIMEOUT : SP_OK;
}

long long sp_conv3x3_wgrad_workspace(int B, int H, int Wd, int Cin, int Cout)
{
    if (B < 1 || H < 1 || Wd < 1 || Cin < 32 || Cout < 32) return -1;
    return wgrad_ws_bytes((long long)B * H * Wd, Cin, Cout);
}

int sp_conv3x3_wgrad(const uint16_t *src0, int C0, int up0, const uint16_t *src1, int C1, const uint16_t *dz, int B,
                     int H, int Wd, int Cout, float *dW, float *db, void *workspace, long long workspace_bytes,
                     void *stream)
{
    if (!src0 || !dz || !dW || !workspace || (C1 && !src1)) return SP_ERR_ARG;
    if (!conv_shape_ok(C0, C1, up0, B, H, Wd, Cout)) return SP_ERR_ARG;
    if (workspace_bytes < wgrad_ws_bytes((long long)B * H * Wd, C0 + C1, Cout)) return SP_ERR_ARG;
    ConvSrc S{(const bf16 *)src0, C0, up0 ? 1 : 0, (const bf16 *)src1, C1};
    cudaError_t e = wgrad_launch(S, (const bf16 *)dz, B, H, Wd, Cout, dW, db, (float *)workspace, (cudaStream_t)stream);
    return e == cudaSuccess ? SP_OK : SP_ERR_CUDA;
}

}  // extern "C"
