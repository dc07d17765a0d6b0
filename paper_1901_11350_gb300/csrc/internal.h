// internal.h -- launchers shared between the library's translation units.
#pragma once

#include "common.cuh"

namespace spgb {

// Per-run LLG constants, per basis atom where they depend on mu_b.
template <typename T> struct LlgConst {
    T dt, alpha;
    T cA[SP_MAX_BASIS];   // -gamma / ((1 + alpha^2) mu_b)
    T sig[SP_MAX_BASIS];  // sqrt(2 alpha kB T mu_b / (gamma dt)), meV
    uint64_t seed, step;
    uint32_t replica;
    int thermal;
    // Philox round keys (k0 + r W0, k1 + r W1), r = 0..9, of `seed`: the
    // kernels read them as operands instead of stepping the key per spin
    uint32_t rk[20];
    // a batch of replicas: n_rep > 1 copies of the lattice stored one after
    // another; replica r has the noise amplitudes rsig[r * nb + b] (device)
    // and the thermal stream replica + r.  n_rep 0 or 1 with rsig null: one
    // lattice with the amplitudes sig[]
    int n_rep, nb;
    const T *rsig;
    // step_base non-null (a batch of replicas replayed from a CUDA graph):
    // the Philox step is *step_base + step, the base a device counter the
    // graph advances
    const unsigned long long *step_base;
};

template <typename T> __host__ __device__ inline int llg_reps(const LlgConst<T> &c) { return c.n_rep > 1 ? c.n_rep : 1; }
template <typename T> __device__ __forceinline__ T noise_amp(const LlgConst<T> &c, int r, int b)
{
    return c.rsig ? c.rsig[r * c.nb + b] : c.sig[b];
}

template <typename T> inline void llg_set_seed(LlgConst<T> &k, uint64_t seed)
{
    k.seed = seed;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (uint32_t r = 0; r < 10; ++r) {
        k.rk[2 * r] = k0 + r * 0x9E3779B9u;  // mod 2^32, as r successive Weyl steps
        k.rk[2 * r + 1] = k1 + r * 0xBB67AE85u;
    }
}

template <typename T> __device__ __forceinline__ uint64_t llg_step_of(const LlgConst<T> &c)
{
    return c.step_base ? *c.step_base + c.step : c.step;
}

// The thermal-field counter block of spin i of replica c.replica + r at
// `step` (the layout of thermal_bits), through the precomputed round keys.
template <typename T>
__device__ __forceinline__ uint4 thermal_bits_at(const LlgConst<T> &c, uint64_t step, uint32_t i, uint32_t r)
{
    return philox4x32_10_keyed(make_uint4(i, (uint32_t)step, (uint32_t)(step >> 32), (c.replica + r) * 8u), c.rk);
}
template <typename T> __device__ __forceinline__ uint4 thermal_bits(const LlgConst<T> &c, uint32_t i, uint32_t r = 0)
{
    return thermal_bits_at(c, llg_step_of(c), i, r);
}

// One system of a batch of different lattices stepped together
// (sp_llg_step_batch): its first record, size, thermal stream and per-basis
// LLG prefactors and noise amplitudes (computed on the host in FP64, as for a
// single call).
template <typename T> struct LlgSys {
    long long spin0;
    int N;
    uint32_t replica;
    T cA[SP_MAX_BASIS], sig[SP_MAX_BASIS];
};

constexpr int kBlock = 256;
// single-CTA LLG path for small FP32 lattices: threads of the CTA, largest
// lattice (3 records of 16 B per spin in shared memory: 96 KB)
constexpr int kSmallThreads = 512;
constexpr int kSmallMax = 2048;
inline int blocks_for(long n, int bs = kBlock) { return (int)((n + bs - 1) / bs); }
// Threads per block of the per-spin LLG kernels: 256, or fewer for lattices
// too small to give every SM of the device a block of 256 (at least 32), so
// that the work spreads over the SMs -- it matters for FP64, whose rate per
// SM is low.
inline int llg_block(long n)
{
    const long sms = 152;
    if (n >= sms * kBlock) return kBlock;
    long per = (n + sms - 1) / sms;
    int bs = (int)((per + 31) / 32 * 32);
    return bs < 32 ? 32 : bs;
}

template <typename T>
cudaError_t launch_field(const Stencil<T> &S, const rec_t<T> *n, const rec_t<T> *Bdd, rec_t<T> *out, T sign,
                         cudaStream_t st);
cudaError_t launch_llg_small(int solver, const Stencil<float> &S, float4 *n, const LlgConst<float> &c, int n_steps,
                             cudaStream_t st);
template <typename T>
cudaError_t launch_llg_pred(int solver, const Stencil<T> &S, const rec_t<T> *n, const rec_t<T> *Bdd, rec_t<T> *np,
                            rec_t<T> *q, const LlgConst<T> &c, cudaStream_t st);
template <typename T>
cudaError_t launch_llg_corr(int solver, const Stencil<T> &S, rec_t<T> *n, const rec_t<T> *np, const rec_t<T> *q,
                            const rec_t<T> *Bdd, const LlgConst<T> &c, cudaStream_t st);
// RK4 stage 0..3 (stage 0 reads src = n; stage 3 writes n).
template <typename T>
cudaError_t launch_rk4_stage(int stage, const Stencil<T> &S, rec_t<T> *n, const rec_t<T> *src, rec_t<T> *dst,
                             rec_t<T> *acc, const rec_t<T> *Bdd, const LlgConst<T> &c, cudaStream_t st);
// Energies (6 FP64 sums) and max torque of the spins n; partials needs
// 8 * blocks_for(N) doubles.  e_out (6) and torque_out (1) may be null.
template <typename T>
cudaError_t launch_energy(const Stencil<T> &S, const rec_t<T> *n, const rec_t<T> *Bdd, double *partials, double *e_out,
                          double *torque_out, cudaStream_t st);

// Covariant Hessian-vector product out = H v at the configuration n (v is
// projected onto the tangent planes first).
template <typename T>
cudaError_t launch_hvp(const Stencil<T> &S, const rec_t<T> *n, const rec_t<T> *v, rec_t<T> *out, cudaStream_t st);

// One pass (0 predictor, 1 corrector) of a batch of systems: blk[b] = (system,
// block of kBlock spins in it), Sv[k] and sys[k] per system, the records of
// system k at sys[k].spin0 in n, np and q; c holds what all share (dt,
// alpha, seed, step, thermal flag).
template <typename T>
cudaError_t launch_llg_batch(int pass, int solver, int n_blk, const int2 *blk, const Stencil<T> *Sv,
                             const LlgSys<T> *sys, rec_t<T> *n, rec_t<T> *np, rec_t<T> *q, const LlgConst<T> &c,
                             cudaStream_t st);

// Finiteness check of results (the device status word): records n[0..n_rec)
// (x, y, z; the padding lane is not looked at) or plain doubles v[0..n_val);
// any non-finite value ORs `site` into *flag, a word of mapped host memory.
template <typename T>
cudaError_t launch_check_records(const rec_t<T> *n, long n_rec, unsigned *flag, unsigned site, cudaStream_t st);
cudaError_t launch_check_doubles(const double *v, long n_val, unsigned *flag, unsigned site, cudaStream_t st);

// Topological charge of a 2D one-atom lattice; flip swaps the triangle
// orientation (for left-handed in-plane lattice vectors); partials needs
// blocks_for(n0 * n1) doubles.
template <typename T>
cudaError_t launch_topo(const Stencil<T> &S, const rec_t<T> *n, int flip, double *partials, double *Q, cudaStream_t st);

}  // namespace spgb
