// field_llg.cu -- effective field, energy/torque reductions and the two-pass
// LLG step (Depondt, Heun, SIB, RK4) for any lattice with a neighbour stencil.
//
// Heun (Appendix B) with the thermal field of Eq. 4, one step in two passes:
//   pass 1 (predictor), per spin i:
//       A_i  = A(n_i, B_i(n) + Bth_i),  f_i = n_i x A_i
//       np_i = normalise(n_i + dt f_i)
//       q_i  = n_i + dt/2 (f_i + np_i x A(np_i, Bth_i))
//   pass 2 (corrector):
//       n_i <- normalise(q_i + dt/2 np_i x A(np_i, B_i(np)))
// A(n, B) is linear in B, so f(np) = np x A(np, B(np)) + np x A(np, Bth):
// the noise-dependent half of the corrector is folded into q in pass 1 and
// neither the noise nor A(n) is recomputed in pass 2.  Depondt folds the same
// way: h_i = A_i/2 + A(np_i, Bth_i)/2 and n_i <- R(h_i + A(np_i, B_i(np))/2) n_i.
// Memory per step: read n, write np and q; read np (stencil) and q (and n
// for Depondt), write n -- 6 (7) records per spin.
#include <algorithm>

#include "internal.h"

// 1: the per-spin LLG passes are launched with programmatic dependent launch
#ifndef SPGB_LLG_PDL
#define SPGB_LLG_PDL 1
#endif

namespace spgb {

// ---------------------------------------------------------------- field
template <typename T>
__global__ void __launch_bounds__(kBlock) k_field(const __grid_constant__ Stencil<T> S, const rec_t<T> *__restrict__ n,
                                                  const rec_t<T> *__restrict__ Bdd, rec_t<T> *__restrict__ out, T sign)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.N) return;
    int b;
    v3<T> ni = ld(n, i);
    v3<T> B = local_field(S, n, i, ni, b);
    if (Bdd) B = B + ld(Bdd, i);
    st(out, i, sign * B);
}

template <typename T>
cudaError_t launch_field(const Stencil<T> &S, const rec_t<T> *n, const rec_t<T> *Bdd, rec_t<T> *out, T sign,
                         cudaStream_t st)
{
    if (S.N == 0) return cudaSuccess;
    k_field<T><<<blocks_for(S.N), kBlock, 0, st>>>(S, n, Bdd, out, sign);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- LLG
// Per-spin bodies of the two passes, shared by the grid kernels (records in
// global memory) and the single-CTA kernel (records in shared memory).
// (r: the replica within a batch, whose noise amplitudes and thermal stream
// the predictor uses; the caller offsets the record pointers.)
template <typename T, int SOLVER, typename R>
__device__ __forceinline__ void pred_spin(const Stencil<T> &S, const R *n, const rec_t<T> *Bdd, R *np, R *q,
                                          const LlgConst<T> &c, int i, int r = 0)
{
    int b;
    v3<T> ni = ld(n, i);
    v3<T> B = local_field(S, n, i, ni, b);
    if (Bdd) B = B + ld(Bdd, i);
    v3<T> Bth = mk(T(0), T(0), T(0));
    if (c.thermal) Bth = noise_amp(c, r, b) * box_muller(thermal_bits(c, (uint32_t)i, (uint32_t)r), T(0));
    v3<T> A = llg_A(c.cA[b], c.alpha, ni, B + Bth);
    if (SOLVER == SP_HEUN) {
        v3<T> f = cross(ni, A);
        v3<T> p = normalised(axpy(c.dt, f, ni));
        v3<T> g = cross(p, llg_A(c.cA[b], c.alpha, p, Bth));
        st(np, i, p);
        st(q, i, axpy(T(0.5) * c.dt, f + g, ni));
    } else if (SOLVER == SP_SIB) {
        // np holds the midpoint (n + x_p)/2, q the thermal part of A there
        v3<T> m = T(0.5) * (ni + sib_solve(ni, A, c.dt));
        st(np, i, m);
        st(q, i, llg_A(c.cA[b], c.alpha, m, Bth));
    } else {
        v3<T> p = rotate(ni, A, c.dt);
        st(np, i, p);
        st(q, i, T(0.5) * (A + llg_A(c.cA[b], c.alpha, p, Bth)));
    }
}

template <typename T, int SOLVER, typename R>
__device__ __forceinline__ void corr_spin(const Stencil<T> &S, R *n, const R *np, const R *q, const rec_t<T> *Bdd,
                                          const LlgConst<T> &c, int i)
{
    int b;
    v3<T> p = ld(np, i);
    v3<T> B = local_field(S, np, i, p, b);
    if (Bdd) B = B + ld(Bdd, i);
    v3<T> Ap = llg_A(c.cA[b], c.alpha, p, B);
    v3<T> qi = ld(q, i);
    if (SOLVER == SP_HEUN) {
        st(n, i, normalised(axpy(T(0.5) * c.dt, cross(p, Ap), qi)));
    } else if (SOLVER == SP_SIB) {
        st(n, i, sib_solve(ldc(n, i), Ap + qi, c.dt));
    } else {
        v3<T> Ac = axpy(T(0.5), Ap, qi);
        st(n, i, rotate(ldc(n, i), Ac, c.dt));
    }
}

template <typename T, int SOLVER>
__global__ void __launch_bounds__(kBlock) k_llg_pred(const __grid_constant__ Stencil<T> S, const rec_t<T> *__restrict__ n,
                                                     const rec_t<T> *__restrict__ Bdd, rec_t<T> *__restrict__ np,
                                                     rec_t<T> *__restrict__ q, const LlgConst<T> c)
{
    allow_dependents();
    wait_prerequisite();  // n (and Bdd) come from the kernels before
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.N) return;
    int r = blockIdx.y;  // replica
    size_t o = (size_t)r * S.N;
    pred_spin<T, SOLVER>(S, n + o, Bdd, np + o, q + o, c, i, r);
}

template <typename T, int SOLVER>
__global__ void __launch_bounds__(kBlock) k_llg_corr(const __grid_constant__ Stencil<T> S, rec_t<T> *__restrict__ n,
                                                     const rec_t<T> *__restrict__ np, const rec_t<T> *__restrict__ q,
                                                     const rec_t<T> *__restrict__ Bdd, const LlgConst<T> c)
{
    allow_dependents();
    wait_prerequisite();  // np, q (and Bdd) come from the kernels before
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.N) return;
    size_t o = (size_t)blockIdx.y * S.N;  // replica
    corr_spin<T, SOLVER>(S, n + o, np + o, q + o, Bdd, c, i);
}

// A batch of different lattices: each block belongs to one system, whose
// constants (prefactors, noise amplitudes, thermal stream) the block takes
// into a shared-memory copy of the common constants; then the per-spin
// bodies of the single-lattice kernels run unchanged, so every system gets
// the result a call on it alone gives.
template <typename T>
__device__ __forceinline__ const LlgConst<T> &batch_const(const LlgConst<T> &c, const LlgSys<T> &s)
{
    __shared__ LlgConst<T> cs;
    if (threadIdx.x == 0) {
        cs = c;
        for (int b = 0; b < SP_MAX_BASIS; ++b) {
            cs.cA[b] = s.cA[b];
            cs.sig[b] = s.sig[b];
        }
        cs.replica = s.replica;
        cs.rsig = nullptr;
        cs.n_rep = 0;
    }
    __syncthreads();
    return cs;
}

template <typename T, int SOLVER>
__global__ void __launch_bounds__(kBlock) k_llg_bpred(const int2 *__restrict__ blk, const Stencil<T> *__restrict__ Sv,
                                                      const LlgSys<T> *__restrict__ sys, const rec_t<T> *__restrict__ n,
                                                      rec_t<T> *__restrict__ np, rec_t<T> *__restrict__ q,
                                                      const LlgConst<T> c)
{
    allow_dependents();
    wait_prerequisite();  // n comes from the kernels before
    const int2 bt = blk[blockIdx.x];
    const LlgConst<T> &cs = batch_const(c, sys[bt.x]);
    const Stencil<T> &S = Sv[bt.x];
    int i = bt.y * kBlock + threadIdx.x;
    if (i >= S.N) return;
    size_t o = (size_t)sys[bt.x].spin0;
    pred_spin<T, SOLVER>(S, n + o, (const rec_t<T> *)nullptr, np + o, q + o, cs, i, 0);
}

template <typename T, int SOLVER>
__global__ void __launch_bounds__(kBlock) k_llg_bcorr(const int2 *__restrict__ blk, const Stencil<T> *__restrict__ Sv,
                                                      const LlgSys<T> *__restrict__ sys, rec_t<T> *__restrict__ n,
                                                      const rec_t<T> *__restrict__ np, const rec_t<T> *__restrict__ q,
                                                      const LlgConst<T> c)
{
    allow_dependents();
    wait_prerequisite();  // np, q come from the kernels before
    const int2 bt = blk[blockIdx.x];
    const LlgConst<T> &cs = batch_const(c, sys[bt.x]);
    const Stencil<T> &S = Sv[bt.x];
    int i = bt.y * kBlock + threadIdx.x;
    if (i >= S.N) return;
    size_t o = (size_t)sys[bt.x].spin0;
    corr_spin<T, SOLVER>(S, n + o, np + o, q + o, (const rec_t<T> *)nullptr, cs, i);
}

template <typename T>
cudaError_t launch_llg_batch(int pass, int solver, int n_blk, const int2 *blk, const Stencil<T> *Sv,
                             const LlgSys<T> *sys, rec_t<T> *n, rec_t<T> *np, rec_t<T> *q, const LlgConst<T> &c,
                             cudaStream_t st)
{
    if (n_blk <= 0) return cudaSuccess;
    dim3 g(n_blk), b(kBlock);
    if (pass == 0) {
        if (solver == SP_HEUN) return launch_pdl(k_llg_bpred<T, SP_HEUN>, g, b, 0, st, blk, Sv, sys, (const rec_t<T> *)n, np, q, c);
        if (solver == SP_SIB) return launch_pdl(k_llg_bpred<T, SP_SIB>, g, b, 0, st, blk, Sv, sys, (const rec_t<T> *)n, np, q, c);
        return launch_pdl(k_llg_bpred<T, SP_DEPONDT>, g, b, 0, st, blk, Sv, sys, (const rec_t<T> *)n, np, q, c);
    }
    if (solver == SP_HEUN)
        return launch_pdl(k_llg_bcorr<T, SP_HEUN>, g, b, 0, st, blk, Sv, sys, n, (const rec_t<T> *)np, (const rec_t<T> *)q, c);
    if (solver == SP_SIB)
        return launch_pdl(k_llg_bcorr<T, SP_SIB>, g, b, 0, st, blk, Sv, sys, n, (const rec_t<T> *)np, (const rec_t<T> *)q, c);
    return launch_pdl(k_llg_bcorr<T, SP_DEPONDT>, g, b, 0, st, blk, Sv, sys, n, (const rec_t<T> *)np, (const rec_t<T> *)q, c);
}

// Small FP32 lattices (N <= kSmallMax): one CTA keeps n, np and q in shared
// memory and runs every step in the kernel, a CTA barrier between the passes
// -- the same per-spin arithmetic as the two grid kernels, without 2 launches
// per step.  (FP64 is not sent here: its rate per SM is low, and spreading
// the spins over the SMs with small blocks is faster.)
template <typename T, int SOLVER>
__global__ void __launch_bounds__(kSmallThreads) k_llg_small(const __grid_constant__ Stencil<T> S,
                                                             rec_t<T> *__restrict__ ng, LlgConst<T> c, int n_steps)
{
    typedef typename ShRec<T>::type R;
    extern __shared__ __align__(16) unsigned char smem_small[];
    R *n = reinterpret_cast<R *>(smem_small);
    R *np = n + S.N, *q = np + S.N;
    for (int i = threadIdx.x; i < S.N; i += blockDim.x) st(n, i, ldc(ng, i));
    __syncthreads();
    const uint64_t step0 = c.step;
    for (int s = 0; s < n_steps; ++s) {
        c.step = step0 + (uint64_t)s;
        for (int i = threadIdx.x; i < S.N; i += blockDim.x) pred_spin<T, SOLVER>(S, (const R *)n, nullptr, np, q, c, i);
        __syncthreads();
        for (int i = threadIdx.x; i < S.N; i += blockDim.x)
            corr_spin<T, SOLVER>(S, n, (const R *)np, (const R *)q, nullptr, c, i);
        __syncthreads();
    }
    for (int i = threadIdx.x; i < S.N; i += blockDim.x) st(ng, i, ld(n, i));
}

cudaError_t launch_llg_small(int solver, const Stencil<float> &S, float4 *n, const LlgConst<float> &c, int n_steps,
                             cudaStream_t st)
{
    typedef float T;
    if (S.N == 0 || n_steps == 0) return cudaSuccess;
    size_t sm = 3 * sizeof(typename ShRec<T>::type) * (size_t)S.N;
    static bool attr[3] = {false, false, false};
    int slot = solver == SP_HEUN ? 0 : (solver == SP_SIB ? 1 : 2);
    const void *fn = solver == SP_HEUN ? (const void *)k_llg_small<T, SP_HEUN>
                                       : (solver == SP_SIB ? (const void *)k_llg_small<T, SP_SIB>
                                                           : (const void *)k_llg_small<T, SP_DEPONDT>);
    if (!attr[slot]) {
        int max_sm = (int)(3 * sizeof(typename ShRec<T>::type) * kSmallMax);
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_sm);
        if (e != cudaSuccess) return e;
        attr[slot] = true;
    }
    if (solver == SP_HEUN)
        k_llg_small<T, SP_HEUN><<<1, kSmallThreads, sm, st>>>(S, n, c, n_steps);
    else if (solver == SP_SIB)
        k_llg_small<T, SP_SIB><<<1, kSmallThreads, sm, st>>>(S, n, c, n_steps);
    else
        k_llg_small<T, SP_DEPONDT><<<1, kSmallThreads, sm, st>>>(S, n, c, n_steps);
    return cudaGetLastError();
}

template <typename... KArgs, typename... Args>
cudaError_t launch_llg_kernel(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args)
{
#if SPGB_LLG_PDL
    return launch_pdl(kern, grid, block, smem, st, args...);
#else
    kern<<<grid, block, smem, st>>>(args...);
    return cudaGetLastError();
#endif
}

template <typename T>
cudaError_t launch_llg_pred(int solver, const Stencil<T> &S, const rec_t<T> *n, const rec_t<T> *Bdd, rec_t<T> *np,
                            rec_t<T> *q, const LlgConst<T> &c, cudaStream_t st)
{
    if (S.N == 0) return cudaSuccess;
    int bs = llg_block((long)S.N * llg_reps(c));
    cudaError_t e;
    if (solver == SP_HEUN)
        e = launch_llg_kernel(k_llg_pred<T, SP_HEUN>, dim3(blocks_for(S.N, bs), llg_reps(c)), dim3(bs), 0, st, S, n, Bdd, np, q, c);
    else if (solver == SP_SIB)
        e = launch_llg_kernel(k_llg_pred<T, SP_SIB>, dim3(blocks_for(S.N, bs), llg_reps(c)), dim3(bs), 0, st, S, n, Bdd, np, q, c);
    else
        e = launch_llg_kernel(k_llg_pred<T, SP_DEPONDT>, dim3(blocks_for(S.N, bs), llg_reps(c)), dim3(bs), 0, st, S, n, Bdd, np, q, c);
    return e;
}

template <typename T>
cudaError_t launch_llg_corr(int solver, const Stencil<T> &S, rec_t<T> *n, const rec_t<T> *np, const rec_t<T> *q,
                            const rec_t<T> *Bdd, const LlgConst<T> &c, cudaStream_t st)
{
    if (S.N == 0) return cudaSuccess;
    int bs = llg_block((long)S.N * llg_reps(c));
    cudaError_t e;
    if (solver == SP_HEUN)
        e = launch_llg_kernel(k_llg_corr<T, SP_HEUN>, dim3(blocks_for(S.N, bs), llg_reps(c)), dim3(bs), 0, st, S, n, np, q, Bdd, c);
    else if (solver == SP_SIB)
        e = launch_llg_kernel(k_llg_corr<T, SP_SIB>, dim3(blocks_for(S.N, bs), llg_reps(c)), dim3(bs), 0, st, S, n, np, q, Bdd, c);
    else
        e = launch_llg_kernel(k_llg_corr<T, SP_DEPONDT>, dim3(blocks_for(S.N, bs), llg_reps(c)), dim3(bs), 0, st, S, n, np, q, Bdd, c);
    return e;
}

// ---------------------------------------------------------------- RK4
// Stage s of the fourth-order Runge-Kutta step on y' = y x A(y, B(y) + B_th),
// the same thermal field in every stage: k = y x A at the stage state y (src),
// acc accumulates k1 + 2 k2 + 2 k3, the next stage state n + c dt k goes to
// dst; stage 3 writes normalise(n + dt/6 (acc + k4)) to n.
template <typename T, int STAGE>
__global__ void __launch_bounds__(kBlock) k_rk4(const __grid_constant__ Stencil<T> S, rec_t<T> *__restrict__ n,
                                                const rec_t<T> *__restrict__ src, rec_t<T> *__restrict__ dst,
                                                rec_t<T> *__restrict__ acc, const rec_t<T> *__restrict__ Bdd,
                                                const LlgConst<T> c)
{
    allow_dependents();
    wait_prerequisite();  // the stage inputs come from the kernels before
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.N) return;
    int r = blockIdx.y;  // replica
    size_t o = (size_t)r * S.N;
    n += o;
    src += o;
    dst += o;
    acc += o;
    int b;
    v3<T> y = ld(src, i);
    v3<T> B = local_field(S, src, i, y, b);
    if (Bdd) B = B + ld(Bdd, i);
    if (c.thermal) B = B + noise_amp(c, r, b) * box_muller(thermal_bits(c, (uint32_t)i, (uint32_t)r), T(0));
    v3<T> k = cross(y, llg_A(c.cA[b], c.alpha, y, B));
    v3<T> ni = ldc(n, i);
    if (STAGE == 0) {
        st(acc, i, k);
        st(dst, i, axpy(T(0.5) * c.dt, k, ni));
    } else if (STAGE < 3) {
        st(acc, i, axpy(T(2), k, ldc(acc, i)));
        st(dst, i, axpy((STAGE == 1 ? T(0.5) : T(1)) * c.dt, k, ni));
    } else {
        st(n, i, normalised(axpy(c.dt / T(6), ldc(acc, i) + k, ni)));
    }
}

template <typename T>
cudaError_t launch_rk4_stage(int stage, const Stencil<T> &S, rec_t<T> *n, const rec_t<T> *src, rec_t<T> *dst,
                             rec_t<T> *acc, const rec_t<T> *Bdd, const LlgConst<T> &c, cudaStream_t st)
{
    if (S.N == 0) return cudaSuccess;
    dim3 g(blocks_for(S.N), llg_reps(c));
    switch (stage) {
    case 0: return launch_llg_kernel(k_rk4<T, 0>, g, dim3(kBlock), 0, st, S, n, src, dst, acc, Bdd, c);
    case 1: return launch_llg_kernel(k_rk4<T, 1>, g, dim3(kBlock), 0, st, S, n, src, dst, acc, Bdd, c);
    case 2: return launch_llg_kernel(k_rk4<T, 2>, g, dim3(kBlock), 0, st, S, n, src, dst, acc, Bdd, c);
    default: return launch_llg_kernel(k_rk4<T, 3>, g, dim3(kBlock), 0, st, S, n, src, dst, acc, Bdd, c);
    }
}

// ---------------------------------------------------------------- energy
// Per-spin energy terms of Eq. 1 (each unique pair contributes half from
// either side) and |n_i x B_i|; FP64 block sums -> partials[8*block].
template <typename T>
__global__ void __launch_bounds__(kBlock) k_energy(const __grid_constant__ Stencil<T> S, const rec_t<T> *__restrict__ n,
                                                   const rec_t<T> *__restrict__ Bdd, double *__restrict__ partials)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    double tmax = 0;
    if (i < S.N) {
        int b, c0, c1, c2;
        decode_site(S, i, b, c0, c1, c2);
        const bool inner = interior_site(S, c0, c1, c2);
        v3<T> ni = ld(n, i);
        v3<T> Bz = mk(S.Bz[b][0], S.Bz[b][1], S.Bz[b][2]);
        v3<T> Kh = mk(S.Kh[b][0], S.Kh[b][1], S.Kh[b][2]);
        T kn = dot(Kh, ni);
        acc[1] = -ddot(ni, Bz);
        acc[2] = -(double)S.K[b] * (double)kn * (double)kn;
        v3<T> B = axpy(T(2) * S.K[b] * kn, Kh, Bz);
        v3<T> Bx = mk(T(0), T(0), T(0)), Bd = mk(T(0), T(0), T(0));
        for (int q = S.off[b]; q < S.off[b + 1]; ++q) {
            const NbrEntry<T> &E = S.e[q];
            int j = nbr_index(S, E, i, inner, c0, c1, c2);
            if (j < 0) continue;
            v3<T> nj = ld(n, j);
            Bx = axpy(E.J, nj, Bx);
            Bd = Bd + cross(nj, mk(E.Dx, E.Dy, E.Dz));
        }
        acc[3] = -0.5 * ddot(ni, Bx);
        acc[4] = -0.5 * ddot(ni, Bd);
        B = B + Bx + Bd;
        if (Bdd) {
            v3<T> bd = ld(Bdd, i);
            acc[5] = -0.5 * ddot(ni, bd);
            B = B + bd;
        }
        acc[0] = acc[1] + acc[2] + acc[3] + acc[4] + acc[5];
        v3<T> t = cross(ni, B);
        tmax = sqrt((double)dot(t, t));
    }
    // warp then block reduction in a fixed order
    __shared__ double sh[kBlock / 32][7];
    for (int k = 0; k < 6; ++k)
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
    for (int o = 16; o > 0; o >>= 1) tmax = nan_max(tmax, __shfl_down_sync(0xffffffffu, tmax, o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        for (int k = 0; k < 6; ++k) sh[w][k] = acc[k];
        sh[w][6] = tmax;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        int k = threadIdx.x;
        double v = sh[0][k];
        for (int ww = 1; ww < kBlock / 32; ++ww) v = (k == 6) ? nan_max(v, sh[ww][k]) : v + sh[ww][k];
        partials[8 * blockIdx.x + k] = v;
    }
}

// Sum the per-block partials in a fixed order (one block).
__global__ void __launch_bounds__(kBlock) k_energy_final(const double *__restrict__ partials, int nblk, double *e_out,
                                                         double *torque_out)
{
    __shared__ double sh[kBlock][7];
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int p = threadIdx.x; p < nblk; p += kBlock) {
        for (int k = 0; k < 6; ++k) acc[k] += partials[8 * p + k];
        acc[6] = nan_max(acc[6], partials[8 * p + 6]);
    }
    for (int k = 0; k < 7; ++k) sh[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int s = kBlock / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 7; ++k)
                sh[threadIdx.x][k] = (k == 6) ? nan_max(sh[threadIdx.x][k], sh[threadIdx.x + s][k])
                                              : sh[threadIdx.x][k] + sh[threadIdx.x + s][k];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (e_out)
            for (int k = 0; k < 6; ++k) e_out[k] = sh[0][k];
        if (torque_out) torque_out[0] = sh[0][6];
    }
}

template <typename T>
cudaError_t launch_energy(const Stencil<T> &S, const rec_t<T> *n, const rec_t<T> *Bdd, double *partials, double *e_out,
                          double *torque_out, cudaStream_t st)
{
    int nblk = blocks_for(S.N > 0 ? S.N : 1);
    k_energy<T><<<nblk, kBlock, 0, st>>>(S, n, Bdd, partials);
    k_energy_final<<<1, kBlock, 0, st>>>(partials, nblk, e_out, torque_out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- status
// One wave of blocks strides over the values; a block that saw a non-finite
// one ORs its site bit into the status word (system scope: the word lives in
// mapped host memory that the host reads between calls).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_check_records(const rec_t<T> *__restrict__ n, long n_rec,
                                                          unsigned *flag, unsigned site)
{
    int bad = 0;
    for (long i = (long)blockIdx.x * kBlock + threadIdx.x; i < n_rec; i += (long)gridDim.x * kBlock) {
        v3<T> v = ld(n, i);
        bad |= !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z));
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr_system(flag, site);
}

__global__ void __launch_bounds__(kBlock) k_check_doubles(const double *__restrict__ v, long n_val, unsigned *flag,
                                                          unsigned site)
{
    int bad = 0;
    for (long i = (long)blockIdx.x * kBlock + threadIdx.x; i < n_val; i += (long)gridDim.x * kBlock)
        bad |= !isfinite(v[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr_system(flag, site);
}

namespace {
int check_grid(long n)
{
    long b = (n + kBlock - 1) / kBlock;
    return (int)std::max(1L, std::min(b, 152L * 4));
}
}  // namespace

template <typename T>
cudaError_t launch_check_records(const rec_t<T> *n, long n_rec, unsigned *flag, unsigned site, cudaStream_t st)
{
    if (n_rec <= 0) return cudaSuccess;
    k_check_records<T><<<check_grid(n_rec), kBlock, 0, st>>>(n, n_rec, flag, site);
    return cudaGetLastError();
}

cudaError_t launch_check_doubles(const double *v, long n_val, unsigned *flag, unsigned site, cudaStream_t st)
{
    if (n_val <= 0) return cudaSuccess;
    k_check_doubles<<<check_grid(n_val), kBlock, 0, st>>>(v, n_val, flag, site);
    return cudaGetLastError();
}

#define SPGB_INST(T)                                                                                                   \
    template cudaError_t launch_field<T>(const Stencil<T> &, const rec_t<T> *, const rec_t<T> *, rec_t<T> *, T,         \
                                         cudaStream_t);                                                                \
    template cudaError_t launch_llg_pred<T>(int, const Stencil<T> &, const rec_t<T> *, const rec_t<T> *, rec_t<T> *,    \
                                            rec_t<T> *, const LlgConst<T> &, cudaStream_t);                            \
    template cudaError_t launch_llg_corr<T>(int, const Stencil<T> &, rec_t<T> *, const rec_t<T> *, const rec_t<T> *,    \
                                            const rec_t<T> *, const LlgConst<T> &, cudaStream_t);                      \
    template cudaError_t launch_rk4_stage<T>(int, const Stencil<T> &, rec_t<T> *, const rec_t<T> *, rec_t<T> *,        \
                                             rec_t<T> *, const rec_t<T> *, const LlgConst<T> &, cudaStream_t);         \
    template cudaError_t launch_energy<T>(const Stencil<T> &, const rec_t<T> *, const rec_t<T> *, double *, double *,   \
                                          double *, cudaStream_t);                                            \
    template cudaError_t launch_check_records<T>(const rec_t<T> *, long, unsigned *, unsigned, cudaStream_t);      \
    template cudaError_t launch_llg_batch<T>(int, int, int, const int2 *, const Stencil<T> *, const LlgSys<T> *,       \
                                             rec_t<T> *, rec_t<T> *, rec_t<T> *, const LlgConst<T> &, cudaStream_t);
SPGB_INST(float)
SPGB_INST(double)

}  // namespace spgb
