// static_step.cu -- sp_llg_step_static: LLG stepping that allocates no device
// memory.  Its predictor state and folded corrector term live in a
// file-scope __device__ array of fixed size instead of context scratch.
//
// Callers that cannot allocate at run time (device memory owned by another
// allocator or a fixed budget, or loops where cudaMalloc's implicit device
// synchronisation is not acceptable) configure a context -- which allocates
// nothing on the device -- and step with this call.
//
// Host code may not pass g_step_scratch to a kernel directly: in host code
// the name is a host-side stand-in, not a device address.  The device
// address is obtained once per device with cudaGetSymbolAddress, with that
// device current, the first time this entry point runs on it.
#include <cmath>
#include <mutex>

#include "ctx.h"

namespace {

// 2 records of at most 32 bytes (FP64) per spin: 4 MiB for 65536 spins.
constexpr size_t kRecMax = 32;
__device__ __align__(256) unsigned char g_step_scratch[2 * kRecMax * SP_STATIC_MAX_SPINS];

constexpr int kMaxDevices = 256;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

// Device address of g_step_scratch on the current device (looked up once).
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_step_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

int fail_static(sp_ctx *c, int code, const char *msg)
{
    c->err = msg;
    return code;
}

template <typename T> int run_static(sp_ctx *c, void *n, const sp_llg_params *p, int n_steps, void *base, cudaStream_t st)
{
    rec_t<T> *np = (rec_t<T> *)base;
    rec_t<T> *q = np + c->N;
    rec_t<T> *nn = (rec_t<T> *)n;
    const Stencil<T> &S = *(const Stencil<T> *)(c->prec == SP_F64 ? (const void *)&c->Sd : (const void *)&c->Sf);
    const CubicParams<T> &CP = *(const CubicParams<T> *)(c->prec == SP_F64 ? (const void *)&c->Cd : (const void *)&c->Cf);
    bool cub = c->cubic && c->use_cubic && (p->solver == SP_HEUN || p->solver == SP_DEPONDT || p->solver == SP_SIB);
    LlgConst<T> k{};
    k.dt = (T)p->dt;
    k.alpha = (T)p->alpha;
    for (int b = 0; b < c->nb; ++b) {
        double mu = c->mu_s[b] * kMuB;
        k.cA[b] = (T)(-kGamma / ((1.0 + p->alpha * p->alpha) * mu));
        k.sig[b] = (T)std::sqrt(2.0 * p->alpha * kBoltzmann * p->T * mu / (kGamma * p->dt));
    }
    llg_set_seed(k, p->seed);
    k.replica = p->replica;
    k.thermal = (p->T > 0 && p->alpha > 0) ? 1 : 0;
    for (int s = 0; s < n_steps; ++s) {
        k.step = p->step0 + (uint64_t)s;
        cudaError_t e = cub ? launch_cubic<T>(0, p->solver, CP, nn, np, q, nn, nullptr, k, cubic_per(c), st,
                                              cubic_rows(c, 0), cubic_lean_taken(c, 0))
                            : launch_llg_pred<T>(p->solver, S, nn, nullptr, np, q, k, st);
        if (e == cudaSuccess)
            e = cub ? launch_cubic<T>(1, p->solver, CP, np, nullptr, q, nn, nullptr, k, cubic_per(c, 1), st,
                                      cubic_rows(c, 1), cubic_lean_taken(c, 1))
                    : launch_llg_corr<T>(p->solver, S, nn, np, q, nullptr, k, st);
        if (e != cudaSuccess) {
            c->err = std::string("LLG launch: ") + cudaGetErrorString(e);
            return SP_ERR_CUDA;
        }
    }
    return SP_OK;
}

}  // namespace

extern "C" int sp_llg_step_static(sp_ctx *c, void *n_dev, const sp_llg_params *p, int n_steps, void *stream)
{
    if (!c) return SP_ERR_ARG;
    if (!c->have_geom || !c->have_ham) return fail_static(c, SP_ERR_STATE, "geometry and Hamiltonian must be set first");
    if (!n_dev || ((uintptr_t)n_dev % (c->prec == SP_F64 ? 32 : 16)) != 0)
        return fail_static(c, SP_ERR_ARG, "spins must be a non-NULL, record-aligned device pointer");
    if (!p) return fail_static(c, SP_ERR_ARG, "NULL parameters");
    if (p->solver < SP_DEPONDT || p->solver > SP_RK4) return fail_static(c, SP_ERR_ARG, "unknown solver");
    if (p->solver == SP_RK4)
        return fail_static(c, SP_ERR_UNSUPPORTED, "sp_llg_step_static: RK4 needs 3 scratch records per spin");
    if (!(p->dt > 0) || !std::isfinite(p->dt)) return fail_static(c, SP_ERR_ARG, "dt must be positive");
    if (!(p->alpha >= 0) || !std::isfinite(p->alpha)) return fail_static(c, SP_ERR_ARG, "alpha must be >= 0");
    if (!(p->T >= 0) || !std::isfinite(p->T)) return fail_static(c, SP_ERR_ARG, "T must be >= 0");
    if (n_steps < 0) return fail_static(c, SP_ERR_ARG, "n_steps must be >= 0");
    if (c->N > SP_STATIC_MAX_SPINS)
        return fail_static(c, SP_ERR_ARG,
                           "sp_llg_step_static: the lattice has more spins than SP_STATIC_MAX_SPINS (65536); "
                           "use sp_llg_step");
    if (c->h.dipole != SP_DIPOLE_NONE)
        return fail_static(c, SP_ERR_UNSUPPORTED, "sp_llg_step_static: the dipole term needs device buffers of its own");
    if (n_steps == 0 || c->N == 0) return SP_OK;
    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) {
        c->err = std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e);
        return SP_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    return c->prec == SP_F64 ? run_static<double>(c, n_dev, p, n_steps, base, st)
                             : run_static<float>(c, n_dev, p, n_steps, base, st);
}
