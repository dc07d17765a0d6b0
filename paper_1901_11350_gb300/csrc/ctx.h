// ctx.h -- the context behind the opaque sp_ctx handle (shared by the
// translation units that implement the C ABI).
#pragma once

#include <algorithm>
#include <string>
#include <vector>

#include "cubic.h"
#include "dipole.h"
#include "internal.h"
#include "minimise.h"

using namespace spgb;

namespace spgb_ctx {

struct HostNbr {
    int b, jb, d[3];
    double J, D[3];
};

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// An instantiated CUDA graph of a run of LLG steps of a replica batch and
// the launch configuration it was captured for.
struct LlgGraph {
    std::vector<char> key;
    cudaGraphExec_t exec;
};

// Pool of CUDA event pairs bracketing kernel launches (sp_profile_*).
struct Profiler {
    static constexpr int kPairs = 4096;
    bool on = false;
    std::vector<cudaEvent_t> ev;  // 2 per pair
    std::vector<int> kind;
    int used = 0;
    double ms[SP_PROF_KINDS] = {0, 0, 0};
    long long count[SP_PROF_KINDS] = {0, 0, 0};

    cudaError_t drain()
    {
        for (int p = 0; p < used; ++p) {
            cudaError_t e = cudaEventSynchronize(ev[2 * p + 1]);
            if (e != cudaSuccess) return e;
            float t = 0;
            e = cudaEventElapsedTime(&t, ev[2 * p], ev[2 * p + 1]);
            if (e != cudaSuccess) return e;
            ms[kind[p]] += t;
            count[kind[p]] += 1;
        }
        used = 0;
        return cudaSuccess;
    }
    // returns the pair index to record into, or -1 when profiling is off
    int begin(int k, cudaStream_t st)
    {
        if (!on) return -1;
        if (ev.empty()) {
            ev.resize(2 * kPairs);
            kind.resize(kPairs);
            for (auto &e : ev) cudaEventCreate(&e);
        }
        if (used == kPairs && drain() != cudaSuccess) return -1;
        int p = used++;
        kind[p] = k;
        cudaEventRecord(ev[2 * p], st);
        return p;
    }
    void end(int p, cudaStream_t st)
    {
        if (p >= 0) cudaEventRecord(ev[2 * p + 1], st);
    }
    ~Profiler()
    {
        for (auto &e : ev) cudaEventDestroy(e);
    }
};

}  // namespace spgb_ctx

using namespace spgb_ctx;

struct McScratch;  // Monte Carlo scratch (mc.cu)
void mc_scratch_destroy(McScratch *m);
struct HessScratch;  // Hessian / Lanczos / MMF scratch (hessian.cu)
void hess_scratch_destroy(HessScratch *h);
struct HtstScratch;  // full-spectrum Lanczos scratch (htst.cu)
void htst_scratch_destroy(HtstScratch *h);

struct sp_ctx {
    int prec = SP_F32;
    int device = 0;
    std::string err;
    bool have_geom = false, have_ham = false;
    // geometry
    double A[3][3] = {};
    int nb = 1;
    double basis[SP_MAX_BASIS][3] = {};
    int nc[3] = {1, 1, 1}, per[3] = {0, 0, 0};
    double a = 1.0;
    double mu_s[SP_MAX_BASIS] = {};
    int N = 0;
    // Hamiltonian
    sp_hamiltonian h = {};
    std::vector<sp_pair> pairs;
    std::vector<HostNbr> nbr;
    Stencil<float> Sf = {};
    Stencil<double> Sd = {};
    // shell-symmetric 27-point fast path (valid when `cubic` is set)
    bool cubic = false;
    bool use_cubic = true;  // cleared by SP_OPT_GENERIC_STENCIL
    bool generic_fft = false;  // SP_OPT_GENERIC_FFT
    bool use_small = true;     // SP_OPT_SMALL_PATH
    bool use_mc_resident = true;  // SP_OPT_MC_RESIDENT
    int gneb_persistent = 0;      // SP_OPT_GNEB_PERSISTENT
    int wait_limit = 0;           // SP_OPT_WAIT_LIMIT (0: default)
    int zc = 0;             // units per CTA of the 27-point path; 0 = balanced (see cubic_per)
    int zc_corr = 0;        // the corrector's, when the autotuner chose it separately
    int zc_auto = 0;        // balanced value, computed on first use
    int zc_auto_corr = 0;   // the same for the corrector pass (its own occupancy)
    int rows[2] = {1, 1};   // columns per thread of the 27-point predictor and corrector (1 or 2)
    int lean = 1;           // the lean FP32 Heun passes where the lattice fits them (SP_OPT_CUBIC_LEAN)
    CubicParams<float> Cf = {};
    CubicParams<double> Cd = {};
    // device scratch (allocated on first use)
    DevBuf pred;      // 2 records per spin: predictor state and folded corrector term
    DevBuf partials;  // reduction partials
    DevBuf bdd;       // dipole field, 1 record per spin
    DevBuf qbuf;      // per-image topological charges of a path analysis
    DevBuf rsig;      // noise amplitudes of the last batch of replicas
    std::vector<double> rsig_key;  // what they were computed from
    DevBuf step_ctr;               // Philox step base of replayed replica graphs
    DevBuf lb_tab;                 // tables of the last batch of lattices (sp_llg_step_batch)
    std::vector<char> lb_key;      // what they were built from
    std::vector<LlgGraph> lg_graphs;
    cudaStream_t lg_stream = nullptr;  // capture stream of those graphs
    // device status word (mapped pinned host memory, allocated on first use;
    // status_d is its device address): word 0 collects the SITE_* bits of
    // non-finite results, word 1 those of bounded waits that gave up
    unsigned *status_h = nullptr, *status_d = nullptr;
    DipolePlan *dip = nullptr;
    MinScratch *mins = nullptr;
    McScratch *mc = nullptr;
    HessScratch *hess = nullptr;
    HtstScratch *htst = nullptr;
    Profiler prof;
};

// Where a non-finite value was seen (bits of status word 0).
enum {
    SITE_STATE = 1,    // spins after LLG steps or Monte Carlo sweeps
    SITE_FIELD = 2,    // effective field or gradient
    SITE_ENERGY = 4,   // energies or max torque
    SITE_RELAX = 8,    // GNEB image energies or forces
    SITE_SAMPLE = 16,  // sampled observables or topological charge
    SITE_HESSIAN = 32  // Hessian-vector product
};
// Device address of ctx's status word (allocated on first use), or null
// with an error set on ctx.
unsigned *status_word(sp_ctx *c);
// SP_OK, or the error a pending status word stands for (the word is read
// without waiting for the device and cleared).
int status_enter(sp_ctx *c);
// Enqueue the finiteness check of n_rec records (spins, fields) or n_val
// doubles (energies, forces) on st.
int status_check_records(sp_ctx *c, const void *recs, long n_rec, unsigned site, cudaStream_t st);
int status_check_doubles(sp_ctx *c, const double *v, long n_val, unsigned site, cudaStream_t st);

// Units per CTA of the 27-point path for a batch of n_rep replicas: the
// user's choice, or all replicas' units spread over one wave of resident CTAs.
inline int cubic_per_batch(sp_ctx *c, int pass, int n_rep)
{
    if (pass == 1 && c->zc_corr > 0) return c->zc_corr;
    if (c->zc > 0) return c->zc;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 1;
    long slots = (long)nsm * cubic_resident_ctas(c->prec, pass);
    long units = cubic_units(c->nc[0], c->nc[1], c->nc[2]) * n_rep;
    return (int)std::max(1L, (units + slots - 1) / slots);
}

// Columns per thread the 27-point pass of a single lattice takes.
inline int cubic_rows(const sp_ctx *c, int pass)
{
    return cubic_rows_taken(c->prec, c->rows[pass], false, c->h.dipole != SP_DIPOLE_NONE);
}

// Whether a Heun pass of this context on the 27-point path takes the lean
// FP32 kernels (cubic_lean.cu): option on, FP32, no dipole field and a
// lattice cut into whole column tiles of the pass's height (32 x 8 rows).
inline bool cubic_lean_taken(const sp_ctx *c, int pass)
{
    return c->lean && c->prec == SP_F32 && c->cubic && c->use_cubic && c->h.dipole == SP_DIPOLE_NONE &&
           cubic_lean_fits(c->nc[0], c->nc[1], cubic_rows(c, pass));
}

// Units per CTA of the 27-point path: the user's choice, or the units spread
// evenly over one wave of resident CTAs on the current device (units of the
// pass's tile height, see cubic_rows).
inline int cubic_per(sp_ctx *c, int pass = 0)
{
    if (pass == 1 && c->zc_corr > 0) return c->zc_corr;
    if (c->zc > 0) return c->zc;
    int &a = pass == 0 ? c->zc_auto : c->zc_auto_corr;
    if (a <= 0) {
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 1;
        const int rows = cubic_rows(c, pass);
        long slots = (long)nsm * (cubic_lean_taken(c, pass) ? cubic_lean_resident_ctas(pass, rows)
                                                             : cubic_resident_ctas(c->prec, pass, rows));
        long units = cubic_units(c->nc[0], c->nc[1], c->nc[2], rows);
        a = (int)std::max(1L, (units + slots - 1) / slots);
    }
    return a;
}
