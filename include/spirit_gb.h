/*
 * spirit_gb.h -- C ABI of the GB300 (sm_103a) atomistic spin library.
 *
 * The library computes the hot path of the atomistic spin method of
 * "Spirit: Multifunctional Framework for Atomistic Spin Simulations"
 * (arXiv:1901.11350): the effective field B_eff = -dH/dn of the extended
 * Heisenberg Hamiltonian (Eq. 1), fused with Landau-Lifshitz-Gilbert time
 * steps (Eq. 3, Appendix B) with the stochastic thermal field (Eq. 4), the
 * velocity-projection minimiser (Appendix D) and the geodesic nudged elastic
 * band force projection (Sec. "Geodesic Nudged Elastic Band Method",
 * Appendix F).
 *
 * Conventions shared by every call
 * --------------------------------
 * Units: energy meV, magnetic field T, moments in Bohr magnetons, time ps,
 * length Angstrom, angle rad.  Fields returned by the library are B_eff in
 * meV (energy per unit spin direction).
 *
 * Spin buffers are DEVICE pointers owned by the caller, one 4-wide record per
 * spin: float4 (16 B, 16-byte aligned) for a context created with SP_F32,
 * double4 (32 B, 32-byte aligned) for SP_F64.  Record i holds (x, y, z, w);
 * w is ignored on input and written as 0 on output.  Spin index
 * i = b + n_basis * (c0 + n0 * (c1 + n1 * c2)) for basis atom b in cell
 * (c0, c1, c2).  Spin directions must have unit length.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 * default stream).  Calls are stream-ordered and asynchronous unless stated
 * otherwise; results in device memory are valid once the stream reaches
 * them.
 *
 * Ownership: the context owns its host-side description of the system and
 * any device scratch it allocates lazily (predictor states, reduction
 * partials, FFT grids); creating and configuring a context allocates no
 * device memory.  Scratch is freed by sp_destroy.  A context may be used by
 * one host thread at a time; calls on one context must be issued on one
 * stream at a time because they share its scratch.
 *
 * Errors: every call returns SP_OK (0) or a negative SP_ERR_* code, and
 * sp_last_error() returns a message for the last failure on that context.
 * Argument errors are detected on the host before anything is launched.
 *
 * Device status word (the boundary's error path for what only the device
 * sees): each context owns a small status word in mapped, pinned host memory
 * (4 words, allocated by the first call that checks a result).  Every
 * stream-ordered compute call enqueues, after its own kernels, a check of
 * what it produced -- the spin state of sp_llg_step, sp_llg_step_replicas
 * and sp_mc_sweeps, the field of sp_effective_field and sp_gradient, the
 * values of sp_energy, sp_max_torque, sp_topological_charge and sp_sample,
 * the image energies and forces of sp_gneb_step and sp_gneb_batch_step (the
 * first chain's context), the product of sp_hessian_apply -- and a non-finite
 * value (NaN or infinity; the padding lane of a record is not looked at)
 * sets a bit in the word.  The word is surfaced as SP_ERR_NAN (SP_ERR_TIMEOUT
 * for a bounded device-side wait that gave up):
 *   - by the next compute call on the context that finds it set: that call
 *     clears the word, launches nothing and returns the error, with the
 *     kind of result that was bad in sp_last_error.  The host reads the word
 *     without waiting, so a call issued before the GPU has reached the
 *     check does not see it yet;
 *   - deterministically by sp_sync_status(ctx), which waits for the device.
 * Calls that return host results (sp_minimise, sp_minimise_batch,
 * sp_gneb_path, sp_lowest_mode, sp_mmf) check those and return SP_ERR_NAN
 * themselves.  The allocation-free sp_llg_step_static takes no part in it.
 */
#ifndef SPIRIT_GB_H
#define SPIRIT_GB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SP_MAX_BASIS 4   /* basis atoms per cell */
#define SP_MAX_SHELLS 8  /* isotropic neighbour shells */
#define SP_MAX_NBR 96    /* directed neighbour entries, all basis atoms together */

enum {
    SP_OK = 0,
    SP_ERR_ARG = -1,         /* invalid argument or size */
    SP_ERR_STATE = -2,       /* call out of order (e.g. no geometry yet) */
    SP_ERR_CUDA = -3,        /* a CUDA runtime call failed */
    SP_ERR_UNSUPPORTED = -4, /* valid request this library does not implement */
    SP_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
    SP_ERR_NAN = -6          /* a non-finite value was detected */
};

enum { SP_F32 = 0, SP_F64 = 1 };
enum { SP_DMI_NONE = 0, SP_DMI_BULK = 1, SP_DMI_INTERFACIAL = 2 };
enum { SP_DIPOLE_NONE = 0, SP_DIPOLE_FFT = 2 };
enum { SP_DEPONDT = 0, SP_HEUN = 1, SP_SIB = 2, SP_RK4 = 3 };

typedef struct sp_ctx sp_ctx;

/* One unique interacting pair <ij> of Eq. 1: basis atom i of cell c with
 * basis atom j of cell c + d, exchange J (meV) and DMI vector D_ij (meV).
 * The library adds the reverse bond with D_ji = -D_ij. */
typedef struct {
    int i, j;
    int d[3];
    double J;
    double D[3];
} sp_pair;

/* The extended Heisenberg Hamiltonian of Eq. 1 (quadruplets excluded).
 * Exchange and DMI may be given by neighbour shells (distinct bond lengths,
 * nearest first), by explicit pairs, or both.  DMI vectors of a shell:
 * SP_DMI_BULK: D_ij = D rhat_ij; SP_DMI_INTERFACIAL: D_ij = D (z x rhat_ij),
 * rhat_ij the unit bond vector from i to j. */
typedef struct {
    double B[3];                    /* external field, T */
    double K[SP_MAX_BASIS];         /* uniaxial anisotropy per basis atom, meV */
    double Khat[SP_MAX_BASIS][3];   /* anisotropy axes (normalised on use) */
    int n_shells;                   /* exchange shells, 0..SP_MAX_SHELLS */
    double J[SP_MAX_SHELLS];        /* exchange per unique pair and shell, meV */
    int dmi_kind;                   /* SP_DMI_* */
    int n_dmi_shells;               /* shells carrying DMI, 0..SP_MAX_SHELLS */
    double D[SP_MAX_SHELLS];        /* DMI magnitude per shell, meV */
    int dipole;                     /* SP_DIPOLE_NONE or SP_DIPOLE_FFT */
    int n_pairs;                    /* explicit unique pairs in `pairs` */
    const sp_pair *pairs;           /* host array, copied by the call */
} sp_hamiltonian;

/* LLG run parameters (Eq. 3, Eq. 4, Appendix B). */
typedef struct {
    int solver;        /* SP_DEPONDT, SP_HEUN, SP_SIB or SP_RK4 */
    double dt;         /* time step, ps (> 0) */
    double alpha;      /* Gilbert damping (>= 0) */
    double T;          /* temperature, K (>= 0); 0 switches the thermal field off */
    uint64_t seed;     /* Philox4x32-10 key of the thermal field */
    uint64_t step0;    /* step counter of the first step (resume = same seed, later step0) */
    uint32_t replica;  /* replica index; selects an independent noise stream */
} sp_llg_params;

/* Kinds of GNEB images (Sec. GNEB): a climbing image converges onto a saddle
 * point, a falling image onto a local minimum along the path. */
enum { SP_IMAGE_NORMAL = 0, SP_IMAGE_CLIMBING = 1, SP_IMAGE_FALLING = 2 };

/* GNEB parameters (Sec. GNEB, Appendix D, Appendix F). */
typedef struct {
    double dt;         /* velocity-projection time step (> 0) */
    double mass;       /* fictitious mass (> 0) */
    double k_spring;   /* spring constant, meV/rad^2 */
    int climbing;      /* 1: the highest-energy interior image climbs (re-chosen each
                          iteration); used only when image_types is NULL */
    const int *image_types; /* HOST, NULL or one SP_IMAGE_* per image (for a batch: all
                               images of all chains in order); endpoints ignored */
    double energy_weight;   /* w in [0, 1): 0 = springs on geodesic distances; w > 0 =
                               springs on the arc length of ((1-w) r, w E(r)) along the
                               cubic interpolation of the path energy (Sec. GNEB) */
} sp_gneb_params;

/* ------------------------------------------------------------------------
 * Context life cycle
 * ------------------------------------------------------------------------ */

/* Create a context computing in `precision` (SP_F32 or SP_F64) on the
 * current CUDA device.  Allocates host memory only. */
int sp_create(sp_ctx **out, int precision);
/* Destroy a context and free its device scratch (synchronises the device
 * first).  NULL is accepted. */
int sp_destroy(sp_ctx *ctx);
/* Message of the last error on ctx (owned by ctx, valid until the next call
 * on it); a static string for ctx == NULL. */
const char *sp_last_error(const sp_ctx *ctx);

/* Waits for the context's device (cudaDeviceSynchronize, with that device
 * current), then reads and clears the context's status word (see the top of
 * this header): SP_OK, SP_ERR_NAN if an earlier call produced a non-finite
 * value, SP_ERR_TIMEOUT if a bounded device-side wait gave up, SP_ERR_CUDA
 * if the synchronisation reported an error. */
int sp_sync_status(sp_ctx *ctx);

/* Geometry (Sec. "Hamiltonian": arbitrary Bravais vectors and basis cells,
 * open or periodic boundaries per direction).
 *   bravais[9]     row-major 3x3, row k = lattice vector a_k in units of
 *                  lattice_constant (host pointer)
 *   n_basis        1..SP_MAX_BASIS basis atoms
 *   basis[3*n_basis] fractional coordinates of the basis atoms
 *   n_cells[3]     cells per direction (>= 1); N = n_basis*n0*n1*n2 < 2^31
 *   periodic[3]    0 open, 1 periodic
 *   lattice_constant  Angstrom (> 0)
 *   mu_s[n_basis]  moments in Bohr magnetons (> 0)
 * Resets any Hamiltonian set before. */
int sp_set_geometry(sp_ctx *ctx, const double *bravais, int n_basis, const double *basis,
                    const int *n_cells, const int *periodic, double lattice_constant,
                    const double *mu_s);

/* Hamiltonian (Eq. 1).  Builds the directed neighbour stencil on the host:
 * shells are the distinct bond lengths of the infinite lattice, nearest
 * first; across an open boundary a neighbour is absent.  SP_ERR_ARG for more
 * than SP_MAX_NBR directed entries; SP_ERR_UNSUPPORTED for the dipole term
 * with a periodic direction of more than one cell. */
int sp_set_hamiltonian(sp_ctx *ctx, const sp_hamiltonian *h);

/* Number of spins N. */
int sp_n_spins(const sp_ctx *ctx, int *n);

/* ------------------------------------------------------------------------
 * Field, gradient and energy (Eq. 1)
 * ------------------------------------------------------------------------ */

/* B_dev[i] = B_eff,i = -dH/dn_i (meV) for the spins n_dev (N records each,
 * 4-wide, w written 0).  n_dev and B_dev must not overlap. */
int sp_effective_field(sp_ctx *ctx, const void *n_dev, void *B_dev, void *stream);

/* grad_dev[i] = dH/dn_i = -B_eff,i (embedding-space gradient, meV). */
int sp_gradient(sp_ctx *ctx, const void *n_dev, void *grad_dev, void *stream);

/* Energies of Eq. 1 written to e_dev (DEVICE, 6 doubles): total, Zeeman,
 * anisotropy, exchange, DMI, dipole-dipole (meV).  Accumulated in FP64 in a
 * fixed order (bitwise reproducible for a given N and launch shape). */
int sp_energy(sp_ctx *ctx, const void *n_dev, double *e_dev, void *stream);

/* max_i |n_i x B_eff,i| (meV) written to torque_dev (DEVICE, 1 double). */
int sp_max_torque(sp_ctx *ctx, const void *n_dev, double *torque_dev, void *stream);

/* Berg-Luescher topological charge (Appendix A) of a 2D lattice with one
 * basis atom (n2 = 1), written to Q_dev (DEVICE, 1 double): the signed solid
 * angles of the two elementary triangles (c0,c1)(c0+1,c1)(c0,c1+1) and
 * (c0+1,c1)(c0+1,c1+1)(c0,c1+1) of every cell, numbered counter-clockwise
 * about +z, summed in FP64 and divided by 4 pi; triangles crossing an open
 * edge are left out.  A_l = 2 atan2(n_i.(n_j x n_k), 1 + n_i.n_j + n_i.n_k +
 * n_j.n_k), the same angle and sign as the paper's half-angle cosine form.
 * SP_ERR_UNSUPPORTED for other lattices. */
int sp_topological_charge(sp_ctx *ctx, const void *n_dev, double *Q_dev, void *stream);

/* ------------------------------------------------------------------------
 * Time stepping (Eq. 3, Eq. 4, Appendix B)
 * ------------------------------------------------------------------------ */

/* n_steps LLG steps on n_dev in place.
 * dn/dt = n x A, A_i = -gamma/((1+alpha^2) mu_i) (B_i + alpha n_i x B_i),
 * B_i = B_eff,i + B_th,i with B_th,i = sqrt(2 alpha kB T mu_i / (gamma dt)) eta_i
 * and eta_i three standard normals from Philox4x32-10 (key = seed, counter =
 * (i, step mod 2^32, step div 2^32, 8*replica)), Box-Muller on
 * (u0,u1) -> eta_x, eta_y and (u2,u3) -> eta_z, u = (x + 1/2) 2^-32; the same
 * eta in all stages of a step.  Heun renormalises predictor and result;
 * Depondt rotates by |A| dt about -A (Rodrigues); SIB (Appendix C) solves the
 * implicit-midpoint predictor with A(n) and the corrector with A at the
 * predictor's midpoint (n + n^p)/2, each M x = M^T n with M = I + skew(dt A/2)
 * (norm-preserving, no renormalisation); RK4 takes four field evaluations
 * and renormalises the result.  Allocates the context's scratch (2 records
 * per spin, 3 for RK4) on first use. */
int sp_llg_step(sp_ctx *ctx, void *n_dev, const sp_llg_params *p, int n_steps, void *stream);

/* n_steps LLG steps of n_rep replicas of the context's system at once, for
 * thermal averages by sampling the stochastic LLG over time (Appendix
 * "Stochastic LLG": a temperature scan of one lattice).  Replica r sits at
 * spins_dev + r N records (replica-major, the layout of sp_mc_sweeps), has
 * temperature T[r] (K, host array) and the thermal stream p->replica + r
 * (Philox counter word 3 = 8 (p->replica + r)); p->T is ignored.  Each
 * replica's result is the one sp_llg_step gives that replica alone with
 * p->T = T[r] and p->replica + r, bit for bit: the noise amplitudes are
 * computed on the host in FP64 in the same way.  All replicas share one launch per
 * pass (the 27-point path spreads all replicas' (tile, plane) units over the
 * device; batches of two or more do not take the small-lattice single-CTA
 * path, a batch of one is sp_llg_step at T[0]).  Where the 27-point split
 * would give fewer than 8 planes per CTA (unless SP_OPT_PLANES_PER_CTA is
 * set) the per-spin kernels run instead.  Runs of up to 32 steps are
 * replayed from a CUDA graph captured on first use for the launch
 * configuration (up to 4 kept per context; not while `stream` is being
 * captured); their Philox step is read from a device counter the call sets.
 * The kernel profiler does not bracket these launches.  Scratch: 2 (RK4:
 * 3) records per spin and replica; the amplitudes are re-uploaded (with a
 * synchronisation of `stream`) only when n_rep, T, dt or alpha change.
 * SP_ERR_UNSUPPORTED with the dipole term; SP_ERR_ARG for n_rep < 1,
 * n_rep N >= 2^31, a negative or non-finite T[r], p->replica + n_rep > 2^29
 * and the checks of sp_llg_step. */
int sp_llg_step_replicas(sp_ctx *ctx, void *spins_dev, int n_rep, const double *T, const sp_llg_params *p,
                         int n_steps, void *stream);

/* n_steps LLG steps of n_sys systems of different lattices and Hamiltonians
 * at once (the stochastic LLG of Eq. 3-4, Appendix B): system k, described
 * by ctxs[k] (all of one precision, no dipole term), holds its N_k records at
 * record offset offsets[k] of ONE device buffer spins_dev (systems must not
 * overlap), sits at temperature T[k] (K, host array; p->T is ignored) and
 * draws its thermal field from stream p->replica + k.  Every pass is one
 * launch over all systems (a table of (system, block of 256 spins));
 * each system's result is, bit for bit, the one sp_llg_step gives it alone
 * with the neighbour-list kernels (SP_OPT_GENERIC_STENCIL = 1,
 * SP_OPT_SMALL_PATH = 0) at T[k] and replica p->replica + k.  Solvers
 * Depondt, Heun and SIB (RK4: SP_ERR_UNSUPPORTED).  Scratch (2 records per
 * spin of the buffer) and tables belong to ctxs[0]; a call with a new batch
 * layout uploads the tables and synchronises `stream`.  Outside a stream
 * capture, runs of up to 32 steps replay a CUDA graph captured for the
 * layout (kernels read the Philox step from a device counter the call sets;
 * graphs are kept as for sp_llg_step_replicas).  The spin state is
 * checked for non-finite values afterwards (the status word of ctxs[0]). */
int sp_llg_step_batch(sp_ctx *const *ctxs, int n_sys, void *spins_dev, const long long *offsets, const double *T,
                      const sp_llg_params *p, int n_steps, void *stream);

/* ------------------------------------------------------------------------
 * Energy minimisation (Appendix D)
 * ------------------------------------------------------------------------ */

/* Velocity-projection minimisation of n_dev in place, velocities v_dev
 * (same layout, caller-owned, carried in and out; zero them to start).
 * Force F_i = B_i - (B_i.n_i) n_i.  Iteration: n <- normalise(n + dt v +
 * dt^2/(2m) F); F' = F(n); v <- v + dt/(2m)(F + F'); v <- (v.F' > 0) ?
 * (v.F')F'/|F'|^2 : 0 (3N-dimensional dot products).  Stops when
 * max_i |F_i| < tol or after max_iter iterations; convergence is tested on
 * the device, and the host waits for the stream every `check_every`
 * iterations (so this call synchronises `stream`).  *iters and *max_torque
 * are host outputs. */
int sp_minimise(sp_ctx *ctx, void *n_dev, void *v_dev, double dt, double mass, double tol,
                int max_iter, int check_every, int *iters, double *max_torque, void *stream);

/* Batched velocity-projection minimisation: n_sys independent systems, one
 * context each (same precision, no dipole term), relaxed together -- every
 * kernel of an iteration covers all systems in one launch -- with the
 * iteration of sp_minimise applied per system (its own 3N dot products,
 * convergence test and iteration count; a converged system stops moving).
 *   spins_dev, vel_dev  ONE device buffer each; system c's N_c records start
 *                       at record offset offsets[c]; systems must not overlap
 *   iters[c], max_torque[c]  host outputs
 * Synchronises `stream` every check_every iterations.  Scratch belongs to
 * ctxs[0]. */
int sp_minimise_batch(sp_ctx *const *ctxs, int n_sys, void *spins_dev, void *vel_dev, const long long *offsets,
                      double dt, double mass, double tol, int max_iter, int check_every, int *iters,
                      double *max_torque, void *stream);

/* ------------------------------------------------------------------------
 * Geodesic nudged elastic band (Sec. GNEB, Appendix F)
 * ------------------------------------------------------------------------ */

/* n_iter GNEB iterations with the velocity-projection optimiser on a chain of
 * n_images >= 3 images, chain_dev = n_images x N records (image-major),
 * vel_dev the same layout (caller-owned, carried in and out).  Endpoints are
 * never moved.  Per iteration: energies E_v; improved tangent (Henkelman and
 * Jonsson 2000) from the neighbouring images, projected per spin onto the
 * tangent space and normalised in 3N dimensions; geodesic distances
 * l = sqrt(sum_i theta_i^2); forces F = -Pg + (Pg.tau)tau +
 * k (l_{v,v+1} - l_{v-1,v}) tau, and for the climbing image
 * F = -Pg + 2 (Pg.tau) tau, Pg the tangent-space projection of dH/dn; a
 * falling image gets F = -Pg (no spring).  With energy_weight w > 0 the
 * spring uses, instead of l, the arc length of the curve ((1-w) r, w E(r))
 * over each segment, E(r) the cubic Hermite interpolant of the two images'
 * energies and slopes dE/dr = Pg.tau (tangents at the endpoints: the
 * one-sided difference to the neighbour), integrated by adaptive Simpson to
 * 1e-13 l; SP_ERR_ARG for w outside [0, 1) or an unknown image type.
 * The force is re-evaluated at the start of each call (no hidden state).
 * Outputs (DEVICE): energies_dev[n_images] (meV, FP64), max_force_dev[1] =
 * max over interior images and spins of |F_v,i| after the last iteration. */
int sp_gneb_step(sp_ctx *ctx, void *chain_dev, void *vel_dev, int n_images, const sp_gneb_params *p,
                 int n_iter, double *energies_dev, double *max_force_dev, void *stream);

/* Path analysis of a chain of n_images >= 2 images (chain_dev as in
 * sp_gneb_step): HOST outputs per image E[v] (meV, FP64 accumulation),
 * reaction coordinate r[v] (cumulative geodesic distance, r[0] = 0) and slope
 * dE/dr = Pg.tau along the image's tangent (improved tangent inside, one-sided
 * at the endpoints); if r_interp and E_interp are not NULL, the cubic Hermite
 * interpolation of E(r) at n_interp >= 1 equally spaced points per segment
 * ((n_images-1) * n_interp + 1 values, ending at the last image); if Q is not
 * NULL, each image's topological charge (Appendix A; 2D one-atom lattices,
 * else SP_ERR_UNSUPPORTED).  Synchronises `stream`. */
int sp_gneb_path(sp_ctx *ctx, const void *chain_dev, int n_images, int n_interp, double *r, double *E, double *slope,
                 double *Q, double *r_interp, double *E_interp, void *stream);

/* Batched GNEB: n_chains independent chains, each with its own context
 * (geometry and Hamiltonian; all contexts of one precision, no dipole term),
 * stepped together -- every kernel of an iteration covers all images of all
 * chains in one launch, whatever their lattice sizes and image counts.
 *   ctxs[c]       context of chain c (host array)
 *   chains_dev    ONE device buffer; chain c's n_images[c] x N_c records start
 *                 at record offset offsets[c] (image-major); chains must not
 *                 overlap
 *   vel_dev       velocities, same layout (caller-owned, carried in and out)
 *   offsets[c], n_images[c] (>= 3)   host arrays
 *   energies_dev  DEVICE, sum(n_images) doubles: chain c's image energies at
 *                 the prefix sum of n_images before c
 *   max_force_dev DEVICE, n_chains doubles: per chain, max over interior
 *                 images and spins of |F|, after the last iteration
 * Same iteration as sp_gneb_step.  Scratch and tables belong to ctxs[0].  The
 * first call with a given batch layout uploads tables and allocates scratch
 * (it synchronises the stream): make it before any stream capture; calls with
 * an unchanged layout only launch kernels.  Outside a capture, runs of
 * iterations are replayed from a CUDA graph on a private stream ordered
 * after and before `stream` by events. */
int sp_gneb_batch_step(sp_ctx *const *ctxs, int n_chains, void *chains_dev, void *vel_dev, const long long *offsets,
                       const int *n_images, const sp_gneb_params *p, int n_iter, double *energies_dev,
                       double *max_force_dev, void *stream);

/* ------------------------------------------------------------------------
 * Metropolis Monte Carlo (Sec. Monte Carlo)
 * ------------------------------------------------------------------------ */

typedef struct {
    uint64_t seed;          /* Philox key */
    uint64_t sweep0;        /* index of the first sweep (Philox counter; resume = same seed, later sweep0) */
    double target_accept;   /* in (0, 1): after every sweep each replica's cone angle is multiplied
                               by exp(acceptance - target) and kept in [1e-4, pi]; 0: fixed cone */
    int sample;             /* 1: accumulate observables after every sweep */
} sp_mc_params;

/* Number of colours of this context's Monte Carlo sweep (the sweep visits
 * them in order; spins of one colour never interact).  Two colourings:
 *  - sum: colour = (c0 + c1 + c2) mod k for the smallest k >= 2 with one
 *    basis atom, k | n0, no pair offset whose coordinate sum k divides, and
 *    k dividing every periodic extent a pair offset crosses (2 for the
 *    nearest neighbours of an even cubic or square lattice, 3 for 15^3);
 *  - product: colour = basis atom and, per direction, the cell index mod 2
 *    (mod 3 for a periodic direction of odd size divisible by 3), when no
 *    offset reaches beyond the next cell and no offset runs along a
 *    direction of one cell.
 * The sum colouring is taken when it exists with no more colours than the
 * product colouring; 0 when neither exists. */
int sp_mc_colours(sp_ctx *ctx, int *n_colours);

/* n_sweeps Metropolis sweeps of n_rep replicas of the context's system,
 * replica r at temperature T[r] (K, host array; 0 = accept only moves that
 * lower the energy).  A trial move of spin i is a direction drawn uniformly
 * on the cap of half-angle cone_dev[r] around n_i (Philox4x32-10, counter
 * (i, sweep lo, sweep hi, 8 r + 1)), accepted with probability
 * min(1, exp(-dE / k_B T)), dE the exact energy change (Zeeman, exchange,
 * DMI, anisotropy; no dipole term).  A sweep updates the lattice colour by
 * colour (spins of one colour do not interact; the paper visits spins in a
 * random sequential order -- both sample the Boltzmann distribution).
 *   spins_dev  n_rep x N records, replica-major
 *   cone_dev   DEVICE, n_rep doubles (radians), in/out
 *   stats_dev  DEVICE, n_rep x 8 doubles, accumulated (not reset): sum of m,
 *              m^2, m^4, E, E^2 (m = |sum_i n_i| / N, E total energy in meV,
 *              each after every sweep when p->sample), the number of samples,
 *              accepted trials and trials
 * SP_ERR_ARG for NULL or misaligned pointers (records 16 B aligned in FP32,
 * 32 B in FP64; cone and stats 8 B), n_rep < 1, n_sweeps < 0, more than
 * 2^31 spins over all replicas, target_accept outside [0, 1) or a negative
 * temperature; SP_ERR_UNSUPPORTED for the dipole term or a lattice without
 * colouring.
 * Runs of sweeps are replayed from a CUDA graph on a private stream ordered
 * after and before `stream` by events. */
int sp_mc_sweeps(sp_ctx *ctx, void *spins_dev, int n_rep, const double *T, const sp_mc_params *p, int n_sweeps,
                 double *cone_dev, double *stats_dev, void *stream);

/* Accumulate the observables of n_rep replicas (n_rep x N records,
 * replica-major) into stats_dev (DEVICE, n_rep x 8 doubles, the layout of
 * sp_mc_sweeps): m, m^2, m^4, E, E^2 and one more sample; the acceptance
 * slots 6 and 7 are not touched.  m = |sum_i n_i| / N and E the total energy
 * of Eq. 1 without the dipole term, both summed in a fixed order to FP64
 * accuracy (FP32 contexts: float-float within a thread and a warp, FP64
 * across warps and blocks).  Stream-ordered, no synchronisation.
 * SP_ERR_ARG for NULL or misaligned pointers; SP_ERR_UNSUPPORTED with the
 * dipole term. */
int sp_sample(sp_ctx *ctx, const void *spins_dev, int n_rep, double *stats_dev, void *stream);

/* ------------------------------------------------------------------------
 * Covariant Hessian, lowest mode and minimum mode following (Sec. MMF and
 * the appendix on the manifold of constant-length spins).  All three return
 * SP_ERR_ARG for NULL pointers or record arrays off a record boundary (16 B
 * in FP32, 32 B in FP64) and SP_ERR_UNSUPPORTED with the dipole term.
 * ------------------------------------------------------------------------ */

/* out = H v: the covariant Hessian of the energy at the configuration n_dev
 * acting on v_dev (N records each; v is first projected per spin onto the
 * tangent plane of n):  H v|_i = P_i (Hbar v)_i - (n_i . grad_i Hbar) v_i,
 * Hbar the second derivatives of the Hamiltonian continued to R^{3N}
 * (exchange, DMI, anisotropy; the Zeeman term is linear), grad_i Hbar = -B_i.
 * out_dev is tangent; it must not alias v_dev.  No dipole term. */
int sp_hessian_apply(sp_ctx *ctx, const void *n_dev, const void *v_dev, void *out_dev, void *stream);

/* Lowest eigenvalue (*lambda, host) and unit eigenvector (mode_dev, N
 * records, in/out: a non-zero mode_dev is the start vector, zero selects a
 * fixed pseudo-random start) of the covariant Hessian at n_dev, by `krylov`
 * (1..256) Lanczos steps with full reorthogonalisation, at most 2N (the
 * tangent space's dimension).  The iteration stops early at an invariant
 * subspace: a residual below 1e-13 (FP64) or 1e-5 (FP32) of the running
 * estimate of the tridiagonal matrix's norm.  In exact arithmetic
 * krylov >= 2N gives the exact lowest pair.  Synchronises `stream`. */
int sp_lowest_mode(sp_ctx *ctx, const void *n_dev, void *mode_dev, int krylov, double *lambda, void *stream);

typedef struct {
    double dt;    /* velocity-projection time step (> 0) */
    double mass;  /* fictitious mass (> 0) */
    int krylov;   /* Lanczos steps per lowest-mode evaluation (1..256) */
} sp_mmf_params;

/* n_iter iterations of minimum mode following: the velocity projection of
 * Appendix D with the effective force F_eff = F - 2 (F.l) l, F the
 * tangent-space force, l the lowest mode of the Hessian at the current
 * state (recomputed by sp_lowest_mode at every force evaluation, started
 * from the previous mode); where the lowest eigenvalue is not negative,
 * F_eff = -(F.l) l (climbs along the lowest mode only).  n_dev, vel_dev and
 * mode_dev (N records each) are carried in and out.  *max_force (host) =
 * max_i |F_i| and *lambda the lowest eigenvalue at the final state.
 * Synchronises `stream`. */
int sp_mmf(sp_ctx *ctx, void *n_dev, void *vel_dev, void *mode_dev, const sp_mmf_params *p, int n_iter,
           double *max_force, double *lambda, void *stream);

/* ------------------------------------------------------------------------
 * Harmonic transition-state theory (Sec. "Harmonic Transition-State Theory",
 * appendix on the curved manifold).  SP_F64 contexts without the dipole term,
 * 1..SP_HTST_MAX_SPINS spins; SP_ERR_UNSUPPORTED for SP_F32 or the dipole
 * term, SP_ERR_ARG for larger lattices or NULL/misaligned pointers.
 * ------------------------------------------------------------------------ */
#define SP_HTST_MAX_SPINS 2048

/* All 2N eigenvalues of the covariant Hessian at n_dev (the operator of
 * sp_hessian_apply in the 2N-dimensional tangent space), ascending, into the
 * HOST array eig[2N].  Lanczos over the whole tangent space with classical
 * Gram-Schmidt reorthogonalisation done twice against every stored vector,
 * restarted from a new pseudo-random tangent field where the Krylov space
 * closes (so degenerate eigenvalues appear with their multiplicity), then
 * bisection on Sturm counts of the resulting tridiagonal matrix.  Device
 * scratch: (2N + 1) N records of 32 B and small buffers (268 MB at 2048
 * spins), kept by the context.  Synchronises `stream`. */
int sp_hessian_spectrum(sp_ctx *ctx, const void *n_dev, double *eig, void *stream);

typedef struct {
    double zero_tol;  /* eigenvalues with |lambda| <= zero_tol (meV) count as zero modes (>= 0) */
    double V_min;     /* phase-space volume of the zero modes at the minimum (1 without any) */
    double V_sad;     /* the same at the saddle point */
} sp_htst_params;

typedef struct {
    double E_min, E_sad, dE;          /* energies (meV, FP64 sums) and barrier dE = E_sad - E_min */
    double log_det_min, log_det_sad;  /* sum of ln(lambda) over the eigenvalues above zero_tol */
    double omega0;                    /* Omega_0 = sqrt(prod' lambda^M / prod' lambda^S) */
    double v;                         /* sqrt(sum' a_i^2 / lambda^S_i), a_i the dynamical
                                         matrix's unstable-mode row in the eigenbasis */
    double lambda_unstable;           /* lowest eigenvalue at the saddle point (meV) */
    double prefactor;                 /* v / (2 pi) Omega_0 V_sad / V_min */
    int n_zero_min, n_zero_sad;       /* zero modes N0^M, N0^S */
    int n_neg_min, n_neg_sad;         /* eigenvalues below -zero_tol (0 and 1 for a minimum
                                         and a first-order saddle) */
} sp_htst_result;

/* HTST rate prefactor of the transition from the minimum n_min_dev over the
 * first-order saddle point n_sad_dev (N records each, device):
 *   Gamma = prefactor (2 pi kB T)^((N0^M - N0^S)/2) exp(-dE / kB T),
 * prefactor = v / (2 pi) Omega_0 V^S / V^M (1/ps when both states have the
 * same number of zero modes).  Omega_0 from the two spectra of
 * sp_hessian_spectrum.  v from the linearised precession without damping,
 * d(dn_i)/dt = (gamma / mu_i) n_i x (H dn)_i (gamma = 0.176085963023
 * rad/(ps T), mu_i = mu_s mu_B): with e_1 the saddle's unstable eigenvector
 * (Ritz vector of the lowest eigenvalue) and u_i = (gamma / mu_i) n_i x e_1,i,
 * v^2 = u . H u at the saddle, which equals sum' a_i^2 / lambda_i up to the
 * zero modes' share (|lambda| <= zero_tol; at most zero_tol |u|^2).  Result
 * in *out (host).  Synchronises `stream`. */
int sp_htst(sp_ctx *ctx, const void *n_min_dev, const void *n_sad_dev, const sp_htst_params *p, sp_htst_result *out,
            void *stream);

/* ------------------------------------------------------------------------
 * Allocation-free LLG stepping
 * ------------------------------------------------------------------------
 * The paper has no counterpart to this entry point.  It is for callers that
 * cannot allocate device memory while they run: programs whose device memory
 * is owned by another allocator or held to a fixed budget, and loops where
 * the implicit device synchronisation of cudaMalloc is not acceptable.
 * Creating and configuring a context allocates no device memory, and this
 * call allocates none either: the predictor state and the folded corrector
 * term (2 records per spin) live in one file-scope device array of
 * 2 * 32 * SP_STATIC_MAX_SPINS bytes (4 MiB) that every GPU loading the
 * library holds until the process exits.
 *
 * Same arguments and the same per-spin arithmetic as sp_llg_step's
 * two-pass launches: bit for bit the result of sp_llg_step whenever that
 * call takes them too (lattices above 2048 spins, or SP_OPT_SMALL_PATH = 0);
 * where sp_llg_step takes its small-lattice path instead, the two agree
 * within the precision's tolerance.  Limits and behaviour:
 *   - N > SP_STATIC_MAX_SPINS: SP_ERR_ARG with a message, nothing launched;
 *   - a Hamiltonian with the dipole term, or the RK4 solver (3 records per
 *     spin): SP_ERR_UNSUPPORTED;
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, once per device, with that device current) and
 *     may load the library's kernels: make that first call before any CUDA
 *     stream capture;
 *   - every call, on every context and stream of a device, shares the one
 *     array, which keeps the last call's contents (nothing in it needs to
 *     start at zero): calls that overlap on the GPU race and give wrong
 *     results, so serialise them (one stream, or events between streams);
 *   - kernel timing (sp_profile_enable) and the device status word (a
 *     result check would need the status word's allocation) do not apply
 *     to this call. */
#define SP_STATIC_MAX_SPINS 65536
int sp_llg_step_static(sp_ctx *ctx, void *n_dev, const sp_llg_params *p, int n_steps, void *stream);

/* ------------------------------------------------------------------------
 * Execution options (how, not what: results agree within the precision's
 * tolerance whichever option is chosen)
 * ------------------------------------------------------------------------ */

enum {
    /* value 1: evaluate the field with the generic neighbour-list kernels even
     * when the shell-symmetric 27-point plane-streaming path applies (one
     * basis atom, bonds within the 3x3x3 cell neighbourhood, one exchange
     * constant per face/edge/corner class, DMI on faces only; LLG steps with
     * any solver, RK4 only without the dipole term); 0: default */
    SP_OPT_GENERIC_STENCIL = 1,
    /* work of one CTA of the 27-point path, in (32 x 8 column tile, plane)
     * units taken in tile-major order (>= 1); 0 (default): the units spread
     * evenly over one wave of the CTAs the device keeps resident (reading
     * the option then returns that value once it has been computed) */
    SP_OPT_PLANES_PER_CTA = 2,
    /* read only: 1 when the 27-point path applies to this Hamiltonian */
    SP_OPT_HAS_CUBIC_PATH = 3,
    /* value 1: evaluate the dipole field with the radix-2 shared-memory FFT
     * kernels even where the FP32 warp-FFT path (1024 x 1024 padded grid)
     * applies; 0: default */
    SP_OPT_GENERIC_FFT = 4,
    /* 1 (default): lattices of at most 2048 spins without the dipole term,
     * stepped with Depondt, Heun or SIB, take the small-lattice paths: in
     * FP32 one CTA keeps the lattice in shared memory and runs all steps of
     * a call in the kernel; in FP64 the per-spin kernels run in small
     * blocks spread over the SMs (both with the generic path's per-spin
     * arithmetic); 0: never */
    SP_OPT_SMALL_PATH = 5,
    /* the corrector pass's work per CTA of the 27-point path, in the units of
     * SP_OPT_PLANES_PER_CTA (>= 1); 0: the corrector takes the value of
     * SP_OPT_PLANES_PER_CTA (default; setting that option, or sp_autotune,
     * overrides this one).  Reading returns the value the corrector uses:
     * its own, else the shared user value, else its balanced split (the
     * corrector keeps more CTAs resident than the predictor) */
    SP_OPT_PLANES_PER_CTA_CORR = 6,
    /* 1 (default): sp_mc_sweeps on a lattice of at most 2048 spins with at
     * most 32 colours runs one CTA per replica, the replica held in shared
     * memory for all sweeps of the call; 0: one launch per colour over all
     * replicas (always taken for larger lattices, where it is faster).  Both
     * give the same spins, cones and counts; the observable sums differ in
     * rounding order. */
    SP_OPT_MC_RESIDENT = 7,
    /* read only: device memory the context's own buffers hold, in KiB rounded
     * up -- the LLG predictor scratch, reduction partials, dipole field,
     * path-analysis charges, replica noise amplitudes and step counter (not
     * the dipole plan, minimiser, Monte Carlo or Hessian workspaces).  0 on a
     * context that has allocated none of them */
    SP_OPT_SCRATCH_KIB = 8,
    /* value 1: the iterations of an sp_gneb_step / sp_gneb_batch_step call
     * (the batch reads the option of its first chain's context) run in one
     * persistent cooperative launch -- every image of every chain, the
     * passes separated by grid-wide barriers, tangent weights and force
     * coefficients computed per work block -- instead of one launch per pass
     * replayed from a CUDA graph; the iterates are bit-identical.  A barrier
     * wait that exceeds SP_OPT_WAIT_LIMIT polls gives up: every block then
     * leaves the kernel, the chain is left part-way through an iteration, and
     * the context's status word reports SP_ERR_TIMEOUT (sp_sync_status or the
     * next call).  0 (default): one launch per pass */
    SP_OPT_GNEB_PERSISTENT = 9,
    /* polls (about 0.1-0.5 us each) a grid-barrier wait of the persistent
     * GNEB kernel makes before it gives up (>= 1); 0: the default, 2^21 */
    SP_OPT_WAIT_LIMIT = 10,
    /* columns per thread of the 27-point kernels, 1 (default) or 2: with 2 a
     * thread owns two columns of a 32 x 16 tile (the same arithmetic per
     * spin, bit-identical results) -- FP32 single lattices without the
     * dipole term only, other calls take 1.  Sets both passes; units of
     * SP_OPT_PLANES_PER_CTA are then (32 x 16 tile, plane).  sp_autotune
     * chooses it per pass.  Reading returns the predictor's value in use */
    SP_OPT_CUBIC_ROWS = 11,
    /* the same for the corrector pass alone */
    SP_OPT_CUBIC_ROWS_CORR = 12,
    /* 1 (default): FP32 stochastic Heun on the 27-point path takes the lean
     * passes where the lattice's xy plane is cut into whole column tiles of
     * the tile height in use (nx a multiple of 32; ny of 8 with one column
     * per thread, of 16 with two); the same method and stencil, fewer
     * instructions per spin, results equal to the general passes within FP32
     * rounding (not bit for bit; one and two columns give the same bits).
     * 0: always the general passes.  Reading returns 1 when the lean passes
     * would be taken for a Heun call of this context */
    SP_OPT_CUBIC_LEAN = 13
};
int sp_set_option(sp_ctx *ctx, int option, int value);
/* Choose the tile height (SP_OPT_CUBIC_ROWS) and the work per CTA of the
 * 27-point path by measurement, for each pass separately (the passes have
 * different register budgets and occupancy): times the LLG predictor and
 * corrector passes (Heun with the thermal field on; they read n_dev and
 * write only context scratch, so the spins are unchanged) with CUDA events
 * on `stream`, for each tile height the balanced split, finer splits and a
 * few fixed run lengths, and keeps the fastest of each pass.  Allocates
 * the LLG scratch if needed and synchronises `stream`.  SP_OK without effect
 * when the 27-point path does not apply.  *chosen (host, may be NULL)
 * receives the predictor's value (SP_OPT_PLANES_PER_CTA reads it back,
 * SP_OPT_PLANES_PER_CTA_CORR the corrector's; setting SP_OPT_PLANES_PER_CTA
 * applies one value to both passes again). */
int sp_autotune(sp_ctx *ctx, const void *n_dev, int *chosen, void *stream);
int sp_get_option(const sp_ctx *ctx, int option, int *value);

/* Choose by measurement how sp_gneb_batch_step runs a batch: for the batch
 * described as in sp_gneb_batch_step, runs a warm-up call and then n_trial
 * (>= 1) iterations with one launch per pass and with the persistent kernel,
 * each from device copies of chains_dev and vel_dev (the caller's buffers
 * are not changed; the copies are allocated and freed by this call), timed
 * with CUDA events on `stream`, and sets SP_OPT_GNEB_PERSISTENT of ctxs[0]
 * to the faster.  *persistent (host, may be NULL) receives the choice, ms
 * (host, may be NULL, 2 doubles) the two times in ms.  Synchronises `stream`;
 * a trial that met a non-finite value or a timed-out wait returns that
 * error. */
int sp_gneb_batch_autotune(sp_ctx *const *ctxs, int n_chains, const void *chains_dev, const void *vel_dev,
                           const long long *offsets, const int *n_images, const sp_gneb_params *p, int n_trial,
                           int *persistent, double *ms, void *stream);

/* ------------------------------------------------------------------------
 * Kernel timing (tracing aid, not part of the method)
 * ------------------------------------------------------------------------ */

enum { SP_PROF_LLG_PREDICTOR = 0, SP_PROF_LLG_CORRECTOR = 1, SP_PROF_DIPOLE = 2, SP_PROF_KINDS = 3 };

/* on != 0: from now on every launch of the LLG predictor and corrector
 * kernels and of the dipole field pipeline is bracketed by a pair of CUDA
 * events recorded on its stream (off by default; do not enable while
 * capturing a CUDA graph).  Events are recycled from a pool of 4096 pairs,
 * waiting for the oldest when the pool is full. */
int sp_profile_enable(sp_ctx *ctx, int on);
/* Waits for all recorded events, then returns the summed device time (ms)
 * and the number of launches of kernel class `kind` since the last read of
 * that class, and resets them.  Host outputs. */
int sp_profile_read(sp_ctx *ctx, int kind, double *total_ms, long long *launches);

#ifdef __cplusplus
}
#endif
#endif
