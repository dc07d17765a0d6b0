/*
 * spo.h -- plain FP64 CPU oracle for the atomistic spin hot path of
 * "Spirit: Multifunctional Framework for Atomistic Spin Simulations"
 * (arXiv:1901.11350).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the independent reference that
 * the CUDA path is checked against.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or constant generator with the CUDA library: everything here
 * is written out directly from the paper's equations, in double precision,
 * with plain loops and no blocking or fusion.
 *
 * Units: energy meV, field T, moments in Bohr magnetons, time ps, length
 * Angstrom, angle rad.  Effective fields B_eff = -dH/dn are in meV.
 *
 * Spin layout: n[3*i + k], i = b + n_basis*(a + n_a*(c1 + n_b*c2)).
 *
 * Every entry point returns 0 on success, a negative SPO_ERR_* code otherwise.
 */
#ifndef SPO_ORACLE_H
#define SPO_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPO_MAX_BASIS 8
#define SPO_MAX_SHELLS 8
#define SPO_MAX_GAUSS 16

enum { SPO_OK = 0, SPO_ERR_ARG = -1, SPO_ERR_STATE = -2, SPO_ERR_UNSUPPORTED = -4 };
enum { SPO_DMI_NONE = 0, SPO_DMI_BULK = 1, SPO_DMI_INTERFACIAL = 2 };
enum { SPO_DIPOLE_NONE = 0, SPO_DIPOLE_DIRECT = 1, SPO_DIPOLE_FFT = 2 };
enum { SPO_DEPONDT = 0, SPO_HEUN = 1, SPO_SIB = 2, SPO_RK4 = 3 };

/* One unique interacting pair <ij> (Eq. 1): basis atom i in cell c interacts
 * with basis atom j in cell c + d, with exchange J and DMI vector D_ij. */
typedef struct {
    int i, j;
    int d[3];
    double J;
    double D[3];
} spo_pair;

/* The extended Heisenberg Hamiltonian, Eq. 1 (quadruplets excluded). */
typedef struct {
    double B[3];                       /* external field, T */
    double K[SPO_MAX_BASIS];           /* uniaxial anisotropy per basis atom, meV */
    double Khat[SPO_MAX_BASIS][3];     /* anisotropy axes */
    int n_shells;                      /* isotropic exchange shells */
    double J[SPO_MAX_SHELLS];          /* meV per unique pair */
    int dmi_kind;                      /* SPO_DMI_* */
    int n_dmi_shells;
    double D[SPO_MAX_SHELLS];          /* DMI magnitude per shell, meV */
    int dipole;                        /* SPO_DIPOLE_* */
    int n_pairs;                       /* extra explicit unique pairs */
    const spo_pair *pairs;
    /* Optional on-site landscape of Appendix G, applied to every spin:
     * sum_g a_g exp(-(1 - n.c_g)^2 / (2 sigma_g^2)); rows (a, sigma, cx, cy, cz),
     * c_g normalised on use.  Test-only: it pins the GNEB oracle. */
    int n_gauss;
    double gauss[SPO_MAX_GAUSS][5];
} spo_hamiltonian;

typedef struct {
    int solver;        /* SPO_DEPONDT, SPO_HEUN, SPO_SIB or SPO_RK4 */
    double dt;         /* ps */
    double alpha;      /* Gilbert damping */
    double T;          /* K */
    uint64_t seed;     /* Philox key */
    uint64_t step0;    /* step counter of the first step */
    uint32_t replica;  /* replica index (Philox counter word 3 = 8*replica) */
} spo_llg_params;

enum { SPO_IMAGE_NORMAL = 0, SPO_IMAGE_CLIMBING = 1, SPO_IMAGE_FALLING = 2 };

typedef struct {
    double dt;         /* fictitious time step */
    double mass;       /* fictitious mass m */
    double k_spring;   /* spring constant, meV/rad^2 */
    int climbing;      /* 1: the highest interior image climbs (used when image_types is NULL) */
    const int *image_types;  /* NULL, or one SPO_IMAGE_* per image (endpoints ignored) */
    double energy_weight;    /* w in [0, 1): spring lengths measured along E(r) (0: geodesic) */
} spo_gneb_params;

typedef struct spo_system spo_system;

int spo_create(spo_system **out);
void spo_destroy(spo_system *s);

/* bravais: 3x3 row-major, row k = lattice vector a_k in units of the lattice
 * constant; basis: n_basis x 3 fractional coordinates; mu_s: n_basis moments. */
int spo_set_geometry(spo_system *s, const double *bravais, int n_basis, const double *basis,
                     const int *n_cells, const int *periodic, double lattice_constant,
                     const double *mu_s);
int spo_set_hamiltonian(spo_system *s, const spo_hamiltonian *h);

int spo_n_spins(const spo_system *s);
int spo_positions(const spo_system *s, double *r);
/* Number of directed neighbour entries and the shell radii actually used. */
int spo_n_neighbours(const spo_system *s, int basis);
int spo_shell_radius(const spo_system *s, int shell, double *radius);

/* B_eff = -dH/dn (meV).  dipole_method overrides the Hamiltonian's dipole
 * mode when >= 0 (lets tests compare DIRECT against FFT). */
int spo_effective_field(const spo_system *s, const double *n, double *B, int dipole_method);
/* Dipole field alone (meV). */
int spo_dipole_field(const spo_system *s, const double *n, double *B, int dipole_method);
/* Direct-sum dipole field at the n_idx sites idx[] only (B is n_idx x 3). */
int spo_dipole_field_direct_at(const spo_system *s, const double *n, int n_idx, const int *idx, double *B);
/* e[0] total, e[1] Zeeman, e[2] anisotropy, e[3] exchange, e[4] DMI,
 * e[5] dipole; each evaluated as a direct sum over its own term of Eq. 1. */
int spo_energy(const spo_system *s, const double *n, double *e);

/* n_steps LLG steps (Appendix B), in place. */
int spo_llg(const spo_system *s, double *n, const spo_llg_params *p, int n_steps);

/* Velocity projection minimiser (Appendix D); v is carried in and out.
 * Stops when max_i |n_i x B_i| < tol or after max_iter iterations. */
int spo_minimise(const spo_system *s, double *n, double *v, double dt, double mass, double tol,
                 int max_iter, int *iters, double *max_torque);

/* GNEB (Section "Geodesic Nudged Elastic Band Method", Appendix F) with the
 * velocity projection optimiser.  chain and vel are n_images x N x 3.
 * Runs n_iter iterations (or stops once max force < tol when tol > 0). */
int spo_gneb(const spo_system *s, double *chain, double *vel, int n_images,
             const spo_gneb_params *p, int n_iter, double tol, double *energies,
             double *max_force, int *iters);
/* One GNEB force evaluation on a chain (forces n_images x N x 3, zero at the
 * endpoints), returning image energies, distances l_{v,v+1} (n_images-1 of
 * them) and the index of the climbing image (-1 if none). */
int spo_gneb_forces(const spo_system *s, const double *chain, int n_images,
                    const spo_gneb_params *p, double *forces, double *energies,
                    double *dist, int *ci);

/* Path analysis of a chain (Sec. GNEB): per image the energy E, reaction
 * coordinate r (cumulative geodesic distance) and slope dE/dr along the
 * tangent (one-sided at the endpoints); the cubic Hermite interpolation of
 * E(r) at n_interp points per segment into r_i, E_i ((M-1)*n_interp + 1
 * values).  Q (may be NULL) receives each image's topological charge. */
int spo_gneb_path(const spo_system *s, const double *chain, int n_images, int n_interp, double *r, double *E,
                  double *slope, double *Q, double *r_i, double *E_i);

/* Energy-weighted length of one path segment: arc length of the curve
 * ((1-w) r, w E(r)), r in [0, h], E the cubic Hermite interpolant with end
 * values Ea, Eb and end slopes da, db (w = 0: h). */
double spo_segment_length(double Ea, double Eb, double da, double db, double h, double w);

/* Metropolis Monte Carlo with cone trial moves (Sec. Monte Carlo). */
typedef struct {
    uint64_t seed;          /* Philox key */
    uint64_t sweep0;        /* index of the first sweep (Philox counter) */
    double target_accept;   /* > 0: adapt each replica's cone after every sweep; 0: fixed cone */
    int sample;             /* 1: accumulate observables after every sweep */
} spo_mc_params;

/* Number of colours of the sweep: k for the sum colouring (c0 + c1 + c2)
 * mod k, else the product colouring's count; 0 when neither applies. */
int spo_mc_colours(const spo_system *s);
/* n_sweeps Metropolis sweeps of n_rep replicas of the system (spins
 * n_rep x N x 3, replica r at temperature T[r] K), each sweep visiting every
 * spin once in a fresh uniformly random order (Sec. Monte Carlo).  cone[r]
 * (radians, in/out) is the trial cone's half-angle.  stats[r*8 + k]
 * accumulates (sum m, m^2, m^4, E, E^2, samples, accepted, trials),
 * m = |sum n_i|/N, E the total energy (meV). */
int spo_mc(const spo_system *s, double *spins, int n_rep, const double *T, const spo_mc_params *p, int n_sweeps,
           double *cone, double *stats);
/* The same Metropolis visits in another sweep order: the colours of the
 * lattice colouring (spo_mc_colours) one after the other, each colour in
 * index order.  A check of a colour-parallel decomposition; SPO_ERR_ARG for
 * a lattice without colouring. */
int spo_mc_coloured(const spo_system *s, double *spins, int n_rep, const double *T, const spo_mc_params *p,
                    int n_sweeps, double *cone, double *stats);

/* Covariant Hessian (Sec. MMF and its appendix on the spin manifold): the
 * action on v (N x 3, projected onto each spin's tangent plane first) of
 * H v|_i = P_i sum_j Hbar_ij v_j - (n_i . grad_i Hbar) v_i, Hbar the second
 * derivatives of the Hamiltonian continued to R^{3N} (no dipole term). */
int spo_hessian_apply(const spo_system *s, const double *n, const double *v, double *out);
/* The same operator as a dense 2N x 2N matrix in the tangent basis
 * T_i = (e1_i, e2_i) (e1 = P_i x or P_i y normalised, e2 = n_i x e1), with
 * the basis itself (N x 3 x 2) in T when not NULL. */
int spo_hessian_dense(const spo_system *s, const double *n, double *H, double *T);

/* Philox4x32-10 block (Salmon et al., SC'11). */
void spo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* The three standard normals of the thermal field of spin i at step `step`. */
void spo_thermal_normals(uint64_t seed, uint64_t step, uint32_t replica, uint32_t i, double eta[3]);

/* Berg-Luescher topological charge of a 2D lattice (Appendix A). */
int spo_topological_charge(const spo_system *s, const double *n, double *Q);

/* Threads the oracle's loops run on (1 without OpenMP). */
int spo_threads(void);

#ifdef __cplusplus
}
#endif
#endif
