/*
 * spo.c -- plain FP64 CPU oracle (test infrastructure only; see spo.h).
 *
 * Written from "Spirit: Multifunctional Framework for Atomistic Spin
 * Simulations" (arXiv:1901.11350):
 *   Eq. 1 (Hamiltonian)            -> field_local(), spo_energy()
 *   Sec. "Dipolar interactions"    -> dipole_direct(), dipole_fft()
 *   Eq. 3/4 (LLG, thermal field)   -> llg_A(), spo_llg()
 *   Appendix B (Heun, Depondt)     -> spo_llg()
 *   Appendix C (SIB), RK4          -> sib_solve(), spo_llg()
 *   Appendix D (velocity proj.)    -> spo_minimise(), spo_gneb()
 *   Sec. GNEB + Appendix F         -> spo_gneb_forces()
 *   Appendix A (topological charge)-> spo_topological_charge()
 *   Appendix G (Gaussian landscape)-> gauss_terms()
 * Readings of passages the paper leaves open are noted where they are used.
 *
 * Everything is a direct loop over the definition; the only library
 * primitives are libm's transcendental functions.
 */
#include "spo.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* CODATA 2018 values, in the oracle's unit system. */
#define MU_B 0.05788381806        /* Bohr magneton, meV/T */
#define K_B 0.08617333262         /* Boltzmann constant, meV/K */
#define GAMMA_E 0.176085963023    /* electron gyromagnetic ratio, rad/(ps T) */
#define C_DIP 0.05368151123574179 /* mu0/(4 pi) mu_B^2 / Angstrom^3, in meV */

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int jb;      /* basis index of the neighbour */
    int d[3];    /* cell offset */
    double J;    /* exchange, meV */
    double D[3]; /* DMI vector D_ij seen from this atom, meV */
} nbr_t;

struct spo_system {
    int have_geom, have_ham;
    double A[3][3]; /* Bravais vectors (rows), units of a */
    int nb;
    double basis[SPO_MAX_BASIS][3];
    int nc[3], per[3];
    double a;
    double mu[SPO_MAX_BASIS];
    int N;
    spo_hamiltonian h; /* copy; h.pairs is not kept */
    int n_nbr[SPO_MAX_BASIS];
    nbr_t *nbr[SPO_MAX_BASIS];
    int n_shell_r;
    double shell_r[SPO_MAX_SHELLS];
};

/* ------------------------------------------------------------------ */
/* small vector helpers                                                */
/* ------------------------------------------------------------------ */
static double dot3(const double *x, const double *y) { return x[0] * y[0] + x[1] * y[1] + x[2] * y[2]; }
static void cross3(const double *x, const double *y, double *z)
{
    double t0 = x[1] * y[2] - x[2] * y[1];
    double t1 = x[2] * y[0] - x[0] * y[2];
    double t2 = x[0] * y[1] - x[1] * y[0];
    z[0] = t0; z[1] = t1; z[2] = t2;
}
static void normalise3(double *x)
{
    double r = sqrt(dot3(x, x));
    if (r > 0) { x[0] /= r; x[1] /= r; x[2] /= r; }
}

int spo_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* geometry (Sec. "Hamiltonian": Bravais vectors and basis cell)       */
/* ------------------------------------------------------------------ */
int spo_create(spo_system **out)
{
    if (!out) return SPO_ERR_ARG;
    *out = (spo_system *)calloc(1, sizeof(spo_system));
    return *out ? SPO_OK : SPO_ERR_STATE;
}

static void free_nbr(spo_system *s)
{
    for (int b = 0; b < SPO_MAX_BASIS; ++b) { free(s->nbr[b]); s->nbr[b] = NULL; s->n_nbr[b] = 0; }
}

void spo_destroy(spo_system *s)
{
    if (!s) return;
    free_nbr(s);
    free(s);
}

int spo_set_geometry(spo_system *s, const double *bravais, int n_basis, const double *basis,
                     const int *n_cells, const int *periodic, double lattice_constant,
                     const double *mu_s)
{
    if (!s || !bravais || !basis || !n_cells || !periodic || !mu_s) return SPO_ERR_ARG;
    if (n_basis < 1 || n_basis > SPO_MAX_BASIS || !(lattice_constant > 0)) return SPO_ERR_ARG;
    long N = n_basis;
    for (int k = 0; k < 3; ++k) {
        if (n_cells[k] < 1) return SPO_ERR_ARG;
        N *= n_cells[k];
    }
    if (N > 0x7fffffffL) return SPO_ERR_ARG;
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) s->A[k][l] = bravais[3 * k + l];
    s->nb = n_basis;
    for (int b = 0; b < n_basis; ++b) {
        for (int l = 0; l < 3; ++l) s->basis[b][l] = basis[3 * b + l];
        s->mu[b] = mu_s[b];
    }
    for (int k = 0; k < 3; ++k) { s->nc[k] = n_cells[k]; s->per[k] = periodic[k] ? 1 : 0; }
    s->a = lattice_constant;
    s->N = (int)N;
    s->have_geom = 1;
    s->have_ham = 0;
    free_nbr(s);
    return SPO_OK;
}

int spo_n_spins(const spo_system *s) { return (s && s->have_geom) ? s->N : SPO_ERR_STATE; }

static void decode(const spo_system *s, int i, int *b, int c[3])
{
    *b = i % s->nb;
    int r = i / s->nb;
    c[0] = r % s->nc[0]; r /= s->nc[0];
    c[1] = r % s->nc[1];
    c[2] = r / s->nc[1];
}

static int encode(const spo_system *s, int b, const int c[3])
{
    return b + s->nb * (c[0] + s->nc[0] * (c[1] + s->nc[1] * c[2]));
}

/* Spin index of basis atom jb in cell c + d, or -1 across an open edge. */
static int neighbour(const spo_system *s, const int c[3], const int d[3], int jb)
{
    int cj[3];
    for (int k = 0; k < 3; ++k) {
        int x = c[k] + d[k];
        if (s->per[k]) {
            x %= s->nc[k];
            if (x < 0) x += s->nc[k];
        } else if (x < 0 || x >= s->nc[k]) {
            return -1;
        }
        cj[k] = x;
    }
    return encode(s, jb, cj);
}

/* r = a * sum_k (x_k) A_k with x in lattice (fractional) coordinates */
static void lattice_to_cart(const spo_system *s, const double x[3], double r[3])
{
    for (int l = 0; l < 3; ++l)
        r[l] = s->a * (x[0] * s->A[0][l] + x[1] * s->A[1][l] + x[2] * s->A[2][l]);
}

int spo_positions(const spo_system *s, double *r)
{
    if (!s || !s->have_geom || !r) return SPO_ERR_STATE;
    for (int i = 0; i < s->N; ++i) {
        int b, c[3];
        decode(s, i, &b, c);
        double x[3] = {c[0] + s->basis[b][0], c[1] + s->basis[b][1], c[2] + s->basis[b][2]};
        lattice_to_cart(s, x, r + 3 * i);
    }
    return SPO_OK;
}

/* Bond vector from basis atom b in cell 0 to basis atom jb in cell d. */
static void bond_vector(const spo_system *s, int b, int jb, const int d[3], double r[3])
{
    double x[3];
    for (int k = 0; k < 3; ++k) x[k] = d[k] + s->basis[jb][k] - s->basis[b][k];
    lattice_to_cart(s, x, r);
}

static int cmp_double(const void *x, const void *y)
{
    double a = *(const double *)x, b = *(const double *)y;
    return (a > b) - (a < b);
}

static int add_nbr(spo_system *s, int b, int jb, const int d[3], double J, const double D[3])
{
    nbr_t *p = (nbr_t *)realloc(s->nbr[b], (size_t)(s->n_nbr[b] + 1) * sizeof(nbr_t));
    if (!p) return SPO_ERR_STATE;
    s->nbr[b] = p;
    nbr_t *e = &p[s->n_nbr[b]++];
    e->jb = jb;
    for (int k = 0; k < 3; ++k) { e->d[k] = d[k]; e->D[k] = D[k]; }
    e->J = J;
    return SPO_OK;
}

/*
 * Neighbour shells (Eq. 1 and its text: "unique pairs", any number of
 * shells).  Brute force: every atom of a box of cells around each basis atom
 * is a candidate; the distinct bond lengths, sorted, are the shells.  Each
 * unique pair <ij> appears twice in the directed list (once from each side),
 * with D_ji = -D_ij, so that sum_i sum_{j in nbr(i)} counts every pair twice.
 * DMI vectors (readings): bulk D_ij = D rhat_ij; interfacial
 * D_ij = D (z x rhat_ij).
 */
int spo_set_hamiltonian(spo_system *s, const spo_hamiltonian *h)
{
    if (!s || !s->have_geom || !h) return SPO_ERR_STATE;
    if (h->n_shells < 0 || h->n_shells > SPO_MAX_SHELLS) return SPO_ERR_ARG;
    if (h->n_dmi_shells < 0 || h->n_dmi_shells > SPO_MAX_SHELLS) return SPO_ERR_ARG;
    if (h->dmi_kind < SPO_DMI_NONE || h->dmi_kind > SPO_DMI_INTERFACIAL) return SPO_ERR_ARG;
    if (h->dipole < SPO_DIPOLE_NONE || h->dipole > SPO_DIPOLE_FFT) return SPO_ERR_ARG;
    if (h->n_gauss < 0 || h->n_gauss > SPO_MAX_GAUSS) return SPO_ERR_ARG;
    if (h->n_pairs < 0 || (h->n_pairs > 0 && !h->pairs)) return SPO_ERR_ARG;
    if (h->dipole != SPO_DIPOLE_NONE)
        for (int k = 0; k < 3; ++k)
            if (s->per[k] && s->nc[k] > 1) return SPO_ERR_UNSUPPORTED;

    free_nbr(s);
    s->h = *h;
    s->h.pairs = NULL;
    for (int b = 0; b < s->nb; ++b) normalise3(s->h.Khat[b]);

    int n_sh = h->n_shells;
    int n_dm = h->dmi_kind == SPO_DMI_NONE ? 0 : h->n_dmi_shells;
    int n_need = n_sh > n_dm ? n_sh : n_dm;
    s->n_shell_r = 0;
    if (n_need > 0) {
        int R[3];
        for (int k = 0; k < 3; ++k) R[k] = s->nc[k] > 1 ? n_need + 3 : 0;
        /* every candidate bond length, sorted; the distinct values are the shells */
        double tol = 1e-8 * s->a;
        long n_cand = 0, cap = 1024;
        double *all = (double *)malloc(sizeof(double) * cap);
        if (!all) return SPO_ERR_STATE;
        for (int b = 0; b < s->nb; ++b)
            for (int jb = 0; jb < s->nb; ++jb)
                for (int d0 = -R[0]; d0 <= R[0]; ++d0)
                    for (int d1 = -R[1]; d1 <= R[1]; ++d1)
                        for (int d2 = -R[2]; d2 <= R[2]; ++d2) {
                            int d[3] = {d0, d1, d2};
                            double r[3];
                            bond_vector(s, b, jb, d, r);
                            double l = sqrt(dot3(r, r));
                            if (l < tol) continue;
                            if (n_cand == cap) {
                                cap *= 2;
                                double *t = (double *)realloc(all, sizeof(double) * cap);
                                if (!t) { free(all); return SPO_ERR_STATE; }
                                all = t;
                            }
                            all[n_cand++] = l;
                        }
        qsort(all, (size_t)n_cand, sizeof(double), cmp_double);
        int nd = 0;
        double dist[SPO_MAX_SHELLS];
        for (long q = 0; q < n_cand && nd < n_need; ++q)
            if (nd == 0 || all[q] - dist[nd - 1] > tol) dist[nd++] = all[q];
        free(all);
        s->n_shell_r = nd;
        for (int q = 0; q < nd; ++q) s->shell_r[q] = dist[q];

        for (int b = 0; b < s->nb; ++b)
            for (int jb = 0; jb < s->nb; ++jb)
                for (int d0 = -R[0]; d0 <= R[0]; ++d0)
                    for (int d1 = -R[1]; d1 <= R[1]; ++d1)
                        for (int d2 = -R[2]; d2 <= R[2]; ++d2) {
                            int d[3] = {d0, d1, d2};
                            double r[3];
                            bond_vector(s, b, jb, d, r);
                            double l = sqrt(dot3(r, r));
                            if (l < tol) continue;
                            int sh = -1;
                            for (int q = 0; q < nd; ++q)
                                if (fabs(dist[q] - l) < tol) sh = q;
                            if (sh < 0) continue;
                            double J = sh < n_sh ? h->J[sh] : 0.0;
                            double D[3] = {0, 0, 0};
                            if (sh < n_dm) {
                                double rh[3] = {r[0] / l, r[1] / l, r[2] / l};
                                if (h->dmi_kind == SPO_DMI_BULK) {
                                    for (int k = 0; k < 3; ++k) D[k] = h->D[sh] * rh[k];
                                } else {
                                    double z[3] = {0, 0, 1};
                                    cross3(z, rh, D);
                                    for (int k = 0; k < 3; ++k) D[k] *= h->D[sh];
                                }
                            }
                            int rc = add_nbr(s, b, jb, d, J, D);
                            if (rc) return rc;
                        }
    }
    for (int p = 0; p < h->n_pairs; ++p) {
        const spo_pair *q = &h->pairs[p];
        if (q->i < 0 || q->i >= s->nb || q->j < 0 || q->j >= s->nb) return SPO_ERR_ARG;
        if (q->i == q->j && q->d[0] == 0 && q->d[1] == 0 && q->d[2] == 0) return SPO_ERR_ARG;
        int md[3] = {-q->d[0], -q->d[1], -q->d[2]};
        double mD[3] = {-q->D[0], -q->D[1], -q->D[2]};
        int rc = add_nbr(s, q->i, q->j, q->d, q->J, q->D);
        if (!rc) rc = add_nbr(s, q->j, q->i, md, q->J, mD);
        if (rc) return rc;
    }
    for (int g = 0; g < h->n_gauss; ++g) normalise3(&s->h.gauss[g][2]);
    s->have_ham = 1;
    return SPO_OK;
}

int spo_n_neighbours(const spo_system *s, int basis)
{
    if (!s || !s->have_ham || basis < 0 || basis >= s->nb) return SPO_ERR_STATE;
    return s->n_nbr[basis];
}

int spo_shell_radius(const spo_system *s, int shell, double *radius)
{
    if (!s || !s->have_ham || shell < 0 || shell >= s->n_shell_r || !radius) return SPO_ERR_ARG;
    *radius = s->shell_r[shell];
    return SPO_OK;
}

/* ------------------------------------------------------------------ */
/* Eq. 1: local part of B_eff = -dH/dn                                 */
/* ------------------------------------------------------------------ */
/* Appendix G landscape: energy and -gradient of one spin. */
static double gauss_terms(const spo_system *s, const double *n, double *B)
{
    double E = 0;
    for (int g = 0; g < s->h.n_gauss; ++g) {
        const double *G = s->h.gauss[g];
        double a = G[0], sig = G[1];
        const double *c = &G[2];
        double u = 1.0 - dot3(n, c);
        double e = a * exp(-u * u / (2 * sig * sig));
        E += e;
        /* d/dn [a exp(-u^2/(2 s^2))] = e * (u / s^2) * c  (du/dn = -c) */
        if (B)
            for (int k = 0; k < 3; ++k) B[k] -= e * (u / (sig * sig)) * c[k];
    }
    return E;
}

static void field_local(const spo_system *s, const double *n, double *B)
{
    const spo_hamiltonian *h = &s->h;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int i = 0; i < s->N; ++i) {
        int b, c[3];
        decode(s, i, &b, c);
        const double *ni = n + 3 * i;
        double Bi[3];
        /* Zeeman: -mu_i B.n_i */
        for (int k = 0; k < 3; ++k) Bi[k] = s->mu[b] * MU_B * h->B[k];
        /* anisotropy: -K (Khat.n)^2 */
        double kn = dot3(h->Khat[b], ni);
        for (int k = 0; k < 3; ++k) Bi[k] += 2.0 * h->K[b] * kn * h->Khat[b][k];
        /* exchange and DMI over the directed neighbour list */
        for (int e = 0; e < s->n_nbr[b]; ++e) {
            const nbr_t *q = &s->nbr[b][e];
            int j = neighbour(s, c, q->d, q->jb);
            if (j < 0) continue;
            const double *nj = n + 3 * j;
            double nxd[3];
            cross3(nj, q->D, nxd); /* d/dn_i [D.(n_i x n_j)] = n_j x D */
            for (int k = 0; k < 3; ++k) Bi[k] += q->J * nj[k] + nxd[k];
        }
        gauss_terms(s, ni, Bi);
        for (int k = 0; k < 3; ++k) B[3 * i + k] = Bi[k];
    }
}

/* ------------------------------------------------------------------ */
/* Dipole-dipole (Eq. 1, last term), two independent evaluations       */
/* ------------------------------------------------------------------ */
/* Reading of the garbled dipole term: E = 1/2 C sum_{i!=j} mu_i mu_j
 * [n_i.n_j - 3 (n_i.rhat)(n_j.rhat)] / r^3, so
 * B_i = C mu_i sum_j mu_j (3 rhat (rhat.n_j) - n_j) / r^3. */
static void dipole_pair_field(const double r[3], const double *nj, double out[3])
{
    double l2 = dot3(r, r);
    double l = sqrt(l2);
    double rh[3] = {r[0] / l, r[1] / l, r[2] / l};
    double p = dot3(rh, nj);
    double il3 = 1.0 / (l2 * l);
    for (int k = 0; k < 3; ++k) out[k] = (3.0 * rh[k] * p - nj[k]) * il3;
}

static void dipole_direct_at(const spo_system *s, const double *n, int n_idx, const int *idx, double *B,
                             const double *pos)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int t = 0; t < n_idx; ++t) {
        int i = idx ? idx[t] : t;
        int bi = i % s->nb;
        double acc[3] = {0, 0, 0};
        for (int j = 0; j < s->N; ++j) {
            if (j == i) continue;
            int bj = j % s->nb;
            double r[3], f[3];
            for (int k = 0; k < 3; ++k) r[k] = pos[3 * j + k] - pos[3 * i + k];
            dipole_pair_field(r, n + 3 * j, f);
            for (int k = 0; k < 3; ++k) acc[k] += s->mu[bj] * f[k];
        }
        for (int k = 0; k < 3; ++k) B[3 * t + k] = C_DIP * s->mu[bi] * acc[k];
    }
}

/* In-place radix-2 Cooley-Tukey FFT of a strided complex sequence of
 * power-of-two length n; sign -1 forward, +1 inverse (unnormalised). */
static void fft1d(double *re, double *im, int n, long stride, int sign)
{
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i * stride]; re[i * stride] = re[j * stride]; re[j * stride] = t;
            t = im[i * stride]; im[i * stride] = im[j * stride]; im[j * stride] = t;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        for (int k = 0; k < len / 2; ++k) {
            double ang = sign * 2.0 * M_PI * k / len;
            double wr = cos(ang), wi = sin(ang);
            for (int i0 = 0; i0 < n; i0 += len) {
                long u = (long)(i0 + k) * stride, v = (long)(i0 + k + len / 2) * stride;
                double xr = re[v] * wr - im[v] * wi;
                double xi = re[v] * wi + im[v] * wr;
                re[v] = re[u] - xr; im[v] = im[u] - xi;
                re[u] += xr; im[u] += xi;
            }
        }
    }
}

static void fft3d(double *re, double *im, const int P[3], int sign)
{
    long s0 = 1, s1 = P[0], s2 = (long)P[0] * P[1];
    if (P[0] > 1)
        for (long z = 0; z < P[2]; ++z)
            for (long y = 0; y < P[1]; ++y) fft1d(re + y * s1 + z * s2, im + y * s1 + z * s2, P[0], s0, sign);
    if (P[1] > 1)
        for (long z = 0; z < P[2]; ++z)
            for (long x = 0; x < P[0]; ++x) fft1d(re + x + z * s2, im + x + z * s2, P[1], s1, sign);
    if (P[2] > 1)
        for (long y = 0; y < P[1]; ++y)
            for (long x = 0; x < P[0]; ++x) fft1d(re + x + y * s1, im + x + y * s1, P[2], s2, sign);
}

static int next_pow2(int x)
{
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

/*
 * Zero-padded FFT convolution (Sec. "Dipolar interactions"): one FFT per
 * sublattice of the moments mu_b n, one kernel transform per sublattice pair,
 * and the field of sublattice b is IFFT(sum_b' Nhat_bb' . Mhat_b').  The grid
 * is padded to the smallest power of two >= 2 n_k - 1 per open direction, so
 * the circular convolution equals the linear one exactly.
 */
static int dipole_fft(const spo_system *s, const double *n, double *B)
{
    int P[3];
    for (int k = 0; k < 3; ++k) P[k] = s->nc[k] > 1 ? next_pow2(2 * s->nc[k] - 1) : 1;
    long M = (long)P[0] * P[1] * P[2];
    int nb = s->nb;
    double *mre = (double *)calloc((size_t)(3 * nb) * M, sizeof(double));
    double *mim = (double *)calloc((size_t)(3 * nb) * M, sizeof(double));
    double *kre = (double *)malloc((size_t)6 * M * sizeof(double));
    double *kim = (double *)malloc((size_t)6 * M * sizeof(double));
    double *bre = (double *)malloc((size_t)3 * M * sizeof(double));
    double *bim = (double *)malloc((size_t)3 * M * sizeof(double));
    if (!mre || !mim || !kre || !kim || !bre || !bim) {
        free(mre); free(mim); free(kre); free(kim); free(bre); free(bim);
        return SPO_ERR_STATE;
    }
    /* moments of each sublattice on the padded grid, then their transforms */
    for (int i = 0; i < s->N; ++i) {
        int b, c[3];
        decode(s, i, &b, c);
        long g = c[0] + (long)P[0] * (c[1] + (long)P[1] * c[2]);
        for (int k = 0; k < 3; ++k) mre[(3 * b + k) * M + g] = s->mu[b] * n[3 * i + k];
    }
    for (int q = 0; q < 3 * nb; ++q) fft3d(mre + q * M, mim + q * M, P, -1);

    for (int b = 0; b < nb; ++b) {
        memset(bre, 0, (size_t)3 * M * sizeof(double));
        memset(bim, 0, (size_t)3 * M * sizeof(double));
        for (int jb = 0; jb < nb; ++jb) {
            /* kernel G(g) = N(r(-g)), r(D) = bond from (b, 0) to (jb, D) */
            memset(kim, 0, (size_t)6 * M * sizeof(double));
            for (long g = 0; g < M; ++g) {
                int gi[3] = {(int)(g % P[0]), (int)((g / P[0]) % P[1]), (int)(g / ((long)P[0] * P[1]))};
                int d[3], ok = 1;
                for (int k = 0; k < 3; ++k) {
                    int x = gi[k] < P[k] - gi[k] ? gi[k] : gi[k] - P[k]; /* signed offset */
                    if (x > s->nc[k] - 1 || x < -(s->nc[k] - 1)) ok = 0;
                    d[k] = -x;
                }
                for (int c6 = 0; c6 < 6; ++c6) kre[c6 * M + g] = 0;
                if (!ok) continue;
                if (jb == b && d[0] == 0 && d[1] == 0 && d[2] == 0) continue;
                double r[3];
                bond_vector(s, b, jb, d, r);
                double l2 = dot3(r, r), l = sqrt(l2), il3 = 1.0 / (l2 * l);
                double rh[3] = {r[0] / l, r[1] / l, r[2] / l};
                /* symmetric tensor (3 rhat rhat^T - I)/r^3: xx xy xz yy yz zz */
                kre[0 * M + g] = (3 * rh[0] * rh[0] - 1) * il3;
                kre[1 * M + g] = 3 * rh[0] * rh[1] * il3;
                kre[2 * M + g] = 3 * rh[0] * rh[2] * il3;
                kre[3 * M + g] = (3 * rh[1] * rh[1] - 1) * il3;
                kre[4 * M + g] = 3 * rh[1] * rh[2] * il3;
                kre[5 * M + g] = (3 * rh[2] * rh[2] - 1) * il3;
            }
            for (int c6 = 0; c6 < 6; ++c6) fft3d(kre + c6 * M, kim + c6 * M, P, -1);
            static const int idx6[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
            for (long g = 0; g < M; ++g)
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) {
                        int t = idx6[k][l];
                        double ar = kre[t * M + g], ai = kim[t * M + g];
                        double xr = mre[(3 * jb + l) * M + g], xi = mim[(3 * jb + l) * M + g];
                        bre[k * M + g] += ar * xr - ai * xi;
                        bim[k * M + g] += ar * xi + ai * xr;
                    }
        }
        for (int k = 0; k < 3; ++k) fft3d(bre + k * M, bim + k * M, P, +1);
        for (int i = 0; i < s->N; ++i) {
            int bi, c[3];
            decode(s, i, &bi, c);
            if (bi != b) continue;
            long g = c[0] + (long)P[0] * (c[1] + (long)P[1] * c[2]);
            for (int k = 0; k < 3; ++k) B[3 * i + k] = C_DIP * s->mu[b] * bre[k * M + g] / (double)M;
        }
    }
    free(mre); free(mim); free(kre); free(kim); free(bre); free(bim);
    return SPO_OK;
}

int spo_dipole_field(const spo_system *s, const double *n, double *B, int dipole_method)
{
    if (!s || !s->have_ham || !n || !B) return SPO_ERR_STATE;
    int m = dipole_method >= 0 ? dipole_method : s->h.dipole;
    if (m == SPO_DIPOLE_NONE) {
        memset(B, 0, sizeof(double) * 3 * (size_t)s->N);
        return SPO_OK;
    }
    for (int k = 0; k < 3; ++k)
        if (s->per[k] && s->nc[k] > 1) return SPO_ERR_UNSUPPORTED;
    if (m == SPO_DIPOLE_FFT) return dipole_fft(s, n, B);
    if (m != SPO_DIPOLE_DIRECT) return SPO_ERR_ARG;
    double *pos = (double *)malloc(sizeof(double) * 3 * (size_t)s->N);
    if (!pos) return SPO_ERR_STATE;
    spo_positions(s, pos);
    dipole_direct_at(s, n, s->N, NULL, B, pos);
    free(pos);
    return SPO_OK;
}

int spo_dipole_field_direct_at(const spo_system *s, const double *n, int n_idx, const int *idx, double *B)
{
    if (!s || !s->have_ham || !n || !B || !idx || n_idx < 0) return SPO_ERR_STATE;
    for (int t = 0; t < n_idx; ++t)
        if (idx[t] < 0 || idx[t] >= s->N) return SPO_ERR_ARG;
    double *pos = (double *)malloc(sizeof(double) * 3 * (size_t)s->N);
    if (!pos) return SPO_ERR_STATE;
    spo_positions(s, pos);
    dipole_direct_at(s, n, n_idx, idx, B, pos);
    free(pos);
    return SPO_OK;
}

int spo_effective_field(const spo_system *s, const double *n, double *B, int dipole_method)
{
    if (!s || !s->have_ham || !n || !B) return SPO_ERR_STATE;
    field_local(s, n, B);
    int m = dipole_method >= 0 ? dipole_method : s->h.dipole;
    if (m == SPO_DIPOLE_NONE) return SPO_OK;
    double *Bd = (double *)malloc(sizeof(double) * 3 * (size_t)s->N);
    if (!Bd) return SPO_ERR_STATE;
    int rc = spo_dipole_field(s, n, Bd, m);
    if (!rc)
        for (long q = 0; q < 3L * s->N; ++q) B[q] += Bd[q];
    free(Bd);
    return rc;
}

/* Eq. 1 term by term, each as a sum over its own definition. */
int spo_energy(const spo_system *s, const double *n, double *e)
{
    if (!s || !s->have_ham || !n || !e) return SPO_ERR_STATE;
    const spo_hamiltonian *h = &s->h;
    double ez = 0, ea = 0, ex = 0, ed = 0, eg = 0;
    for (int i = 0; i < s->N; ++i) {
        int b, c[3];
        decode(s, i, &b, c);
        const double *ni = n + 3 * i;
        ez -= s->mu[b] * MU_B * dot3(h->B, ni);
        double kn = dot3(h->Khat[b], ni);
        ea -= h->K[b] * kn * kn;
        for (int q = 0; q < s->n_nbr[b]; ++q) {
            const nbr_t *p = &s->nbr[b][q];
            int j = neighbour(s, c, p->d, p->jb);
            if (j < 0) continue;
            const double *nj = n + 3 * j;
            double x[3];
            cross3(ni, nj, x);
            /* each unique pair is met twice in the directed list */
            ex -= 0.5 * p->J * dot3(ni, nj);
            ed -= 0.5 * dot3(p->D, x);
        }
        eg += gauss_terms(s, ni, NULL);
    }
    double edd = 0;
    if (h->dipole == SPO_DIPOLE_DIRECT) {
        double *pos = (double *)malloc(sizeof(double) * 3 * (size_t)s->N);
        if (!pos) return SPO_ERR_STATE;
        spo_positions(s, pos);
        for (int i = 0; i < s->N; ++i)
            for (int j = 0; j < s->N; ++j) {
                if (i == j) continue;
                double r[3];
                for (int k = 0; k < 3; ++k) r[k] = pos[3 * j + k] - pos[3 * i + k];
                double l2 = dot3(r, r), l = sqrt(l2);
                double rh[3] = {r[0] / l, r[1] / l, r[2] / l};
                const double *ni = n + 3 * i, *nj = n + 3 * j;
                edd += 0.5 * C_DIP * s->mu[i % s->nb] * s->mu[j % s->nb] *
                       (dot3(ni, nj) - 3.0 * dot3(ni, rh) * dot3(nj, rh)) / (l2 * l);
            }
        free(pos);
    } else if (h->dipole == SPO_DIPOLE_FFT) {
        double *Bd = (double *)malloc(sizeof(double) * 3 * (size_t)s->N);
        if (!Bd) return SPO_ERR_STATE;
        int rc = dipole_fft(s, n, Bd);
        if (rc) { free(Bd); return rc; }
        for (int i = 0; i < s->N; ++i) edd -= 0.5 * dot3(n + 3 * i, Bd + 3 * i);
        free(Bd);
    }
    e[1] = ez; e[2] = ea; e[3] = ex; e[4] = ed; e[5] = edd;
    e[0] = ez + ea + ex + ed + edd + eg;
    return SPO_OK;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller     */
/* ------------------------------------------------------------------ */
void spo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Reading of the unspecified random source: key = seed, counter = (spin
 * index, step low word, step high word, 8*replica + 0); uniforms
 * u = (x + 1/2) 2^-32; Box-Muller on (u0,u1) gives eta_x, eta_y and on
 * (u2,u3) gives eta_z. */
void spo_thermal_normals(uint64_t seed, uint64_t step, uint32_t replica, uint32_t i, double eta[3])
{
    uint32_t ctr[4] = {i, (uint32_t)step, (uint32_t)(step >> 32), replica * 8u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    spo_philox4x32_10(ctr, key, x);
    double u[4];
    for (int k = 0; k < 4; ++k) u[k] = ((double)x[k] + 0.5) / 4294967296.0;
    double r0 = sqrt(-2.0 * log(u[0])), r1 = sqrt(-2.0 * log(u[2]));
    eta[0] = r0 * cos(2.0 * M_PI * u[1]);
    eta[1] = r0 * sin(2.0 * M_PI * u[1]);
    eta[2] = r1 * cos(2.0 * M_PI * u[3]);
}

/* ------------------------------------------------------------------ */
/* LLG (Eq. 3) in the form dn/dt = n x A (Appendix B)                   */
/* ------------------------------------------------------------------ */
/* A_i = -gamma / ((1 + alpha^2) mu_i) (B_i + alpha n_i x B_i), mu_i in meV/T */
static void llg_A(double mu_meV_T, double alpha, const double *n, const double *B, double *A)
{
    double nxb[3];
    cross3(n, B, nxb);
    double f = -GAMMA_E / ((1.0 + alpha * alpha) * mu_meV_T);
    for (int k = 0; k < 3; ++k) A[k] = f * (B[k] + alpha * nxb[k]);
}

/* Depondt rotation: dn/dt = n x A = (-A) x n, i.e. rotation about -Ahat by
 * the angle |A| dt (Rodrigues' formula). */
static void rotate(const double *n, const double *A, double dt, double *out)
{
    double w = sqrt(dot3(A, A));
    if (w == 0.0) { out[0] = n[0]; out[1] = n[1]; out[2] = n[2]; return; }
    double ax[3] = {-A[0] / w, -A[1] / w, -A[2] / w};
    double th = w * dt, ct = cos(th), st = sin(th);
    double axn[3];
    cross3(ax, n, axn);
    double an = dot3(ax, n);
    for (int k = 0; k < 3; ++k) out[k] = n[k] * ct + axn[k] * st + ax[k] * an * (1.0 - ct);
}

static double det3(const double m[3][3])
{
    return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
           m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
}

/* Appendix C: the implicit-midpoint update x = n + dt (n + x)/2 x A, written
 * as M x = M^T n with M = I + skew(a), a = dt A / 2 (reading: the matrix of
 * Appendix C carries the factor dt/2 of the midpoint rule), solved by
 * Cramer's rule x_k = det(M^k) / det(M), M^k = M with column k replaced by
 * the right-hand side M^T n = n + n x a. */
static void sib_solve(const double *n, const double *A, double dt, double *x)
{
    double a[3] = {0.5 * dt * A[0], 0.5 * dt * A[1], 0.5 * dt * A[2]};
    double M[3][3] = {{1.0, -a[2], a[1]}, {a[2], 1.0, -a[0]}, {-a[1], a[0], 1.0}};
    double nxa[3];
    cross3(n, a, nxa);
    double rhs[3] = {n[0] + nxa[0], n[1] + nxa[1], n[2] + nxa[2]};
    double d = det3(M);
    for (int k = 0; k < 3; ++k) {
        double Mk[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) Mk[r][c] = (c == k) ? rhs[r] : M[r][c];
        x[k] = det3(Mk) / d;
    }
}

/* Fourth-order Runge-Kutta (named in Sec. LLG) for dn/dt = n x A(n, B(n) + B_th)
 * with the same thermal field in all four stages, the result renormalised. */
static int rk4_step(const spo_system *s, double *n, const spo_llg_params *p, const double *Bth)
{
    size_t sz = sizeof(double) * 3 * (size_t)s->N;
    double *y = (double *)malloc(sz), *B = (double *)malloc(sz), *acc = (double *)malloc(sz);
    if (!y || !B || !acc) { free(y); free(B); free(acc); return SPO_ERR_STATE; }
    static const double cy[4] = {0.5, 0.5, 1.0, 0.0}; /* next stage state: n + cy*dt*k */
    static const double w[4] = {1.0, 2.0, 2.0, 1.0};
    memcpy(y, n, sz);
    memset(acc, 0, sz);
    int rc = SPO_OK;
    for (int st = 0; st < 4 && !rc; ++st) {
        rc = spo_effective_field(s, y, B, -1);
        if (rc) break;
        for (int i = 0; i < s->N; ++i) {
            double mu = s->mu[i % s->nb] * MU_B, Bi[3], A[3], k[3];
            for (int c = 0; c < 3; ++c) Bi[c] = B[3 * i + c] + Bth[3 * i + c];
            llg_A(mu, p->alpha, y + 3 * i, Bi, A);
            cross3(y + 3 * i, A, k);
            for (int c = 0; c < 3; ++c) acc[3 * i + c] += w[st] * k[c];
            if (st < 3)
                for (int c = 0; c < 3; ++c) y[3 * i + c] = n[3 * i + c] + cy[st] * p->dt * k[c];
        }
    }
    if (!rc)
        for (int i = 0; i < s->N; ++i) {
            for (int c = 0; c < 3; ++c) n[3 * i + c] += p->dt / 6.0 * acc[3 * i + c];
            normalise3(n + 3 * i);
        }
    free(y); free(B); free(acc);
    return rc;
}

int spo_llg(const spo_system *s, double *n, const spo_llg_params *p, int n_steps)
{
    if (!s || !s->have_ham || !n || !p) return SPO_ERR_STATE;
    if (p->solver < SPO_DEPONDT || p->solver > SPO_RK4) return SPO_ERR_ARG;
    if (!(p->dt > 0) || p->alpha < 0 || p->T < 0 || n_steps < 0) return SPO_ERR_ARG;
    size_t sz = sizeof(double) * 3 * (size_t)s->N;
    double *B = (double *)malloc(sz), *np = (double *)malloc(sz), *A = (double *)malloc(sz),
           *Bth = (double *)malloc(sz);
    if (!B || !np || !A || !Bth) { free(B); free(np); free(A); free(Bth); return SPO_ERR_STATE; }
    int rc = SPO_OK;
    for (int st = 0; st < n_steps && !rc; ++st) {
        uint64_t step = p->step0 + (uint64_t)st;
        /* thermal field (Eq. 4): sqrt(2 alpha kB T mu_i / (gamma dt)) eta_i,
         * the same eta in both stages of the step */
        for (int i = 0; i < s->N; ++i) {
            double eta[3] = {0, 0, 0};
            double mu = s->mu[i % s->nb] * MU_B;
            double sig = sqrt(2.0 * p->alpha * K_B * p->T * mu / (GAMMA_E * p->dt));
            if (p->T > 0) spo_thermal_normals(p->seed, step, p->replica, (uint32_t)i, eta);
            for (int k = 0; k < 3; ++k) Bth[3 * i + k] = sig * eta[k];
        }
        if (p->solver == SPO_RK4) {
            rc = rk4_step(s, n, p, Bth);
            continue;
        }
        rc = spo_effective_field(s, n, B, -1);
        if (rc) break;
        for (int i = 0; i < s->N; ++i) {
            double mu = s->mu[i % s->nb] * MU_B, Bi[3];
            for (int k = 0; k < 3; ++k) Bi[k] = B[3 * i + k] + Bth[3 * i + k];
            llg_A(mu, p->alpha, n + 3 * i, Bi, A + 3 * i);
            if (p->solver == SPO_SIB) {
                /* predictor (Appendix C): implicit midpoint with A(n);
                 * np holds the midpoint (n + n^p)/2 for the corrector */
                double x[3];
                sib_solve(n + 3 * i, A + 3 * i, p->dt, x);
                for (int k = 0; k < 3; ++k) np[3 * i + k] = 0.5 * (n[3 * i + k] + x[k]);
            } else if (p->solver == SPO_DEPONDT) {
                rotate(n + 3 * i, A + 3 * i, p->dt, np + 3 * i);
            } else {
                double f[3];
                cross3(n + 3 * i, A + 3 * i, f);
                for (int k = 0; k < 3; ++k) np[3 * i + k] = n[3 * i + k] + p->dt * f[k];
                normalise3(np + 3 * i); /* reading: renormalise every stage */
            }
        }
        rc = spo_effective_field(s, np, B, -1);
        if (rc) break;
        for (int i = 0; i < s->N; ++i) {
            double mu = s->mu[i % s->nb] * MU_B, Bi[3], Ap[3];
            for (int k = 0; k < 3; ++k) Bi[k] = B[3 * i + k] + Bth[3 * i + k];
            llg_A(mu, p->alpha, np + 3 * i, Bi, Ap);
            if (p->solver == SPO_SIB) {
                /* corrector: implicit midpoint with A at the midpoint state */
                double x[3];
                sib_solve(n + 3 * i, Ap, p->dt, x);
                for (int k = 0; k < 3; ++k) n[3 * i + k] = x[k];
            } else if (p->solver == SPO_DEPONDT) {
                double Ac[3];
                for (int k = 0; k < 3; ++k) Ac[k] = 0.5 * (A[3 * i + k] + Ap[k]);
                double out[3];
                rotate(n + 3 * i, Ac, p->dt, out);
                for (int k = 0; k < 3; ++k) n[3 * i + k] = out[k];
            } else {
                double f[3], fp[3];
                cross3(n + 3 * i, A + 3 * i, f);
                cross3(np + 3 * i, Ap, fp);
                for (int k = 0; k < 3; ++k) n[3 * i + k] += 0.5 * p->dt * (f[k] + fp[k]);
                normalise3(n + 3 * i);
            }
        }
    }
    free(B); free(np); free(A); free(Bth);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Velocity projection (Appendix D)                                     */
/* ------------------------------------------------------------------ */
/* Reading: the force is the projected effective field, F_i = B_i - (B_i.n_i) n_i
 * (the tangent-space part of -dH/dn_i), so |F_i| = |n_i x B_i|. */
static int projected_force(const spo_system *s, const double *n, double *F)
{
    int rc = spo_effective_field(s, n, F, -1);
    if (rc) return rc;
    for (int i = 0; i < s->N; ++i) {
        double bn = dot3(F + 3 * i, n + 3 * i);
        for (int k = 0; k < 3; ++k) F[3 * i + k] -= bn * n[3 * i + k];
    }
    return SPO_OK;
}

static double max_norm3(const double *x, long count)
{
    double m = 0;
    for (long i = 0; i < count; ++i) {
        double v = sqrt(dot3(x + 3 * i, x + 3 * i));
        if (v > m) m = v;
    }
    return m;
}

int spo_minimise(const spo_system *s, double *n, double *v, double dt, double mass, double tol,
                 int max_iter, int *iters, double *max_torque)
{
    if (!s || !s->have_ham || !n || !v) return SPO_ERR_STATE;
    if (!(dt > 0) || !(mass > 0) || max_iter < 0) return SPO_ERR_ARG;
    size_t sz = sizeof(double) * 3 * (size_t)s->N;
    double *F = (double *)malloc(sz), *Fn = (double *)malloc(sz);
    if (!F || !Fn) { free(F); free(Fn); return SPO_ERR_STATE; }
    int rc = projected_force(s, n, F);
    int it = 0;
    double m = max_norm3(F, s->N);
    while (!rc && it < max_iter && !(m < tol)) {
        /* x(t+dt) = x + dt v + dt^2/(2m) F, renormalised */
        for (int i = 0; i < s->N; ++i) {
            for (int k = 0; k < 3; ++k)
                n[3 * i + k] += dt * v[3 * i + k] + dt * dt / (2.0 * mass) * F[3 * i + k];
            normalise3(n + 3 * i);
        }
        rc = projected_force(s, n, Fn);
        if (rc) break;
        /* v(t+dt) = v + dt/(2m) (F + F'), then projection on F' */
        double vf = 0, ff = 0;
        for (long q = 0; q < 3L * s->N; ++q) {
            v[q] += dt / (2.0 * mass) * (F[q] + Fn[q]);
            vf += v[q] * Fn[q];
            ff += Fn[q] * Fn[q];
        }
        for (long q = 0; q < 3L * s->N; ++q) v[q] = (vf > 0 && ff > 0) ? vf / ff * Fn[q] : 0.0;
        memcpy(F, Fn, sz);
        m = max_norm3(F, s->N);
        ++it;
    }
    if (iters) *iters = it;
    if (max_torque) *max_torque = m;
    free(F); free(Fn);
    return rc;
}

/* ------------------------------------------------------------------ */
/* GNEB (Sec. GNEB, Appendix F)                                         */
/* ------------------------------------------------------------------ */
/* Reading: geodesic distance l = sqrt(sum_i theta_i^2), theta_i the
 * great-circle angle between the two images' spins i. */
static double geodesic(long N, const double *x, const double *y)
{
    double acc = 0;
    for (long i = 0; i < N; ++i) {
        double c[3];
        cross3(x + 3 * i, y + 3 * i, c);
        double th = atan2(sqrt(dot3(c, c)), dot3(x + 3 * i, y + 3 * i));
        acc += th * th;
    }
    return sqrt(acc);
}

/* Cubic Hermite interpolant of E on [0, h] with values Ea, Eb and slopes da,
 * db at the ends: value and derivative at s. */
static void hermite(double Ea, double Eb, double da, double db, double h, double s, double *E, double *dE)
{
    double t = s / h;
    double h00 = 2 * t * t * t - 3 * t * t + 1, h10 = t * t * t - 2 * t * t + t;
    double h01 = -2 * t * t * t + 3 * t * t, h11 = t * t * t - t * t;
    *E = h00 * Ea + h10 * h * da + h01 * Eb + h11 * h * db;
    double g00 = 6 * t * t - 6 * t, g10 = 3 * t * t - 4 * t + 1, g01 = -6 * t * t + 6 * t, g11 = 3 * t * t - 2 * t;
    *dE = (g00 * Ea + g01 * Eb) / h + g10 * da + g11 * db;
}

/* Reading of the energy-weighted spring (Sec. GNEB: springs measured along
 * the cubic interpolation of the path energy, with a weight between energy
 * and reaction coordinate): the length of the segment of the curve
 * ((1-w) r, w E(r)) over the geodesic distance h, E(r) the cubic Hermite
 * interpolant; integrated by adaptive Simpson (Lyness' criterion |S2 - S1|
 * <= 15 eps, Richardson-corrected) to eps = 1e-13 h.  w = 0 gives h. */
typedef struct { double Ea, Eb, da, db, h, w; } seg_t;

static double seg_integrand(const seg_t *g, double s)
{
    double E, dE;
    hermite(g->Ea, g->Eb, g->da, g->db, g->h, s, &E, &dE);
    return sqrt((1 - g->w) * (1 - g->w) + g->w * g->w * dE * dE);
}

static double simpson_step(const seg_t *g, double a, double b, double fa, double fm, double fb, double whole,
                           double eps, int depth)
{
    double m = 0.5 * (a + b), lm = 0.5 * (a + m), rm = 0.5 * (m + b);
    double flm = seg_integrand(g, lm), frm = seg_integrand(g, rm);
    double left = (m - a) / 6 * (fa + 4 * flm + fm), right = (b - m) / 6 * (fm + 4 * frm + fb);
    double d = left + right - whole;
    if (depth <= 0 || fabs(d) <= 15 * eps) return left + right + d / 15;
    return simpson_step(g, a, m, fa, flm, fm, left, 0.5 * eps, depth - 1) +
           simpson_step(g, m, b, fm, frm, fb, right, 0.5 * eps, depth - 1);
}

double spo_segment_length(double Ea, double Eb, double da, double db, double h, double w)
{
    if (w == 0.0) return h;
    if (!(h > 0)) return 0.0;
    seg_t g = {Ea, Eb, da, db, h, w};
    double fa = seg_integrand(&g, 0), fm = seg_integrand(&g, 0.5 * h), fb = seg_integrand(&g, h);
    return simpson_step(&g, 0, h, fa, fm, fb, h / 6 * (fa + 4 * fm + fb), 1e-13 * h, 40);
}

/* Tangent of image v (improved tangent of Henkelman and Jonsson 2000 for
 * interior images; the one-sided difference to the neighbour at the
 * endpoints), projected per spin onto the tangent space of the image and
 * normalised in 3N dimensions. */
static void image_tangent(long N, const double *chain, int M, int v, const double *E, double *tau)
{
    size_t img = 3 * (size_t)N;
    const double *x = chain + v * img;
    if (v == 0 || v == M - 1) {
        const double *a = v == 0 ? x : chain + (v - 1) * img, *b = v == 0 ? chain + img : x;
        for (long q = 0; q < 3 * N; ++q) tau[q] = b[q] - a[q];
    } else {
        const double *xp = chain + (v + 1) * img, *xm = chain + (v - 1) * img;
        double Ep = E[v + 1], E0 = E[v], Em = E[v - 1];
        double wp, wm;
        if (Ep > E0 && E0 > Em) { wp = 1; wm = 0; }
        else if (Ep < E0 && E0 < Em) { wp = 0; wm = 1; }
        else {
            double dmax = fmax(fabs(Ep - E0), fabs(Em - E0));
            double dmin = fmin(fabs(Ep - E0), fabs(Em - E0));
            if (Ep > Em) { wp = dmax; wm = dmin; }
            else { wp = dmin; wm = dmax; }
        }
        for (long q = 0; q < 3 * N; ++q) tau[q] = wp * (xp[q] - x[q]) + wm * (x[q] - xm[q]);
    }
    /* project onto the tangent space of the image, then normalise in 3N dimensions */
    double tt = 0;
    for (long i = 0; i < N; ++i) {
        double tn = dot3(tau + 3 * i, x + 3 * i);
        for (int k = 0; k < 3; ++k) tau[3 * i + k] -= tn * x[3 * i + k];
        tt += dot3(tau + 3 * i, tau + 3 * i);
    }
    double tn = sqrt(tt);
    if (tn > 0)
        for (long q = 0; q < 3 * N; ++q) tau[q] /= tn;
}

/* Energies, fields, tangents, slopes dE/dr = Pg.tau and distances of a chain. */
static int chain_state(const spo_system *s, const double *chain, int M, double *E, double *B, double *tau,
                       double *slope, double *l)
{
    long N = s->N;
    size_t img = 3 * (size_t)N;
    int rc = SPO_OK;
    for (int v = 0; v < M && !rc; ++v) {
        double e[6];
        rc = spo_energy(s, chain + v * img, e);
        E[v] = e[0];
        if (!rc) rc = spo_effective_field(s, chain + v * img, B + v * img, -1);
    }
    if (rc) return rc;
    for (int v = 0; v + 1 < M; ++v) l[v] = geodesic(N, chain + v * img, chain + (v + 1) * img);
    for (int v = 0; v < M; ++v) {
        const double *x = chain + v * img;
        double *t = tau + v * img;
        image_tangent(N, chain, M, v, E, t);
        double gt = 0;
        for (long i = 0; i < N; ++i) {
            const double *b = B + v * img + 3 * i;
            double bn = dot3(b, x + 3 * i);
            for (int k = 0; k < 3; ++k) gt += -(b[k] - bn * x[3 * i + k]) * t[3 * i + k];
        }
        slope[v] = gt;
    }
    return SPO_OK;
}

int spo_gneb_forces(const spo_system *s, const double *chain, int M, const spo_gneb_params *p,
                    double *forces, double *energies, double *dist, int *ci_out)
{
    if (!s || !s->have_ham || !chain || !forces || !p || M < 2) return SPO_ERR_STATE;
    if (!(p->energy_weight >= 0 && p->energy_weight < 1)) return SPO_ERR_ARG;
    long N = s->N;
    size_t img = 3 * (size_t)N;
    double *E = energies ? energies : (double *)malloc(sizeof(double) * M);
    double *l = (double *)malloc(sizeof(double) * (M - 1));
    double *L = (double *)malloc(sizeof(double) * (M - 1));
    double *slope = (double *)malloc(sizeof(double) * M);
    double *B = (double *)malloc(sizeof(double) * img * M);
    double *tau = (double *)malloc(sizeof(double) * img * M);
    if (!E || !l || !L || !slope || !B || !tau) {
        if (!energies) free(E);
        free(l); free(L); free(slope); free(B); free(tau);
        return SPO_ERR_STATE;
    }
    int rc = chain_state(s, chain, M, E, B, tau, slope, l);
    for (int v = 0; v + 1 < M && !rc; ++v)
        L[v] = spo_segment_length(E[v], E[v + 1], slope[v], slope[v + 1], l[v], p->energy_weight);
    /* image kinds: explicit, or the highest interior image climbs */
    int ci = -1;
    if (!p->image_types && p->climbing && M > 2) {
        ci = 1;
        for (int v = 2; v < M - 1; ++v)
            if (E[v] > E[ci]) ci = v;
    }
    memset(forces, 0, sizeof(double) * img * M);
    for (int v = 1; v < M - 1 && !rc; ++v) {
        const double *x = chain + v * img, *t = tau + v * img;
        int kind = p->image_types ? p->image_types[v] : (v == ci ? SPO_IMAGE_CLIMBING : SPO_IMAGE_NORMAL);
        double *F = forces + v * img;
        double gt = slope[v];
        /* Reading of Eq. Spring_Force: F^S = k (L_{v,v+1} - L_{v-1,v}) tau */
        double fs = p->k_spring * (L[v] - L[v - 1]);
        for (long i = 0; i < N; ++i) {
            const double *b = B + v * img + 3 * i;
            double bn = dot3(b, x + 3 * i);
            for (int k = 0; k < 3; ++k) {
                long q = 3 * i + k;
                double pg = -(b[k] - bn * x[q]);
                if (kind == SPO_IMAGE_CLIMBING) F[q] = -pg + 2.0 * gt * t[q];
                else if (kind == SPO_IMAGE_FALLING) F[q] = -pg; /* no spring, full gradient: falls to a minimum */
                else F[q] = -pg + gt * t[q] + fs * t[q];
            }
        }
    }
    if (dist) memcpy(dist, l, sizeof(double) * (M - 1));
    if (ci_out) *ci_out = ci;
    if (!energies) free(E);
    free(l); free(L); free(slope); free(B); free(tau);
    return rc;
}

int spo_gneb_path(const spo_system *s, const double *chain, int M, int n_interp, double *r, double *E, double *slope,
                  double *Q, double *r_i, double *E_i)
{
    if (!s || !s->have_ham || !chain || M < 2 || n_interp < 1 || !r || !E || !slope) return SPO_ERR_ARG;
    long N = s->N;
    size_t img = 3 * (size_t)N;
    double *B = (double *)malloc(sizeof(double) * img * M);
    double *tau = (double *)malloc(sizeof(double) * img * M);
    double *l = (double *)malloc(sizeof(double) * (M - 1));
    if (!B || !tau || !l) { free(B); free(tau); free(l); return SPO_ERR_STATE; }
    int rc = chain_state(s, chain, M, E, B, tau, slope, l);
    if (!rc) {
        r[0] = 0;
        for (int v = 1; v < M; ++v) r[v] = r[v - 1] + l[v - 1];
        if (r_i && E_i) {
            for (int v = 0; v + 1 < M; ++v)
                for (int q = 0; q < n_interp; ++q) {
                    double sq = l[v] * q / n_interp, e, de;
                    hermite(E[v], E[v + 1], slope[v], slope[v + 1], l[v], sq, &e, &de);
                    r_i[v * n_interp + q] = r[v] + sq;
                    E_i[v * n_interp + q] = e;
                }
            r_i[(M - 1) * n_interp] = r[M - 1];
            E_i[(M - 1) * n_interp] = E[M - 1];
        }
        if (Q)
            for (int v = 0; v < M && !rc; ++v) rc = spo_topological_charge(s, chain + v * img, &Q[v]);
    }
    free(B); free(tau); free(l);
    return rc;
}

int spo_gneb(const spo_system *s, double *chain, double *vel, int M, const spo_gneb_params *p, int n_iter,
             double tol, double *energies, double *max_force, int *iters)
{
    if (!s || !s->have_ham || !chain || !vel || !p || M < 2 || n_iter < 0) return SPO_ERR_STATE;
    if (!(p->dt > 0) || !(p->mass > 0)) return SPO_ERR_ARG;
    long N = s->N;
    size_t img = 3 * (size_t)N;
    double *F = (double *)malloc(sizeof(double) * img * M);
    double *Fn = (double *)malloc(sizeof(double) * img * M);
    double *E = (double *)malloc(sizeof(double) * M);
    if (!F || !Fn || !E) { free(F); free(Fn); free(E); return SPO_ERR_STATE; }
    double dt = p->dt, m = p->mass;
    int rc = spo_gneb_forces(s, chain, M, p, F, E, NULL, NULL);
    double fmax_ = max_norm3(F + img, N * (M - 2));
    int it = 0;
    while (!rc && it < n_iter && !(tol > 0 && fmax_ < tol)) {
        for (int v = 1; v < M - 1; ++v)
            for (long i = 0; i < N; ++i) {
                double *x = chain + v * img + 3 * i;
                const double *vv = vel + v * img + 3 * i, *f = F + v * img + 3 * i;
                for (int k = 0; k < 3; ++k) x[k] += dt * vv[k] + dt * dt / (2.0 * m) * f[k];
                normalise3(x);
            }
        rc = spo_gneb_forces(s, chain, M, p, Fn, E, NULL, NULL);
        if (rc) break;
        /* velocity update and projection, per image */
        for (int v = 1; v < M - 1; ++v) {
            double *vv = vel + v * img;
            const double *f0 = F + v * img, *f1 = Fn + v * img;
            double vf = 0, ff = 0;
            for (long q = 0; q < 3 * N; ++q) {
                vv[q] += dt / (2.0 * m) * (f0[q] + f1[q]);
                vf += vv[q] * f1[q];
                ff += f1[q] * f1[q];
            }
            for (long q = 0; q < 3 * N; ++q) vv[q] = (vf > 0 && ff > 0) ? vf / ff * f1[q] : 0.0;
        }
        memcpy(F, Fn, sizeof(double) * img * M);
        fmax_ = max_norm3(F + img, N * (M - 2));
        ++it;
    }
    if (energies) memcpy(energies, E, sizeof(double) * M);
    if (max_force) *max_force = fmax_;
    if (iters) *iters = it;
    free(F); free(Fn); free(E);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Topological charge, Berg-Luescher (Appendix A)                       */
/* ------------------------------------------------------------------ */
/* Signed solid angle A_l of the spherical triangle (a, b, c) (Appendix A):
 * cos(A/2) = (1 + a.b + a.c + b.c) / sqrt(2 (1 + a.b)(1 + b.c)(1 + c.a)),
 * sign(A) = sign(a.(b x c)).  For unit vectors the same denominator gives
 * sin(A/2) = a.(b x c) / sqrt(...), so A is taken as 2 atan2(sin, cos):
 * the same angle and sign, without acos's loss of precision near A = 0. */
static double solid_angle(const double *a, const double *b, const double *c)
{
    double ab = dot3(a, b), bc = dot3(b, c), ca = dot3(c, a);
    double x[3];
    cross3(b, c, x);
    double trip = dot3(a, x);
    double den = sqrt(2.0 * (1.0 + ab) * (1.0 + bc) * (1.0 + ca));
    double cs = (1.0 + ab + ca + bc) / den;
    double sn = trip / den;
    return 2.0 * atan2(sn, cs);
}

int spo_topological_charge(const spo_system *s, const double *n, double *Q)
{
    if (!s || !s->have_geom || !n || !Q) return SPO_ERR_STATE;
    if (s->nb != 1 || s->nc[2] != 1) return SPO_ERR_UNSUPPORTED;
    double acc = 0;
    /* two elementary triangles per cell: (0,0)(1,0)(0,1) and (1,0)(1,1)(0,1) */
    static const int tri[2][3][2] = {{{0, 0}, {1, 0}, {0, 1}}, {{1, 0}, {1, 1}, {0, 1}}};
    double e1[3], e2[3];
    {
        double x1[3] = {1, 0, 0}, x2[3] = {0, 1, 0};
        lattice_to_cart(s, x1, e1);
        lattice_to_cart(s, x2, e2);
    }
    for (int c1 = 0; c1 < s->nc[1]; ++c1)
        for (int c0 = 0; c0 < s->nc[0]; ++c0)
            for (int t = 0; t < 2; ++t) {
                int idx[3], ok = 1;
                double p[3][2];
                for (int v = 0; v < 3; ++v) {
                    int c[3] = {c0, c1, 0};
                    int d[3] = {tri[t][v][0], tri[t][v][1], 0};
                    idx[v] = neighbour(s, c, d, 0);
                    if (idx[v] < 0) ok = 0;
                    p[v][0] = d[0] * e1[0] + d[1] * e2[0];
                    p[v][1] = d[0] * e1[1] + d[1] * e2[1];
                }
                if (!ok) continue;
                /* counter-clockwise about +z */
                double cr = (p[1][0] - p[0][0]) * (p[2][1] - p[0][1]) - (p[1][1] - p[0][1]) * (p[2][0] - p[0][0]);
                int j = idx[1], k = idx[2];
                if (cr < 0) { j = idx[2]; k = idx[1]; }
                acc += solid_angle(n + 3 * idx[0], n + 3 * j, n + 3 * k);
            }
    *Q = acc / (4.0 * M_PI);
    return SPO_OK;
}

/* ------------------------------------------------------------------ */
/* Metropolis Monte Carlo (Sec. Monte Carlo)                            */
/* ------------------------------------------------------------------ */
/* The sweep (Sec. Monte Carlo): every spin is visited once per iteration,
 * sequentially, in a random order -- spo_mc draws a fresh permutation of the
 * spins for every sweep of every replica by a Fisher-Yates shuffle.  Each
 * visit is a Metropolis step with the rest of the system fixed: a cone trial
 * move accepted with probability min(1, exp(-dE / kB T)).
 *
 * spo_mc_coloured is a second, separately named sweep order that serves as a
 * check of a parallel decomposition, not as the definition: it visits the
 * colours of a lattice colouring one after the other (spins of one colour
 * never interact, so a colour may be updated in any order).  It samples the
 * same Boltzmann distribution.  Two colourings:
 *  - the sum colouring, colour = (c0 + c1 + c2) mod k (mc_sum_modulus);
 *  - the product colouring, colour = basis atom and, per direction, the cell
 *    index modulo 2, or modulo 3 for a periodic direction of odd size
 *    divisible by 3 (mc_moduli).
 * The sum colouring is taken where it exists with no more colours than the
 * product colouring (or where the product colouring does not exist). */
static int mc_moduli(const spo_system *s, int m[3])
{
    for (int d = 0; d < 3; ++d) {
        int any = 0;
        for (int b = 0; b < s->nb; ++b)
            for (int e = 0; e < s->n_nbr[b]; ++e) {
                int dd = s->nbr[b][e].d[d];
                if (dd > 1 || dd < -1) return 0;
                if (dd != 0) any = 1;
            }
        if (s->nc[d] == 1) {
            if (any) return 0;
            m[d] = 1;
        } else if (!s->per[d] || s->nc[d] % 2 == 0) {
            m[d] = 2;
        } else if (s->nc[d] % 3 == 0) {
            m[d] = 3;
        } else {
            return 0;
        }
    }
    return 1;
}

/* The smallest k >= 2 for which (c0 + c1 + c2) mod k is a colouring, 0 if
 * there is none.  Conditions: one basis atom; no bond with d0 + d1 + d2
 * divisible by k (a bond changes the sum by d0 + d1 + d2); every periodic
 * direction a bond crosses has an extent divisible by k (the wrap then
 * changes the sum by a multiple of k); and k divides the first extent, so
 * that every row (c1, c2) holds n0 / k sites of each colour. */
static int mc_sum_modulus(const spo_system *s)
{
    if (s->nb != 1) return 0;
    for (int k = 2; k <= s->nc[0]; ++k) {
        if (s->nc[0] % k) continue;
        int ok = 1;
        for (int e = 0; e < s->n_nbr[0]; ++e) {
            const int *d = s->nbr[0][e].d;
            if ((d[0] + d[1] + d[2]) % k == 0) ok = 0;
            for (int a = 0; a < 3; ++a)
                if (d[a] != 0 && s->per[a] && s->nc[a] % k) ok = 0;
        }
        if (ok) return k;
    }
    return 0;
}

/* Colours of the sweep; *k = the sum colouring's modulus, 0 for the product
 * colouring with moduli m. */
static int mc_colouring(const spo_system *s, int *k, int m[3])
{
    int ks = mc_sum_modulus(s);
    int prod = mc_moduli(s, m) ? s->nb * m[0] * m[1] * m[2] : 0;
    if (ks && (!prod || ks <= prod)) {
        *k = ks;
        return ks;
    }
    *k = 0;
    return prod;
}

int spo_mc_colours(const spo_system *s)
{
    int k, m[3];
    if (!s || !s->have_ham) return 0;
    return mc_colouring(s, &k, m);
}

/* Field terms linear in n_i: Zeeman, exchange and DMI. */
static void mc_linear_field(const spo_system *s, const double *n, int i, double *Bl)
{
    int b, c[3];
    decode(s, i, &b, c);
    for (int k = 0; k < 3; ++k) Bl[k] = s->mu[b] * MU_B * s->h.B[k];
    for (int e = 0; e < s->n_nbr[b]; ++e) {
        const nbr_t *q = &s->nbr[b][e];
        int j = neighbour(s, c, q->d, q->jb);
        if (j < 0) continue;
        double nxd[3];
        cross3(n + 3 * j, q->D, nxd);
        for (int k = 0; k < 3; ++k) Bl[k] += q->J * n[3 * j + k] + nxd[k];
    }
}

/* Energy of spin i's own terms that are not linear in n_i: anisotropy and
 * the Gaussian landscape. */
static double mc_self_energy(const spo_system *s, int b, const double *ni)
{
    double kn = dot3(s->h.Khat[b], ni);
    double dummy[3] = {0, 0, 0};
    return -s->h.K[b] * kn * kn + gauss_terms(s, ni, dummy);
}

/* One Metropolis visit of spin i of replica r (spins x) in sweep `sweep`:
 * three uniforms in (0, 1) from Philox (counter (i, sweep lo, sweep hi,
 * 8 r + 1)) give the azimuth, the cone angle and the acceptance test.
 * Returns 1 if the trial was accepted. */
static int mc_visit(const spo_system *s, double *x, long i, uint64_t sweep, int r, double ct, double T,
                    const uint32_t key[2])
{
    int b, c[3];
    decode(s, (int)i, &b, c);
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)sweep, (uint32_t)(sweep >> 32), 8u * (uint32_t)r + 1u};
    uint32_t o[4];
    spo_philox4x32_10(ctr, key, o);
    double u0 = (o[0] + 0.5) * 2.3283064365386963e-10;
    double u1 = (o[1] + 0.5) * 2.3283064365386963e-10;
    double u2 = (o[2] + 0.5) * 2.3283064365386963e-10;
    /* trial direction: uniform on the cap of half-angle theta_cone around
     * n_i (cos theta uniform in [cos theta_cone, 1]) */
    double *ni = x + 3 * i;
    double cth = 1.0 - u1 * (1.0 - ct), sth = sqrt(fmax(0.0, 1.0 - cth * cth));
    double ph = 2.0 * M_PI * u0;
    double a[3] = {1, 0, 0};
    if (fabs(ni[0]) >= 0.9) { a[0] = 0; a[1] = 1; }
    double an = dot3(a, ni), e1[3], e2[3];
    for (int k = 0; k < 3; ++k) e1[k] = a[k] - an * ni[k];
    normalise3(e1);
    cross3(ni, e1, e2);
    double nt[3];
    for (int k = 0; k < 3; ++k) nt[k] = cth * ni[k] + sth * (cos(ph) * e1[k] + sin(ph) * e2[k]);
    normalise3(nt);
    double Bl[3];
    mc_linear_field(s, x, (int)i, Bl);
    double dE = -(dot3(nt, Bl) - dot3(ni, Bl)) + mc_self_energy(s, b, nt) - mc_self_energy(s, b, ni);
    int acc = T > 0 ? (u2 < exp(-dE / (K_B * T))) : (dE < 0);
    if (acc)
        for (int k = 0; k < 3; ++k) ni[k] = nt[k];
    return acc;
}

/* After a sweep of replica r: acceptance counts, the adaptive cone and the
 * sampled observables. */
static void mc_sweep_end(const spo_system *s, const double *x, int r, double accepted, const spo_mc_params *p,
                         double *cone, double *stats)
{
    long N = s->N;
    double *st = stats + 8 * (size_t)r;
    st[6] += accepted;
    st[7] += (double)N;
    /* reading of the adaptive cone: multiplicative feedback towards the
     * target acceptance ratio, theta <- theta exp(ratio - target), kept in
     * [1e-4, pi] */
    if (p->target_accept > 0) {
        double th = cone[r] * exp(accepted / (double)N - p->target_accept);
        cone[r] = fmin(M_PI, fmax(1e-4, th));
    }
    if (p->sample) {
        double M[3] = {0, 0, 0};
        for (long i = 0; i < N; ++i)
            for (int k = 0; k < 3; ++k) M[k] += x[3 * i + k];
        double mm = sqrt(dot3(M, M)) / (double)N;
        double e[6];
        spo_energy(s, x, e);
        st[0] += mm;
        st[1] += mm * mm;
        st[2] += mm * mm * mm * mm;
        st[3] += e[0];
        st[4] += e[0] * e[0];
        st[5] += 1;
    }
}

static int mc_check(const spo_system *s, double *spins, int n_rep, const double *T, const spo_mc_params *p,
                    int n_sweeps, double *cone, double *stats)
{
    if (!s || !s->have_ham || !spins || n_rep < 1 || !T || !p || n_sweeps < 0 || !cone || !stats) return SPO_ERR_ARG;
    if (s->h.dipole != SPO_DIPOLE_NONE) return SPO_ERR_ARG;
    return SPO_OK;
}

int spo_mc(const spo_system *s, double *spins, int n_rep, const double *T, const spo_mc_params *p, int n_sweeps,
           double *cone, double *stats)
{
    int rc = mc_check(s, spins, n_rep, T, p, n_sweeps, cone, stats);
    if (rc) return rc;
    long N = s->N;
    uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
    int bad = 0;
    /* replicas are independent Markov chains: one per thread */
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int r = 0; r < n_rep; ++r) {
        long *order = (long *)malloc(sizeof(long) * (size_t)(N > 0 ? N : 1));
        if (!order) {
            bad = 1;
            continue;
        }
        double *x = spins + 3 * N * (size_t)r;
        for (int sw = 0; sw < n_sweeps; ++sw) {
            uint64_t sweep = p->sweep0 + (uint64_t)sw;
            /* the visiting order: a uniformly random permutation (Fisher-Yates,
             * uniforms from Philox counter (k, sweep lo, sweep hi, 8 r + 2)) */
            for (long i = 0; i < N; ++i) order[i] = i;
            for (long k = N - 1; k > 0; --k) {
                uint32_t ctr[4] = {(uint32_t)k, (uint32_t)sweep, (uint32_t)(sweep >> 32), 8u * (uint32_t)r + 2u};
                uint32_t o[4];
                spo_philox4x32_10(ctr, key, o);
                long j = (long)((((uint64_t)o[0] << 32) | o[1]) % (uint64_t)(k + 1));
                long t = order[k];
                order[k] = order[j];
                order[j] = t;
            }
            double ct = cos(cone[r]);
            double accepted = 0;
            for (long q = 0; q < N; ++q) accepted += mc_visit(s, x, order[q], sweep, r, ct, T[r], key);
            mc_sweep_end(s, x, r, accepted, p, cone, stats);
        }
        free(order);
    }
    return bad ? SPO_ERR_STATE : SPO_OK;
}

int spo_mc_coloured(const spo_system *s, double *spins, int n_rep, const double *T, const spo_mc_params *p,
                    int n_sweeps, double *cone, double *stats)
{
    int rc = mc_check(s, spins, n_rep, T, p, n_sweeps, cone, stats);
    if (rc) return rc;
    int k, m[3];
    const int n_col = mc_colouring(s, &k, m);
    if (!n_col) return SPO_ERR_ARG;
    long N = s->N;
    uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
    for (int sw = 0; sw < n_sweeps; ++sw) {
        uint64_t sweep = p->sweep0 + (uint64_t)sw;
        for (int r = 0; r < n_rep; ++r) {
            double *x = spins + 3 * N * (size_t)r;
            double ct = cos(cone[r]);
            double accepted = 0;
            for (int col = 0; col < n_col; ++col)
                for (long i = 0; i < N; ++i) {
                    int b, c[3];
                    decode(s, (int)i, &b, c);
                    int cc = k ? (c[0] + c[1] + c[2]) % k
                               : b + s->nb * (c[0] % m[0] + m[0] * (c[1] % m[1] + m[1] * (c[2] % m[2])));
                    if (cc == col) accepted += mc_visit(s, x, i, sweep, r, ct, T[r], key);
                }
            mc_sweep_end(s, x, r, accepted, p, cone, stats);
        }
    }
    return SPO_OK;
}

/* ------------------------------------------------------------------ */
/* Covariant Hessian (Sec. MMF and its appendix on the spin manifold)  */
/* ------------------------------------------------------------------ */
/* Embedding second derivatives applied to w: the negative of the field's
 * terms that are linear in the spins -- exchange J w_j, DMI w_j x D_ij,
 * anisotropy 2 K (Khat.w_i) Khat -- and the Gaussian landscape's
 * (e/s^2)(u^2/s^2 - 1) c (c.w_i). */
static void hbar_apply(const spo_system *s, const double *n, const double *w, long i, double *out)
{
    int b, c[3];
    decode(s, (int)i, &b, c);
    const spo_hamiltonian *h = &s->h;
    double acc[3] = {0, 0, 0};
    double kw = dot3(h->Khat[b], w + 3 * i);
    for (int k = 0; k < 3; ++k) acc[k] = 2.0 * h->K[b] * kw * h->Khat[b][k];
    for (int e = 0; e < s->n_nbr[b]; ++e) {
        const nbr_t *q = &s->nbr[b][e];
        int j = neighbour(s, c, q->d, q->jb);
        if (j < 0) continue;
        double wxd[3];
        cross3(w + 3 * j, q->D, wxd);
        for (int k = 0; k < 3; ++k) acc[k] += q->J * w[3 * j + k] + wxd[k];
    }
    for (int k = 0; k < 3; ++k) out[k] = -acc[k];
    const double *ni = n + 3 * i;
    for (int g = 0; g < h->n_gauss; ++g) {
        const double *G = h->gauss[g];
        double a = G[0], sig = G[1];
        const double *cc = &G[2];
        double u = 1.0 - dot3(ni, cc);
        double eg = a * exp(-u * u / (2 * sig * sig));
        double f = eg / (sig * sig) * (u * u / (sig * sig) - 1.0) * dot3(cc, w + 3 * i);
        for (int k = 0; k < 3; ++k) out[k] += f * cc[k];
    }
}

int spo_hessian_apply(const spo_system *s, const double *n, const double *v, double *out)
{
    if (!s || !s->have_ham || !n || !v || !out) return SPO_ERR_ARG;
    if (s->h.dipole != SPO_DIPOLE_NONE) return SPO_ERR_ARG;
    long N = s->N;
    double *w = (double *)malloc(sizeof(double) * 3 * N), *B = (double *)malloc(sizeof(double) * 3 * N);
    if (!w || !B) { free(w); free(B); return SPO_ERR_STATE; }
    for (long i = 0; i < N; ++i) {
        double vn = dot3(v + 3 * i, n + 3 * i);
        for (int k = 0; k < 3; ++k) w[3 * i + k] = v[3 * i + k] - vn * n[3 * i + k];
    }
    int rc = spo_effective_field(s, n, B, -1);
    for (long i = 0; i < N && !rc; ++i) {
        double hb[3];
        hbar_apply(s, n, w, i, hb);
        const double *ni = n + 3 * i;
        double hn = dot3(hb, ni);
        double nB = dot3(ni, B + 3 * i); /* -(n . grad Hbar) = n . B */
        for (int k = 0; k < 3; ++k) out[3 * i + k] = hb[k] - hn * ni[k] + nB * w[3 * i + k];
    }
    free(w); free(B);
    return rc;
}

/* Tangent basis of spin i: e1 = P x (or P y when |n_x| >= 0.9), normalised;
 * e2 = n x e1. */
static void tangent_basis(const double *ni, double *e1, double *e2)
{
    double a[3] = {1, 0, 0};
    if (fabs(ni[0]) >= 0.9) { a[0] = 0; a[1] = 1; }
    double an = dot3(a, ni);
    for (int k = 0; k < 3; ++k) e1[k] = a[k] - an * ni[k];
    normalise3(e1);
    cross3(ni, e1, e2);
}

int spo_hessian_dense(const spo_system *s, const double *n, double *H, double *T)
{
    if (!s || !s->have_ham || !n || !H) return SPO_ERR_ARG;
    long N = s->N, M = 2 * N;
    double *Tb = (double *)malloc(sizeof(double) * 6 * N);
    double *v = (double *)calloc(3 * N, sizeof(double)), *hv = (double *)malloc(sizeof(double) * 3 * N);
    if (!Tb || !v || !hv) { free(Tb); free(v); free(hv); return SPO_ERR_STATE; }
    for (long i = 0; i < N; ++i) {
        double e1[3], e2[3];
        tangent_basis(n + 3 * i, e1, e2);
        for (int k = 0; k < 3; ++k) {
            Tb[6 * i + 2 * k] = e1[k];
            Tb[6 * i + 2 * k + 1] = e2[k];
        }
    }
    int rc = SPO_OK;
    for (long col = 0; col < M && !rc; ++col) {
        long j = col / 2;
        int a = (int)(col % 2);
        memset(v, 0, sizeof(double) * 3 * N);
        for (int k = 0; k < 3; ++k) v[3 * j + k] = Tb[6 * j + 2 * k + a];
        rc = spo_hessian_apply(s, n, v, hv);
        for (long row = 0; row < M && !rc; ++row) {
            long i = row / 2;
            int bb = (int)(row % 2);
            double x = 0;
            for (int k = 0; k < 3; ++k) x += Tb[6 * i + 2 * k + bb] * hv[3 * i + k];
            H[row * M + col] = x;
        }
    }
    if (T) memcpy(T, Tb, sizeof(double) * 6 * N);
    free(Tb); free(v); free(hv);
    return rc;
}

