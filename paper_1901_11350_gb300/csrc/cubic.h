// cubic.h -- parameters of the shell-symmetric 27-point stencil path (cubic.cu).
#pragma once

#include "internal.h"

namespace spgb {

template <typename T> struct CubicParams {
    int nx, ny, nz, per0, per1, per2;
    T J1, J2, J3;          // exchange on faces, edges, corners of the 3x3x3 cell neighbourhood
    T Dx[3], Dy[3], Dz[3]; // DMI vectors of the +x, +y, +z faces (the -o face carries -D_o)
    T Bz[3];               // Zeeman field mu B, meV
    T K, Kh[3];            // anisotropy
    int dmi_mode;          // 0 none, 1 bulk (D_o = D ohat, one D), 2 any face vectors
};

// Columns per thread the 27-point kernels take for a request of `rows` (1 or
// 2): two only in FP32, for a single lattice without the dipole field.
int cubic_rows_taken(int prec, int rows, bool replicas, bool dipole);
// Work units of the 27-point path: (32 x 8 rows column tile, plane) pairs.
long cubic_units(int nx, int ny, int nz, int rows = 1);
// Resident 256-thread CTAs per SM of the 27-point kernels (occupancy query).
int cubic_resident_ctas(int prec, int pass, int rows = 1);

// pass 0: predictor (stencil on src = n, writes np and q);
// pass 1: corrector (stencil on src = np, reads q, writes nout = n).
// CTA b streams the units [b*per, (b+1)*per), tile-major; with c.n_rep > 1
// the units of all replicas (stored one after another), replica-major.
// rows: columns per thread (1 or 2, see cubic_rows_taken); per counts units
// of that tile height.  lean: FP32 stochastic Heun passes of one lattice
// without the dipole field take launch_cubic_lean where the lattice fits it.
template <typename T>
cudaError_t launch_cubic(int pass, int solver, const CubicParams<T> &P, const rec_t<T> *src, rec_t<T> *np, rec_t<T> *q,
                         rec_t<T> *nout, const rec_t<T> *Bdd, const LlgConst<T> &c, int per, cudaStream_t st,
                         int rows = 1, bool lean = false);

// The lean stochastic Heun passes (cubic_lean.cu): FP32, one lattice without
// the dipole field cut into whole 32 x 8 rows column tiles (nx % 32 == 0,
// ny % (8 rows) == 0: cubic_lean_fits); the same (tile, plane) units and
// `per` as launch_cubic with the same rows (1 or 2 columns per thread).
bool cubic_lean_fits(int nx, int ny, int rows);
cudaError_t launch_cubic_lean(int pass, const CubicParams<float> &P, const float4 *src, float4 *np, float4 *q,
                              float4 *nout, const LlgConst<float> &c, int per, cudaStream_t st, int rows);
int cubic_lean_resident_ctas(int pass, int rows);

}  // namespace spgb
