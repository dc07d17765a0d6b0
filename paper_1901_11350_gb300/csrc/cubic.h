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

// pass 0: predictor (stencil on src = n, writes np and q);
// pass 1: corrector (stencil on src = np, reads q, writes nout = n).
template <typename T>
cudaError_t launch_cubic(int pass, int solver, const CubicParams<T> &P, const rec_t<T> *src, rec_t<T> *np, rec_t<T> *q,
                         rec_t<T> *nout, const rec_t<T> *Bdd, const LlgConst<T> &c, int zc, cudaStream_t st);

}  // namespace spgb
