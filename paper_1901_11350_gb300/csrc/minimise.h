// minimise.h -- velocity-projection minimiser (Appendix D) and GNEB
// (Sec. GNEB, Appendix F) drivers, single system / single chain and batched.
#pragma once

#include <vector>

#include "common.cuh"

namespace spgb {

struct MinScratch;
void min_scratch_destroy(MinScratch *s);

struct MinArgs {
    double dt, mass, tol;
    int max_iter, check_every;
};

struct GnebArgs {
    double dt, mass, k;
    int climbing, M, n_iter;
    const int *kinds;  // host, one SP_IMAGE_* per image of all chains, or NULL
    double w;          // energy weight of the spring lengths (0: geodesic)
    // 1: the iterations of a call run in one persistent cooperative launch
    // (grid barriers between the passes) instead of one launch per pass
    int persistent = 0;
    long long wait_limit = 0;   // polls of a grid-barrier wait before it gives up (persistent)
    unsigned *status = nullptr; // device address of the context's status word (timeouts), or null
};

template <typename T>
int vp_minimise(MinScratch **s, const Stencil<T> &S, void *n, void *v, const MinArgs &a, int *iters, double *max_torque,
                cudaStream_t st);

template <typename T>
int gneb_run(MinScratch **s, const Stencil<T> &S, void *chain, void *vel, const GnebArgs &a, double *E_dev,
             double *fmax_dev, cudaStream_t st);

// Batched GNEB: chain c has M[c] images of stencils[c].N spins stored from
// record offset spin0[c] of chain/vel; energies[img0[c] + v] and
// fmax[c] receive the results, img0 the prefix sums of M.
template <typename T>
int gneb_batch_run(MinScratch **s, const std::vector<Stencil<T>> &stencils, const std::vector<int> &M,
                   const std::vector<long long> &spin0, void *chain, void *vel, const GnebArgs &a, double *E_dev,
                   double *fmax_dev, cudaStream_t st);

// Path analysis of one chain: per image the FP64 energy, geodesic distance
// to the next image and slope dE/dr (host arrays of M; dist has M-1).
template <typename T>
int gneb_path_scalars(MinScratch **s, const Stencil<T> &S, const void *chain, int M, double *E, double *dist,
                      double *slope, cudaStream_t st);

// Batched velocity projection: system c has stencils[c].N spins from record
// offset spin0[c]; iters[c] and max_torque[c] (host) receive the results.
template <typename T>
int vp_batch_run(MinScratch **s, const std::vector<Stencil<T>> &stencils, const std::vector<long long> &spin0,
                 void *spins, void *vel, const MinArgs &a, int *iters, double *max_torque, cudaStream_t st);

}  // namespace spgb
