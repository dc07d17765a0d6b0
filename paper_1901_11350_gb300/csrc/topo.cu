// topo.cu -- Berg-Luescher topological charge of a 2D one-atom lattice
// (Appendix A): Q = (1/4 pi) sum_l A_l over the two elementary triangles of
// every cell, A_l the signed solid angle of the spins at its corners,
// evaluated as 2 atan2(n_i.(n_j x n_k), 1 + n_i.n_j + n_i.n_k + n_j.n_k).
#include "internal.h"

namespace spgb {

namespace {

template <typename T>
__global__ void __launch_bounds__(kBlock) k_topo(const __grid_constant__ Stencil<T> S, const rec_t<T> *__restrict__ n,
                                                 int flip, double *__restrict__ partials)
{
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0;
    if (cell < S.n0 * S.n1) {
        int c0 = cell % S.n0, c1 = cell / S.n0;
        // corners (0,0) (1,0) (0,1) and (1,0) (1,1) (0,1)
        const int tri[2][3][2] = {{{0, 0}, {1, 0}, {0, 1}}, {{1, 0}, {1, 1}, {0, 1}}};
        for (int t = 0; t < 2; ++t) {
            int idx[3];
            bool ok = true;
            for (int v = 0; v < 3; ++v) {
                int x = wrap(c0 + tri[t][v][0], S.n0, S.per0), y = wrap(c1 + tri[t][v][1], S.n1, S.per1);
                ok = ok && x >= 0 && y >= 0;
                idx[v] = x + S.n0 * y;
            }
            if (!ok) continue;
            v3<T> a = ld(n, idx[0]), b = ld(n, flip ? idx[2] : idx[1]), c = ld(n, flip ? idx[1] : idx[2]);
            double trip = (double)dot(a, cross(b, c));
            double den = 1.0 + (double)dot(a, b) + (double)dot(a, c) + (double)dot(b, c);
            acc += 2.0 * atan2(trip, den);
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double sh[kBlock / 32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0;
        for (int w = 0; w < kBlock / 32; ++w) v += sh[w];
        partials[blockIdx.x] = v;
    }
}

__global__ void __launch_bounds__(kBlock) k_topo_final(const double *__restrict__ partials, int nblk, double *Q)
{
    __shared__ double sh[kBlock];
    double acc = 0;
    for (int p = threadIdx.x; p < nblk; p += kBlock) acc += partials[p];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kBlock / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) Q[0] = sh[0] / (4.0 * 3.14159265358979323846);
}

}  // namespace

template <typename T>
cudaError_t launch_topo(const Stencil<T> &S, const rec_t<T> *n, int flip, double *partials, double *Q, cudaStream_t st)
{
    int nblk = blocks_for(S.n0 * S.n1);
    k_topo<T><<<nblk, kBlock, 0, st>>>(S, n, flip, partials);
    k_topo_final<<<1, kBlock, 0, st>>>(partials, nblk, Q);
    return cudaGetLastError();
}

template cudaError_t launch_topo<float>(const Stencil<float> &, const float4 *, int, double *, double *, cudaStream_t);
template cudaError_t launch_topo<double>(const Stencil<double> &, const dq4 *, int, double *, double *, cudaStream_t);

}  // namespace spgb
