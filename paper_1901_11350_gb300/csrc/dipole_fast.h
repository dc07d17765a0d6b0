// dipole_fast.h -- warp-FFT dipole path for FP32 on a 1024 x 1024 padded grid.
#pragma once

#include <cuda_runtime.h>

namespace spgb {

// Raise the kernels' dynamic shared-memory limits (once per device).
cudaError_t dipole_fast_setup();
// Field of the spins n (n0 x n1, 257..512 per side) into out; ST: 3 x 513 x n1
// complex scratch; Kt: transformed kernel [513][6][1024] (structure of arrays
// per column), scaled.
cudaError_t dipole_fast_run(int n0, int n1, const float4 *n, float2 *ST, const float *Kt, float4 *out, cudaStream_t st);

}  // namespace spgb
