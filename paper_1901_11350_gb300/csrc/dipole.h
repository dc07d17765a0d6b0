// dipole.h -- dipole-dipole field by zero-padded FFT convolution (Sec.
// "Dipolar interactions"): one transform of the moments, multiplication by
// the transformed interaction tensor, one inverse transform.
#pragma once

#include "common.cuh"

namespace spgb {

struct DipoleGeom {
    int nc[3];
    double A[3][3];  // Bravais vectors times the lattice constant, Angstrom
    int nb;
    double mu[SP_MAX_BASIS];
    double basis[SP_MAX_BASIS][3];
};

struct DipolePlan;

// Records the geometry on the host (no device memory yet).  SP_ERR_UNSUPPORTED
// unless one basis atom, n2 = 1 and padded sides <= 4096.
int dipole_create(DipolePlan **out, const DipoleGeom &g);
void dipole_destroy(DipolePlan *p);
// Dipole field (meV) of the spins n into out (prec SP_F32: float4, SP_F64:
// 32-byte records).  Builds the transformed kernel on first use.
cudaError_t dipole_field(DipolePlan *p, int prec, const void *n, void *out, cudaStream_t st);
// Use the radix-2 shared-memory transforms even where the FP32 warp-FFT path
// applies (to compare the two).
void dipole_force_generic(DipolePlan *p, bool on);

}  // namespace spgb
