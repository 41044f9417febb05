#pragma once
#include "ie_common.cuh"

namespace ie {

// Apply the folded spectral blocks in place to spec[2Ny][2Nx][R * 3Nz].
// Returns -1 if R > 4.
template <typename T>
int launch_contract(C<T> *spec, const C<T> *qf, int Nx, int Ny, int Nz, int R, cudaStream_t s);

// Shared memory needed by the contraction CTA.
size_t contract_smem_bytes(int Nz, int R, size_t elem);

}  // namespace ie
