#pragma once
#include "ie_common.cuh"

namespace ie {

// Apply the folded spectral blocks in place to spec[2Ny][2Nx][R * 3Nz].
// Returns -1 if R > 4, 3 Nz > 1024 or a launch fails (nothing is applied then).
template <typename T>
int launch_contract(C<T> *spec, const C<T> *qf, int Nx, int Ny, int Nz, int R, cudaStream_t s);

// Use the TMA-pipelined kernel where it applies (c64, Nz in {16, 24, 32, 48}, R <= 2).
extern bool contract_tma_enabled;
// Error code recorded by a contraction kernel since the last call (0: none); resets it.
int contract_take_error();

}  // namespace ie
