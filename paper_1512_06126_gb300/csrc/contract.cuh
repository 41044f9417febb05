#pragma once
#include "ie_common.cuh"

namespace ie {

// Kernel variants of the contraction: the TMA ring with one slot and two CTAs per SM
// (two output rows per thread for two right-hand sides), the ring with three slots and
// one CTA per SM (both c64, Nz in {16, 24, 32, 48}, R <= 2), the panel-staged kernel
// (any precision and Nz with 3 Nz <= 1024), the one-slot ring with one output row
// per thread (two right-hand sides only), and two kernels feeding 3xTF32 tensor-core
// MMAs (c64, Nz in {16, 32, 48}, R <= 2): a producer warp with a two-slot ring and
// fragments read in place, or the one-slot ring with an unpacking pass.
// Variants 6 and 7 run on the 5th-generation tensor cores: tcgen05.mma with the block in
// tensor memory and FP32 accumulators there (c64, Nz in {16, 32}, R <= 2): 6 kind::tf32
// on the 3xTF32 split, 7 kind::f16 on a scaled two-way FP16 split (the same 22
// significant bits, half the instructions; needs the per-wavenumber exponents of
// launch_block_exponents).  Variant 8 takes the 3xTF32 mma.sync path one Nz x Nz
// matrix of the block at a time, staging and unpacking one matrix per sub-step (c64,
// Nz in {16, 32, 48, 64}, R <= 2): the tensor-core variant for Nz = 64.
enum ContractVariant {
  kContractAuto = -1, kContractTma1 = 0, kContractTma3 = 1, kContractPanel = 2, kContractTma1Row = 3,
  kContractMma = 4, kContractMmaUnpack = 5, kContractTc = 6, kContractTc16 = 7, kContractMmaComp = 8
};
constexpr int kContractVariants = 9;
bool contract_variant_available(int variant, int Nz, int R, bool c64);
// Whether the panel kernel, the fallback of every variant, can stage a contraction of
// Nz layers and R right-hand sides (c64 or c128) in shared memory.
bool contract_fits(int Nz, int R, bool c64);

// Apply the folded spectral blocks in place to the R right-hand sides whose spectrum
// vectors are spec[(ky 2Nx + kx) ldz + 0 .. R 3Nz) (ldz >= R 3Nz).  variant: one of
// ContractVariant (kContractAuto: the TMA ring where it applies, else the panel kernel;
// an unavailable variant falls back to the panel kernel).  Returns -1 if R > 4,
// 3 Nz > 1024, ldz < R 3Nz or a launch fails (nothing is applied then).
// err: device word in which a kernel records a wait that ran out (kContractTimeout; the
// wavenumbers it had not reached stay uncontracted); NULL: the library's own word.
// qexp, qh: the per-wavenumber exponents of launch_block_exponents and the FP16-split
// blocks of launch_split_f16 (variant 7 only; either NULL makes variant 7 fall back).
template <typename T>
int launch_contract(C<T> *spec, const C<T> *qf, int Nx, int Ny, int Nz, int R, int ldz, int variant, int *err,
                    cudaStream_t s, const int *qexp = nullptr, const void *qh = nullptr);
// qexp[w] = the exponent that scales the largest |re|, |im| of the packed c64 block of
// folded wavenumber w into [2^13, 2^14) (nf blocks of 2 Nz (2 Nz + 1) complex).
void launch_block_exponents(const float2 *qf, int *qexp, long long nf, int Nz, cudaStream_t s);
// The packed c64 blocks scaled by 2^qexp[w] and split into FP16 pairs, the layout of qf
// with 8 bytes per complex: (hi(re) | lo(re) << 16, hi(im) | lo(im) << 16), hi =
// fp16(x 2^e), lo = fp16(x 2^e - hi) (round to nearest): the A operand of variant 7,
// split once at set-up instead of in every product.
void launch_split_f16(const float2 *qf, const int *qexp, void *qh, long long nf, int Nz, cudaStream_t s);

// Double-float copy of packed blocks: qdf[i] = (hi, lo of re, hi, lo of im) of q64[i],
// hi = fl32(x), lo = fl32(x - hi).
void launch_split_df(const double2 *q64, float4 *qdf, long long count, cudaStream_t s);
// The contraction of c128 spectra in compensated double-float arithmetic (the FP32
// pipe; about twice-FP32 accuracy) from the double-float copy of the blocks.  R <= 4;
// returns -1 (nothing applied) if the grid or R does not fit or the launch fails.
int launch_contract_df(double2 *spec, const float4 *qdf, int Nx, int Ny, int Nz, int R, int ldz, cudaStream_t s);

// Use the TMA-pipelined kernel where it applies (c64, Nz in {16, 24, 32, 48}, R <= 2).
extern bool contract_tma_enabled;
// Error code recorded in err (NULL: the library's own word) by a contraction kernel
// since the last call (0: none; -1 if it cannot be read); waits for stream s, resets it.
int contract_take_error(int *err, cudaStream_t s);
// Polls of the main waits of every contraction launched afterwards (< 0: the default;
// 0: every main wait gives up without polling, which tests the error path).
void set_wait_limit(long long polls);

}  // namespace ie
