#pragma once
#include "ie_common.cuh"

namespace ie {

void launch_embed(const double2 *qreal, double2 *emb, int Nx, int Ny, int Nz, long long e0, long long E,
                  cudaStream_t s);
void launch_pack(const double2 *spec, double2 *q64, float2 *q32, int Nx, int Ny, int Nz, long long e0, long long E,
                 cudaStream_t s);
void launch_cast64to32(const double2 *a, float2 *b, long long n, cudaStream_t s);
void launch_cast32to64(const float2 *a, double2 *b, long long n, cudaStream_t s);

}  // namespace ie
