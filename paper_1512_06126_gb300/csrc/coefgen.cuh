#pragma once
#include "ie_common.cuh"

namespace ie {

struct CoefGenInput {
  int nx, ny, nz;
  double hx, hy;
  const double *z_edges;     // nz + 1
  const int *cell_layer;     // layer index of every z-cell
  int n_interfaces;          // L
  const double *interfaces;  // d_1 .. d_L
  const double *sigma;       // L + 1 complex (interleaved)
  double freq;
};

enum class CoefGenStatus { kOk, kUnsupported, kCuda };

// Compressed real-space tensor [Ny][Nx][6][Nz][Nz] (c128) written to q_dev.
CoefGenStatus generate_coefficients(const CoefGenInput &in, double2 *q_dev, cudaStream_t s);

}  // namespace ie
