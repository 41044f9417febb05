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

// Receiver kernels for a point at depth z_r (in layer r_layer) above the grid, for
// every lateral offset i in [0, Ny), j in [0, Nx) (receiver minus cell) and source
// z-cell b: tab_dev c128 [Ny][Nx][Nz][10], entries E_xx, E_yy, E_xy, E_xz, E_yz,
// H_xx, H_yx, H_xy, H_xz, H_yz (E_yx = E_xy, H_yy = -H_xx).  Cells not strictly
// below z_r get zeros.  offs_host (optional): n_off_host real offsets (Dy, Dx) in metres
// (receiver minus cell centre) in place of the quadrant of cell offsets: tab_dev then
// holds [n_off_host][Nz][10].
CoefGenStatus generate_receiver_tables(const CoefGenInput &in, double z_r, int r_layer, double2 *tab_dev,
                                       cudaStream_t s, const double *offs_host = nullptr, int n_off_host = 0);

}  // namespace ie
