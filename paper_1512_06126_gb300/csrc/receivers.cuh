#pragma once
#include "ie_common.cuh"

namespace ie {

// Receiver-side kernels of the MT misfit and its gradient (eq. (APR_lab)).
// tab: c128 [Ny][Nx][Nz][10] receiver kernels (see generate_receiver_tables) for
// offsets (receiver minus cell) in the non-negative quadrant; the other quadrants
// follow from the lateral parities of the kernels.  rec_ix/rec_iy: receiver cell
// columns (device, n_rec each).  Vectors are c128 [nrhs][3][Nz][Ny][Nx].

// f[p][r][4] = (Ex, Ey, Hx, Hy) at receiver r for solution p: the normal field of
// polarisation pol[p] (0: x, E_x = en, H_y = hn; 1: y, E_y = en, H_x = -hn) plus
// sum over cells of the kernels times the current jfac * u (jfac = 2 s gamma).
// rec_grp: NULL for receivers at cell centres (tab: the quadrant table above); otherwise
// the group of every receiver, tab [group][2 Ny][2 Nx][Nz][10] over offsets (rec_iy - i,
// rec_ix - j) in [-Ny, Ny) x [-Nx, Nx), signs included (arbitrary sites).
void launch_receiver_fields(const double2 *tab, const int *rec_ix, const int *rec_iy, const int *rec_grp,
                            int n_rec, const double2 *u, const double2 *jfac, int nrhs, int nx, int ny, int nz,
                            int pol0, int pol1, int pol2, int pol3, double2 en, double2 hn, double2 *f,
                            cudaStream_t s);

// rhs[p] = jfac * (G^T c[p]): c[p][r][4] are receiver sources for (Ex, Ey, Hx, Hy).
void launch_receiver_adjoint(const double2 *tab, const int *rec_ix, const int *rec_iy, const int *rec_grp,
                             int n_rec, const double2 *c, const double2 *jfac, int nrhs, int nx, int ny, int nz,
                             double2 *rhs, cudaStream_t s);

// rho[k] = |z[k]|^2 / (omega mu0), phase[k] = arg z[k] in degrees (k < n)
void launch_mt_apparent(const double2 *z, int n, double omega, double *rho, double *phase, cudaStream_t s);

// Per receiver: Z = E H^-1 from f[2][n_rec][4] (x then y polarisation), phi_r =
// 1/2 sum |Z - Zobs|^2, and the adjoint sources c[2][n_rec][4] of dPhi.
void launch_mt_misfit(const double2 *f, const double2 *zobs, int n_rec, double2 *z, double *phi_r, double2 *c,
                      cudaStream_t s);

// grad[m] += Re sum_p gdiv[m] (w[p]_m . u[p]_m)  (bilinear in the three components)
void launch_gradient_accumulate(const double2 *u, const double2 *w, const double2 *gdiv, int nrhs, long long ncell,
                                double *grad, cudaStream_t s);

// e = u times the per-cell factor fac, for nvec vectors of ncell cells each
void launch_cell_scale(const double2 *u, const double2 *fac, int nvec, long long ncell, double2 *e, cudaStream_t s);

}  // namespace ie
