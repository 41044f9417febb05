/*
 * ie.h -- C ABI of the GB300 (sm_103a) Galerkin integral-equation solver.
 *
 * The library solves the discretised contracting integral equation of
 * Kruglyakov & Bloshanskaya ("High-performance parallel solver for integral
 * equations of electromagnetics based on Galerkin method"):
 *
 *   U_n - sum_m gamma_m K_n^m U_m = U_n^0                       eq. (slae1)
 *   K_n^m = I + (2/V_n) sqrt(Re s_b^m Re s_b^n) B_n^m,
 *   gamma_m = (s_a^m - s_b^m) / (s_a^m + conj s_b^m)            eq. (slae_matricies)
 *
 * whose matrix is A = S + R1 B R2 with S = diag(1 - gamma), R1 = -diag(2 s / V),
 * R2 = diag(s gamma), s = sqrt(Re sigma_b) and B block-Toeplitz in x and y
 * (eq. (matrix_convolv), (bcyl)).  B is applied with zero-padded 2-D FFTs and a
 * per-wavenumber contraction of the symmetry-compressed blocks (Sect. 3.1, 3.3).
 *
 * Conventions.  SI units; time dependence exp(-i omega t); z positive downwards,
 * the earth surface at z = 0.  Complex numbers are interleaved (re, im) pairs of
 * double (c128) or float (c64).  A field vector for R right-hand sides is
 * [R][3][Nz][Ny][Nx] (component x, y, z; x fastest).  Cell arrays are [Nz][Ny][Nx].
 *
 * Ownership.  Pointers named *_host are host memory read during the call; the
 * library keeps no reference to them.  Pointers named *_dev are device memory on
 * the context's device, owned by the caller, and must stay valid until the call
 * that uses them has completed on its stream.  The context owns its coefficient
 * tensors and workspaces and frees them in ie_destroy.
 *
 * Errors.  Every call returns an ie_status; nothing is thrown across the ABI.
 * On IE_ERR_* the outputs are unspecified.  A solve that reaches its iteration
 * cap returns IE_NOT_CONVERGED with info filled and the best iterate in u.
 * The contraction kernels wait on asynchronous copies with a bounded number of
 * polls; a wait that runs out is recorded in the context's error word and reported
 * as IE_ERR_TIMEOUT by the next solve synchronisation (restart or end of a solve) or,
 * for asynchronous products, by ie_sync (ie_noalloc_sync without a context).
 *
 * Streams.  Calls are ordered on the context's stream (ie_ctx_stream); matvec
 * accepts an explicit stream.  ie_setup and the solves synchronise before they
 * return.
 */
#ifndef IE_GB300_H
#define IE_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ie_ctx ie_ctx;

typedef enum {
  IE_OK = 0,
  IE_NOT_CONVERGED = 1,  /* iteration cap reached; best iterate returned */
  IE_BREAKDOWN = 2,      /* a Krylov vector vanished before convergence */
  IE_ERR_ARG = -1,       /* invalid argument (null pointer, size, enum) */
  IE_ERR_GEOMETRY = -2,  /* a cell straddles a layer interface, or Re sigma_b <= 0 in the domain */
  IE_ERR_COEFF = -3,     /* coefficient tensor missing or inconsistent */
  IE_ERR_OOM = -4,       /* device allocation failed */
  IE_ERR_CUDA = -5,      /* a CUDA call failed */
  IE_ERR_SCRATCH = -6,   /* the problem needs more work space than ie_matvec_noalloc's fixed array */
  IE_ERR_TIMEOUT = -7    /* a bounded wait inside a contraction kernel ran out: that product is incomplete */
} ie_status;

enum { IE_C64 = 0, IE_C128 = 1, IE_C128_DF = 7 };  /* element type of matvec vectors (see ie_matvec) */
enum { IE_FP64 = 0, IE_MIXED = 1, IE_MIXED_FP64K = 2 };  /* solve precision (see ie_solve) */

/* Grid of Nx*Ny*Nz cells (eq. (bcyl)): equal lateral sizes hx, hy; z_edges_host holds
 * the nz+1 increasing cell boundaries (m).  x0, y0 are the lateral origin (m). */
typedef struct {
  int nx, ny, nz;
  double hx, hy;
  const double *z_edges_host;
  double x0, y0;
} ie_grid;

/* Layered background (Appendix B): n_interfaces = L values d_1..d_L (d_1 = 0, the
 * surface); sigma_host holds L+1 complex conductivities (interleaved) for the air
 * (layer 0), the finite layers and the basement, in S/m. */
typedef struct {
  int n_interfaces;
  const double *interfaces_host;
  const double *sigma_host;
} ie_layers;

typedef struct {
  int restart;       /* GMRES restart length m (2..63); 0 selects 30 */
  int max_iter;      /* cap on inner iterations per solve; 0 selects 2000 */
  double inner_tol;  /* mixed precision: relative tolerance of each inner c64 solve; 0 selects 1e-3 */
  int max_outer;     /* mixed precision: cap on refinement steps; 0 selects 50 */
  int autotune;      /* 0 or 1: time the c64 contraction variants at set-up and keep the
                        fastest per right-hand-side count; -1: built-in choice */
} ie_options;

typedef struct {
  int outer_iters;       /* FP64 residual evaluations (refinement steps) */
  int inner_iters;       /* total Krylov iterations */
  double final_rel_res;  /* max over right-hand sides of ||b - A u|| / ||b|| with the c128 operator */
  double t_solve;        /* wall time of the solve, s */
  int reorth;            /* Gram-Schmidt steps that took a second projection (all right-hand sides) */
} ie_solve_info;

/* Build a context for one grid, one layered background, one anomaly and n_freq
 * frequencies (one operator instance per frequency).
 *   sigma_a_host : Nz*Ny*Nx complex anomaly conductivities (interleaved), cell order.
 *   freq_host    : n_freq frequencies in Hz.
 *   q_real_host  : n_freq compressed real-space coefficient tensors, each
 *                  [Ny][Nx][6][Nz][Nz] complex (block order xx, yy, zz, xy, xz, yz;
 *                  offsets i in [0,Ny), j in [0,Nx); the storage of eq. (matrix_symm)),
 *                  i.e. the 3x3 blocks B_n^m of Appendix A; or NULL, in which case the
 *                  library generates them on the device (ie_generate_coefficients).
 *   max_rhs      : largest number of right-hand sides passed to one call (1..16); a
 *                  product (ie_matvec) or a per-instance block of a batched solve takes
 *                  at most 4.
 * The tensors are transformed on the device (2N-periodic embedding with the
 * parities of Lemma 2, 2-D DFT) and kept in c128 and c64. */
ie_status ie_setup(const ie_grid *grid, const ie_layers *layers, const double *sigma_a_host, int n_freq,
                   const double *freq_host, const double *q_real_host, int max_rhs, const ie_options *opt,
                   ie_ctx **out);

/* Allocation-free c64 product y = A x for callers that cannot allocate device memory
 * (an allocator-free host policy, or a plug-in restricted to the buffers it is given):
 * no context, no cudaMalloc/cudaFree, no allocating library call.  The paper has no
 * counterpart; it is the same five kernels as ie_matvec with their two FFT work arrays
 * placed in one fixed device array of 64 MiB that the library reserves on every GPU
 * that loads it, for the life of the process.
 *   qf_dev        : folded spectral coefficients, c64 [(Ny+1)(Nx+1)][2Nz(2Nz+1)]: for
 *                   kx in [0, Nx], ky in [0, Ny] the DFT of the 2N-periodic embedding of
 *                   Q, blocks xx, yy, zz, xy as packed upper triangles (row-major, a <= b)
 *                   then xz, yz in full (the layout ie_setup builds internally).
 *   in_scale_dev  : c64 per cell [Nz][Ny][Nx], R2 = s gamma (forward product).
 *   out_scale_dev : c64 per cell, R1 / (4 Nx Ny) = -2 s / (V 4 Nx Ny).
 *   diag_dev      : c64 per cell, S = 1 - gamma (may be NULL for y = R1 B R2 x).
 *   x_dev, y_dev  : c64 [nrhs][3][Nz][Ny][Nx], must not alias; nrhs 1..4.
 * The work space needs (6 Nx Ny) * nrhs * 3 Nz * 8 bytes; larger problems return
 * IE_ERR_SCRATCH.  Shapes the contraction cannot stage in shared memory return
 * IE_ERR_ARG before anything is launched: 3 Nz <= 1024 and 24 Nz (MAXC + 17) <= 227 KiB
 * with MAXC = 4, 8, 16 for 1, 2, 3..4 right-hand sides (Nz <= 341 for one or two,
 * Nz <= 293 for three or four).  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call outside any stream capture.  All calls
 * share the array: calls whose kernels overlap on the GPU (two streams, two threads)
 * race on it and must be serialised by the caller.  Nothing in the array needs to
 * start at zero (each call writes everything it reads).  Asynchronous on stream
 * (a cudaStream_t, NULL for the legacy default stream). */
ie_status ie_matvec_noalloc(int nx, int ny, int nz, int nrhs, const void *qf_dev, const void *in_scale_dev,
                            const void *out_scale_dev, const void *diag_dev, const void *x_dev, void *y_dev,
                            void *stream);

/* Wait for stream (a cudaStream_t, NULL for the legacy default stream) and report
 * whether a contraction launched by ie_matvec_noalloc since the last call ran out of a
 * bounded wait (IE_ERR_TIMEOUT; the word is cleared) or not (IE_OK).  No allocation. */
ie_status ie_noalloc_sync(void *stream);

/* Generate the compressed real-space coefficient tensor of one frequency on the device
 * (Appendices A-C): the vertical integrals (Ver_Int) of the layered-medium fundamental
 * functions (recursions (pq_req), amplitudes (A_rs), form (UU2)) on a master grid of
 * lambda, uniform in ln(lambda); the lateral cell-to-cell Hankel kernels of (Hor_Int)
 * integrated by Gauss-Legendre panels per offset and mapped onto that grid (the
 * separable structure of the filter of Appendix C); their product; and, for cells
 * whose footprints touch, the quasi-static part in closed form.
 * q_dev: device c128 [Ny][Nx][6][Nz][Nz]; stream: cudaStream_t or NULL.  Synchronous.
 * Supports up to 24 interfaces and Nz <= 256. */
ie_status ie_generate_coefficients(const ie_grid *grid, const ie_layers *layers, double freq, void *q_dev,
                                   void *stream);

/* y = A x (transpose = 0) or y = A^T x (transpose = 1) for instance inst, with nrhs
 * right-hand sides.  dtype selects c64 (IE_C64, the c64 coefficient copy) or c128
 * (IE_C128; IE_C128_DF: c128 vectors and FFTs with the contraction in compensated
 * double-float arithmetic on the FP32 pipe, as in the residuals of the mixed-precision
 * solver: about twice-FP32 accuracy, no counterpart in the paper).
 * x_dev, y_dev: device arrays [nrhs][3][Nz][Ny][Nx] of that type; they must not
 * alias.  stream: a cudaStream_t, or NULL for the context stream.  Asynchronous: a
 * contraction wait that ran out is reported by ie_sync. */
ie_status ie_matvec(ie_ctx *ctx, int inst, const void *x_dev, void *y_dev, int nrhs, int dtype, int transpose,
                    void *stream);

/* Wait for stream (NULL: the context stream) and return IE_ERR_TIMEOUT if a
 * contraction of this context ran out of a bounded wait since the last check (the
 * error word is then cleared), IE_OK otherwise. */
ie_status ie_sync(ie_ctx *ctx, void *stream);

/* In-cell electric field E_n = U_n / a_n, a_n = (sigma_a^n + conj sigma_b^n) / (2 s_n),
 * s_n = sqrt(Re sigma_b^n): the change of variables of eq. (iEH320op) undone for nrhs
 * solutions U (u_dev) into e_dev, both device c128 [nrhs][3][Nz][Ny][Nx] (they may be
 * the same array).  nrhs <= max_rhs.  stream: a cudaStream_t or NULL for the context
 * stream.  Asynchronous. */
ie_status ie_fields(ie_ctx *ctx, const void *u_dev, void *e_dev, int nrhs, void *stream);

/* Solve A u = b for instance inst (Sect. 3.3 (ii): restarted GMRES; classical
 * Gram-Schmidt with a second projection wherever the first one cancels more than
 * 15/16 of the new vector's norm).  precision IE_FP64: c128 vectors and every product
 * with the c128 operator.  IE_MIXED: iterative refinement whose residual uses the c128
 * operator (FP64 vectors and FFTs, double-float contraction) and whose corrections come
 * from GMRES in c64 (c64 operator, c64 Krylov vectors, FP32 rotations; Hessenberg
 * entries and cross-thread sums in FP64).  IE_MIXED_FP64K: the same refinement with the
 * FP64 contraction in the residual and inner GMRES on the c64 operator with FP64 Krylov
 * vectors and FP64 rotations; its Gram-Schmidt dot products and updates of the FP64
 * vectors run in double-float arithmetic (FP32 pairs, about 2^-46 relative to the sum
 * of magnitudes; the Hessenberg entries and norms are FP64).
 * Stops when ||b - A u|| <= tol ||b|| for every right-hand side.
 * b_dev, u_dev: device c128 [nrhs][3][Nz][Ny][Nx]; if use_x0 the initial guess is
 * read from u_dev, otherwise it is zero. */
ie_status ie_solve(ie_ctx *ctx, int inst, const void *b_dev, void *u_dev, int nrhs, double tol, int precision,
                   int use_x0, ie_solve_info *info);

/* Solve the systems of n_inst instances together (a batch over frequencies of one
 * grid): instance inst_host[k] with nrhs right-hand sides (1..4) at block k of
 * b_dev, u_dev (c128 [n_inst][nrhs][3][Nz][Ny][Nx]); n_inst * nrhs <= max_rhs.  One
 * restarted GMRES advances every right-hand side in lockstep, each in its own Krylov
 * space; every product runs the FFT passes once for all of them and one contraction
 * per instance on its slice of the spectrum.  transpose = 1 solves A^T w = b.
 * Otherwise as ie_solve (info: worst residual over all right-hand sides). */
ie_status ie_solve_batch(ie_ctx *ctx, int n_inst, const int *inst_host, const void *b_dev, void *u_dev, int nrhs,
                         double tol, int precision, int use_x0, int transpose, ie_solve_info *info);

/* Contraction variants (no counterpart in the paper): 0 the TMA ring with one slot and
 * two CTAs per SM, 1 the TMA ring with three slots and one CTA per SM (both c64,
 * Nz in {16, 24, 32, 48}, 1-2 right-hand sides), 2 the panel-staged kernel (any case),
 * 3 as 0 with one output row per thread (two right-hand sides), 4 and 5 warp-level
 * TF32 MMAs (mma.sync) with the 3xTF32 split (FP32 accuracy; c64, Nz in {16, 32, 48},
 * 1-2 right-hand sides): 4 a producer warp and a two-slot ring, the fragments read
 * where the copies land; 5 the one-slot ring with an unpacking pass; 6 and 7 the
 * 5th-generation tensor cores (tcgen05.mma with the block in tensor memory; c64,
 * Nz in {16, 32}, 1-2 right-hand sides): 6 kind::tf32 on the 3xTF32 split, 7 kind::f16
 * on a two-way FP16 split of the block and of the vectors, each scaled by a power of two
 * (the same 22 significant bits as 6, half the MMA instructions); 8 the mma.sync path of
 * 5 one Nz x Nz matrix of the block at a time, one matrix staged and unpacked per
 * sub-step (c64, Nz in {16, 32, 48, 64}, 1-2 right-hand sides; the tensor-core variant
 * for Nz = 64).
 * ie_contract_tuning reports the c64 variant used for 1..4 right-hand sides per
 * instance (variant_host[4]; -1: built-in choice) and the autotuner's timings
 * (ms_host[4][9], ms per launch, 0 where not timed; may be NULL).
 * ie_set_contract_variant overrides the choice for one right-hand-side count
 * (-1: built-in choice); IE_ERR_ARG if the variant does not apply to this grid. */
ie_status ie_contract_tuning(ie_ctx *ctx, int *variant_host, double *ms_host);

/* Stage order (radices) of the FFT plan of one axis (0: the 2Nx row transforms, 1: the
 * 2Ny column transforms), used by the mixed-radix Stockham kernels of the c128 product
 * and of every c64 length without a register-blocked kernel (Sect. 3.3, steps 1 and 3).
 * With the autotuner on, ie_setup times the candidate orders of each length (radix-4
 * stages first, radix-8 first, odd factors first, a radix-2 stage first) in the c128
 * forward passes and keeps the fastest.  radix_host: at least 20 ints; *n_stages the
 * count; *ms (may be NULL): the chosen plan's time per pass for one right-hand side
 * (0 if not tuned).  IE_ERR_ARG for an axis other than 0 or 1. */
ie_status ie_fft_plan(ie_ctx *ctx, int axis, int *radix_host, int *n_stages, double *ms);
/* Override the plan of one axis with n_stages radices from {2, 3, 4, 5, 7, 8, 11, 13}
 * whose product is the axis's transform length (2Nx or 2Ny); IE_ERR_ARG otherwise
 * (the plan is left unchanged). */
ie_status ie_set_fft_plan(ie_ctx *ctx, int axis, const int *radix_host, int n_stages);
ie_status ie_set_contract_variant(ie_ctx *ctx, int nrhs, int variant);

/* Solve the transposed system A^T w = b (same arguments as ie_solve).  The
 * transpose uses the complex symmetry B^T = B of Lorentz reciprocity, so
 * A^T = S + R2 B R1. */
ie_status ie_adjoint_solve(ie_ctx *ctx, int inst, const void *b_dev, void *w_dev, int nrhs, double tol,
                           int precision, int use_x0, ie_solve_info *info);

/* Right-hand side U^0 of eq. (slae_matricies) for a magnetotelluric plane wave:
 * the 1-D normal field of the background, normalised by H_y(0) = 1 (x-polarisation,
 * pol = 0) or H_x(0) = -1 (y-polarisation, pol = 1), averaged over every cell and
 * scaled by sqrt(Re sigma_b).  u0_dev: device c128 [3][Nz][Ny][Nx]. */
ie_status ie_rhs_mt(ie_ctx *ctx, int inst, int pol, void *u0_dev);

/* Replace the anomaly conductivities (host, complex interleaved [Nz][Ny][Nx], S/m)
 * without regenerating the coefficient tensors: S, R2 and the per-cell current and
 * gradient factors are rebuilt in place.  Waits for the context's stream first.
 * IE_ERR_GEOMETRY if receivers are set and an anomalous cell would touch their
 * plane (the context keeps its previous conductivities then). */
ie_status ie_set_sigma(ie_ctx *ctx, const double *sigma_a_host);

/* Magnetotelluric receivers: n_rec points at the lateral centres of grid cells
 * (ix_host[r], iy_host[r]), all at depth z_rec with surface <= z_rec <= top of the
 * grid.  Generates on the device, for every instance's frequency, the kernels that
 * give E_x, E_y, H_x, H_y at a receiver from the uniform current of a cell (eq.
 * (APR_lab) with the Green's tensors of eqs. (geh), (green_tensor), (G1G2g), (Ge2):
 * the vertical functions of U_1, U_sigma at the receiver depth and the point-to-cell
 * lateral integrals), and the normal field at z_rec.  Only cells strictly below
 * z_rec radiate; an anomalous cell touching the receiver plane gives
 * IE_ERR_GEOMETRY.  Synchronous. */
ie_status ie_set_receivers(ie_ctx *ctx, int n_rec, const int *ix_host, const int *iy_host, double z_rec);

/* Receivers at arbitrary lateral sites (x_host[r], y_host[r]) in metres, in the grid's
 * frame (cell j spans [x0 + j hx, x0 + (j + 1) hx]), within the grid's lateral extent,
 * all at depth z_rec as for ie_set_receivers (eq. (APR_lab), field recovery at any
 * point outside the domain).  Sites that share their position relative to the cell
 * centres (a profile or map on a lattice of the cell size) share one table of kernels
 * over every receiver-minus-cell offset: c128 [group][2 Ny][2 Nx][Nz][10] per instance,
 * generated on the device, 4 Nx Ny Nz 160 bytes per group.  ie_receiver_fields,
 * ie_mt_misfit and ie_receiver_adjoint then act on these sites.  IE_ERR_ARG for a site
 * outside the grid's extent; IE_ERR_GEOMETRY as for ie_set_receivers.  Synchronous. */
ie_status ie_set_receivers_xy(ie_ctx *ctx, int n_rec, const double *x_host, const double *y_host, double z_rec);

/* The MT maps from impedances: for the n_rec 2 x 2 impedances z_dev (c128 [n_rec][4],
 * as written by ie_mt_misfit) of instance inst, rho_dev[r][k] = |Z_k|^2 / (omega mu0)
 * (apparent resistivity, ohm m) and phase_dev[r][k] = arg Z_k (degrees), k = xx, xy, yx,
 * yy (device FP64 arrays [n_rec][4]).  Synchronous. */
ie_status ie_mt_apparent(ie_ctx *ctx, int inst, const void *z_dev, int n_rec, void *rho_dev, void *phase_dev);

/* Fields at the receivers for nrhs solutions U of instance inst, whose sources are
 * the plane waves pol_host[p] (0: x, 1: y): f_dev c128 [nrhs][n_rec][4] =
 * (E_x, E_y, H_x, H_y), the normal field plus sum over cells of the kernels times the
 * current J = 2 s gamma U (eq. (APR_lab)).  u_dev: c128 [nrhs][3][Nz][Ny][Nx].
 * Synchronous. */
ie_status ie_receiver_fields(ie_ctx *ctx, int inst, const void *u_dev, int nrhs, const int *pol_host, void *f_dev);

/* MT impedance and misfit of one frequency from the fields of its x- and
 * y-polarisation solutions, f_dev c128 [2][n_rec][4] (x first): Z = E H^-1 with
 * E = [[Ex1, Ex2], [Ey1, Ey2]], H = [[Hx1, Hx2], [Hy1, Hy2]] (z_dev c128
 * [n_rec][2][2], row-major), phi_host = 1/2 sum |Z - Zobs|^2 (zobs_dev like z_dev),
 * and the adjoint sources of the misfit, c_dev c128 [2][n_rec][4]: for polarisation
 * j, c^E_i = (H^-1 D^T)_{ji}, c^H_i = -(H^-1 D^T Z)_{ji}, D = conj(Z - Zobs), so that
 * dPhi = Re sum c . d(E_x, E_y, H_x, H_y).  Synchronous. */
ie_status ie_mt_misfit(ie_ctx *ctx, const void *f_dev, const void *zobs_dev, void *z_dev, double *phi_host,
                       void *c_dev);

/* Right-hand sides of the adjoint solves: rhs_dev c128 [nrhs][3][Nz][Ny][Nx] =
 * 2 s gamma (G^T c), the transpose of the receiver operator of instance inst applied
 * to the sources c_dev [nrhs][n_rec][4].  Synchronous. */
ie_status ie_receiver_adjoint(ie_ctx *ctx, int inst, const void *c_dev, int nrhs, void *rhs_dev);

/* grad_dev (double [Nz][Ny][Nx]) += Re sum_p (dgamma/dln sigma_a)(w_p . u_p)/gamma
 * for the anomalous cells (gamma != 0; unchanged elsewhere): the misfit gradient in
 * ln sigma_a from forward solutions u_dev and adjoint solutions w_dev (A^T w = the
 * adjoint right-hand side), both c128 [nrhs][3][Nz][Ny][Nx].  Synchronous. */
ie_status ie_gradient_accumulate(ie_ctx *ctx, const void *u_dev, const void *w_dev, int nrhs, void *grad_dev);

/* The context's CUDA stream (a cudaStream_t). */
void *ie_ctx_stream(ie_ctx *ctx);

/* Bytes of device memory held by the context. */
long long ie_ctx_device_bytes(ie_ctx *ctx);

/* Profiling (no counterpart in the paper).  ie_profile(ctx, 1) clears earlier records
 * and starts recording a pair of CUDA events around every launch of the
 * wavenumber-contraction kernel (step 2 of Sect. 3.3) on the stream it runs on;
 * ie_profile(ctx, 2) also records, in every iteration of the Krylov solver, the
 * operator product, the Gram-Schmidt step and the Givens step; ie_profile(ctx, 0)
 * stops.  ie_profile_read waits for the recorded events and returns the summed
 * duration (ms) and the number of records of one kind: IE_C64 or IE_C128 (the
 * contraction) or one of IE_PROF_*. */
enum {
  IE_PROF_PRODUCT_C64 = 2, IE_PROF_PRODUCT_C128 = 3, IE_PROF_GS_C64 = 4, IE_PROF_GS_C128 = 5, IE_PROF_GIVENS = 6
};
ie_status ie_profile(ie_ctx *ctx, int enable);
ie_status ie_profile_read(ie_ctx *ctx, int dtype, double *total_ms, long long *n_launch);

/* Average duration (ms) of each of the five kernels of one matrix-vector product
 * (row FFT, column FFT, contraction, inverse column FFT, inverse row FFT + scaling),
 * measured with CUDA events over n_iter products on the context's workspaces
 * (values are whatever the workspaces hold).  ms_out_host: 5 doubles. */
ie_status ie_profile_matvec(ie_ctx *ctx, int inst, int nrhs, int dtype, int n_iter, double *ms_out_host);

/* Number of kernels the library has launched in this process (all contexts). */
long long ie_kernel_launches(void);

/* Testing aid (no counterpart in the paper): the number of polls after which the main
 * waits of every contraction launched afterwards give up (a negative value restores the
 * default, 2^28).  0 makes every such wait give up at once, so that the IE_ERR_TIMEOUT
 * path can be exercised without a GPU fault; each kernel still drains its own copies in
 * flight with the default limit before it returns. */
void ie_debug_set_wait_limit(long long polls);

void ie_destroy(ie_ctx *ctx);
const char *ie_status_str(ie_status s);

#ifdef __cplusplus
}
#endif
#endif /* IE_GB300_H */
