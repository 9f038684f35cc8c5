/*
 * voxcap.h -- C ABI of the GB300 (sm_103a) implementation of the VoxCap
 * FFT-accelerated capacitance solver (arxiv 2004.02609).
 *
 * All compute runs in CUDA kernels of libvoxcap.so on the device that is
 * current when voxcap_setup is called.  No call aborts or traps: every entry
 * point returns a status (VOXCAP_OK = 0, negative on error) and
 * voxcap_last_error() returns a thread-local message for the last failure.
 *
 * Units.  voxcap_matvec / voxcap_solve work in the normalised system of the
 * paper's Eq. 4: voxel edge 1, Green's function 1/(4 pi r), panel area 1, so
 * conductor rows read  sum_l P'_kl rho_l = Phi_k  and dielectric rows
 * I'_k rho_k + sum_l E'_kl rho_l = 0.  The physical system at voxel edge dv
 * is this one scaled by dv^3/eps0 (P, Eq. 5) and dv^2/eps0 (E and I, Eqs. 6-7,
 * Appendix C); physical charges are rho = (eps0/dv) rho'.
 * voxcap_capacitance returns farads: C = eps0 * dv * C' (Eq. 8).
 *
 * Panels (Sec. II.A-B).  A face between one conductor voxel and one
 * non-conductor voxel is a conductor panel; a face between two non-conductor
 * voxels of different eps_r is a dielectric panel; outside the grid is vacuum
 * (eps_r = 1).  Every panel normal is the +axis direction: side a is the voxel
 * on the -axis side, side b on the +axis side, and a dielectric panel has
 * I' = (eps_a + eps_b) / (2 (eps_a - eps_b)) (Eq. 7).  Canonical panel order:
 * conductor panels, then dielectric panels (Eq. 4); within each, orientation
 * x < y < z (Eq. 9), then ascending face index, where the x-face (i,j,k),
 * i in [0,N_x], has index i + (N_x+1)(j + N_y k), and likewise for y and z
 * faces.  Vectors are column-major N x nrhs arrays in this order.
 *
 * Pointers.  Arguments documented as "device" must point to device memory
 * of the handle's device (any CUDA allocation, e.g. from PyTorch); "host"
 * arguments are ordinary host memory.  The library copies what it keeps and
 * never retains caller pointers past a call.  All device work is issued on
 * the stream given to voxcap_setup (NULL = legacy default stream) and the
 * calls that return host data synchronise that stream.
 */
#ifndef VOXCAP_H
#define VOXCAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define VOXCAP_OK 0
#define VOXCAP_ERR_ARG (-1)            /* invalid argument */
#define VOXCAP_ERR_SHORT (-2)          /* two different conductors share a face */
#define VOXCAP_ERR_NO_CONDUCTOR (-3)   /* capacitance of a structure without conductors */
#define VOXCAP_ERR_OOM (-4)            /* device allocation failed */
#define VOXCAP_ERR_CUDA (-5)           /* a CUDA call failed */
#define VOXCAP_ERR_NOT_CONVERGED (-6)  /* solver hit its iteration cap; results written */
#define VOXCAP_ERR_UNSUPPORTED (-7)    /* e.g. an FFT length that is not 2/3/5/7-smooth */

/* preconditioners (Sec. II.D, Eq. 14; the last three are the paper's
 * comparison cases of Sec. III.A) */
#define VOXCAP_PRECOND_BDD 0    /* block-diagonal on conductor rows, 1/I' on dielectric rows */
#define VOXCAP_PRECOND_BD 1     /* conventional block-diagonal over all panels of a box */
#define VOXCAP_PRECOND_DIAG 2   /* 1/A_kk */
#define VOXCAP_PRECOND_NONE 3

/* solver precision */
#define VOXCAP_FP64 0            /* plain FP64 GMRES with FP64 FFT products */
#define VOXCAP_FP32_REFINE 1     /* FP32 GMRES / FP32 FFT products inside FP64 iterative refinement */

/* precision of the generated Toeplitz entries (voxcap_opts.entries) */
#define VOXCAP_ENTRIES_AUTO 0    /* FP32 far field under VOXCAP_FP32_REFINE when the permittivity
                                    contrast (max/min eps_r of the dielectric labels and the vacuum
                                    outside) is at most 1e4, else FP64 */
#define VOXCAP_ENTRIES_FP64 1    /* every entry in FP64 (near-field closed forms, far-field quadrature) */
#define VOXCAP_ENTRIES_FAR32 2   /* near-field closed forms in FP64, far-field quadrature sums in FP32
                                    (entries to about 1e-7 relative, the FP32 products' accuracy);
                                    the kernel spectra are then transformed in FP32 as well and the
                                    FP64 products use their widening.  At high contrast the dielectric
                                    rows' I' + E' nearly cancel and amplify entry errors by about the
                                    contrast: FAR32 is meant for contrasts up to about 1e4 */

/* dtypes of voxcap_matvec */
#define VOXCAP_F32 0
#define VOXCAP_F64 1

/* voxcap_matvec flags */
#define VOXCAP_MV_PRECOND 1      /* y = R (A x) with the configured preconditioner R (Eq. 14) */
#define VOXCAP_MV_ADJOINT 2      /* y = A^T x */
#define VOXCAP_MV_RONLY 4        /* y = R x (no product with A) */

typedef struct voxcap voxcap_t;

/*
 * voxcap_tucker -- Tucker-compressed canonical Toeplitz tensors (Eq. 13,
 * Sec. II.C), produced once at installation (paper_2004_02609_gb300/tucker.py)
 * in normalised units.  Tensor t:
 *   0  Ppar[h][s][t]  potential of parallel panels, offsets (h, s, t)
 *   1  Epar[h][s][t]  its derivative along the normal offset h
 *   2  Port[a][b][c]  potential of orthogonal panels at offsets
 *                     (a + 1/2, b + 1/2, c): test normal, source normal, shared axis
 *   3  Eort[a][b][c]  its derivative along the test normal
 * X ~ core x1 U1 x2 U2 x3 U3 with core[r1][r2][r3] (last index fastest) and
 * factor[t][n] a dims[t][n] x ranks[t][n] row-major matrix; all host memory,
 * copied during voxcap_setup.  Every dims[t][n] must be >= max(nx, ny, nz) + 1.
 */
typedef struct voxcap_tucker {
  int dims[4][3];
  int ranks[4][3];
  const double* core[4];
  const double* factor[4][3];
} voxcap_tucker;

typedef struct voxcap_opts {
  int precision;       /* VOXCAP_FP64 or VOXCAP_FP32_REFINE (default) */
  int restart;         /* GMRES restart length (default 35, Sec. III; at most 512) */
  double inner_tol;    /* FP32 inner GMRES: tightest relative tolerance of one refinement sweep
                          (default 1e-4); a sweep stops earlier when that already meets tol */
  int max_iters;       /* cap on GMRES iterations per solve (default 2000) */
  int max_sweeps;      /* cap on refinement sweeps (default 20) */
  int nv[3];           /* small-box size of the preconditioner in voxels (default 10, Sec. II.D) */
  int precond;         /* VOXCAP_PRECOND_* (default BDD) */
  int pad_mode;        /* padded FFT length per axis, all >= 2N+1 (Appendix B):
                          0: the cheapest even 2/3/5/7-smooth length within 25% by
                             the FFT engine's cost model (default);
                          1: the paper's M = 2(N+1) (must be 2/3/5/7-smooth);
                          2: the smallest even 2/3/5/7-smooth length */
  int entries;         /* VOXCAP_ENTRIES_* (default AUTO): precision of the generated entries */
  const voxcap_tucker* tucker; /* NULL: generate the Toeplitz tensors (Eqs. 5-6, precision
                          per `entries`); else restore them from these Tucker
                          factors on the tensor cores (Sec. II.C), cropped to the grid */
  int fast_refine;     /* FP32_REFINE only.  0 (default): FP64 in every refinement residual and
                          in the Arnoldi orthogonalisation's arithmetic.  1: FP32 arithmetic
                          for the FP32 basis's Gram-Schmidt updates and each lane's partial dot
                          product (FP64 from the lane sums on), and an FP32 product for the
                          residual of a column whose last sweep only had to reach a relative
                          residual >= 1e-5; convergence is still decided on FP64 residuals.
                          Faster on GPUs with slow FP64; C to about 1e-7 of the FP64 solve. */
} voxcap_opts;

typedef struct voxcap_stats {
  int iterations;          /* total GMRES iterations (all sweeps) */
  int sweeps;              /* refinement sweeps (1 for plain FP64) */
  int matvecs;             /* products with A issued (all precisions) */
  int converged;           /* 1 if every right-hand side met tol */
  double rel_residual;     /* max over RHS of ||b - A x||_2 / ||b||_2 in FP64 */
  double seconds;          /* wall time of the call */
} voxcap_stats;

/* Fill *o with the defaults listed above. */
void voxcap_default_opts(voxcap_opts* o);

/* Thread-local message of the last failed call ("" if none). */
const char* voxcap_last_error(void);

/*
 * voxcap_setup -- build everything the iterative solution needs (Sec. II):
 * panels from the voxel labels (Sec. II.A-B), the block-Toeplitz tensors of
 * Eqs. 5-6 on the device (Appendix A-B; near field in FP64, far field in FP32
 * or FP64 as opts->entries selects) or restored from Tucker factors, their
 * block-circulant embedding and its FFT (Eqs. 11-12, Appendix B), and the
 * preconditioner (Eq. 14; blocks of up to 224 panels are inverted in FP32,
 * larger ones in FP64).  The first set-up of a grid shape and batch in a
 * process also times the launch variants of the FP32 product on its own
 * products and keeps the fastest (see voxcap_set_product_tiles); later
 * set-ups of that shape reuse the choice.
 *
 *  labels       [n_struct][nz][ny][nx] int32, x fastest; host or device
 *               (detected with cudaPointerGetAttributes).  Each entry is a
 *               material label in [0, n_labels).
 *  n_struct     number of independent structures sharing one grid shape
 *               and one material table; they share the FFT'd kernel tensors
 *               and are solved as one batch (>= 1).
 *  conductor_id host [n_labels]: conductor index >= 0, or -1 for a dielectric
 *  eps_r        host [n_labels]: relative permittivity (> 0; ignored for conductors)
 *  voxel_size_m voxel edge in metres (> 0), used only for farads.
 *  opts         NULL for defaults.
 *  cuda_stream  cudaStream_t to issue all work on (NULL = default stream).
 *  out          receives the handle; free it with voxcap_destroy.
 * Errors: VOXCAP_ERR_ARG (bad sizes/labels), VOXCAP_ERR_SHORT, VOXCAP_ERR_OOM,
 * VOXCAP_ERR_CUDA, VOXCAP_ERR_UNSUPPORTED (pad_mode 1 with a non-smooth 2(N+1)).
 */
int voxcap_setup(const int32_t* labels, int nx, int ny, int nz, int n_struct,
                 const int32_t* conductor_id, const double* eps_r, int n_labels,
                 double voxel_size_m, const voxcap_opts* opts, void* cuda_stream,
                 voxcap_t** out);

/* Release every device buffer of the handle.  NULL is ignored. */
void voxcap_destroy(voxcap_t* h);

/*
 * voxcap_num_panels -- sizes of structure s (0 <= s < n_struct): conductor
 * panels, dielectric panels, conductors.  n_total (may be NULL) receives the
 * handle's total panel count N over all structures; structure s occupies
 * rows [offset, offset + n_cond + n_diel) with offset written to *offset
 * (may be NULL).
 */
int voxcap_num_panels(const voxcap_t* h, int s, int64_t* n_cond, int64_t* n_diel,
                      int* n_conductors, int64_t* n_total, int64_t* offset);

/*
 * voxcap_panel_map -- the panels of structure s in canonical order (host
 * outputs, n_cond + n_diel entries each; any pointer may be NULL):
 * orientation (0/1/2 = normal along x/y/z), face index in that orientation's
 * face grid, kind (0 conductor, 1 dielectric), owner conductor (-1 for
 * dielectric), I' of Eq. 7 (0 for conductor panels), free-charge factor
 * eps_r of the conductor panel's non-conductor side (0 for dielectric).
 */
int voxcap_panel_map(const voxcap_t* h, int s, int8_t* orient, int32_t* face_idx,
                     int8_t* kind, int16_t* owner, double* idiag, double* qscale);

/*
 * voxcap_matvec -- y = A x for nrhs columns (Eqs. 9-11) by the FFT method:
 * scatter onto the x/y/z face grids, zero-padded 3-D FFTs, products with the
 * 15 FFT'd block-circulant kernels (Eq. 12 folds P^yx, P^zx, P^zy into
 * P^xy, P^xz, P^yz), inverse FFTs and gather; dielectric rows add I' x.
 *  x_dev, y_dev  device, N x nrhs column-major, float (VOXCAP_F32) or double
 *                (VOXCAP_F64); N = total panels of the handle; must not alias.
 *  flags         VOXCAP_MV_PRECOND: y = R A x; VOXCAP_MV_ADJOINT: y = A^T x;
 *                VOXCAP_MV_RONLY: y = R x.
 */
int voxcap_matvec(voxcap_t* h, const void* x_dev, void* y_dev, int nrhs, int dtype,
                  int flags);

/*
 * voxcap_matvec_noalloc -- the same product as voxcap_matvec (same arguments,
 * flags and results) for callers that must not allocate device memory while
 * they run.  The paper has no counterpart: this is a deployment variant.
 *
 * Who needs it: voxcap_matvec keeps its FFT intermediates in a workspace the
 * handle allocates on first use (and grows for larger nrhs), and its
 * VOXCAP_MV_PRECOND form allocates a temporary on every call.  Callers that
 * run on a fixed device-memory budget fixed at start-up, callers whose device
 * memory is owned by another allocator, and latency-critical loops that
 * cannot afford the implicit device synchronisation of cudaMalloc / cudaFree
 * cannot accept that.  This entry point calls no cudaMalloc, cudaFree or
 * allocating library routine: its scratch is one fixed 16 MiB array in the
 * library's device image.  A device holds it from the first call on that
 * device (which loads the library's device module, array included) until
 * the process exits.
 *
 * Limits and sharing: a call whose scratch would exceed 16 MiB (it grows with
 * the padded grid and with nrhs) is rejected with VOXCAP_ERR_ARG and a message
 * giving the bytes it needs; use voxcap_matvec or fewer columns then.  All
 * calls on one device share the array and it keeps the last call's contents;
 * every element a call reads is written earlier in the same call, so nothing
 * has to start at zero.  Calls that overlap on the GPU (issued on different
 * streams or from different threads without ordering) race on the array.
 * Every call looks up the array's device address with the handle's device
 * current; the first call on a device also loads the module there (a set-up
 * step), so make that first call before any stream capture.
 */
int voxcap_matvec_noalloc(voxcap_t* h, const void* x_dev, void* y_dev, int nrhs, int dtype,
                          int flags);

/*
 * voxcap_solve -- solve A X = B (Eq. 4) for nrhs right-hand sides by
 * left-preconditioned GMRES(restart) (Eq. 14, Sec. III), in plain FP64 or in
 * FP32 inside FP64 iterative refinement per opts->precision, until
 * ||b - A x||_2 <= tol ||b||_2 for every column.
 *  B_dev, X_dev  device double, N x nrhs column-major; X is overwritten.
 *  st            may be NULL.
 * Returns VOXCAP_ERR_NOT_CONVERGED (with X and st written) at the caps.
 */
int voxcap_solve(voxcap_t* h, const double* B_dev, int nrhs, double tol, double* X_dev,
                 voxcap_stats* st);

/*
 * voxcap_capacitance -- capacitance matrices (Eq. 8): one unit-potential
 * solve per conductor, all conductors of all structures in one batch, then
 * C_ij = eps0 dv sum_{k in conductor i} eps_r(k) rho'_jk (free-charge scaling
 * of conductors embedded in a dielectric).
 *  C_host   host double: the m_s x m_s row-major matrices of the structures
 *           back to back (sum over s of m_s^2 values).
 *  rho_dev  optional device double N x m_max (NULL: not returned), the charges
 *           of each unit-potential solve (column j = conductor j of each
 *           structure; zero columns for structures with fewer conductors).
 */
int voxcap_capacitance(voxcap_t* h, double tol, double* C_host, double* rho_dev,
                       voxcap_stats* st);

/*
 * voxcap_capacitance_columns -- columns j0 .. j1-1 of the capacitance
 * matrices (Eq. 8): the unit-potential solves of conductors j0 .. j1-1 only,
 * in one batch.  A column's solve does not depend on which other columns
 * share its batch (every reduction is summed in an order fixed by N, every
 * column keeps its own tolerances), so column blocks computed apart -- on
 * several GPUs, each with its own handle of the same structure -- assemble
 * into the matrix voxcap_capacitance returns, bit for bit (the multi-GPU
 * sharding of conductors).
 *  C_host  host double: for each structure the m x (j1-j0) row-major block
 *          (rows = all conductors i, columns = conductors j0 .. j1-1), back
 *          to back.
 * Returns VOXCAP_ERR_ARG for a range outside [0, m) and the codes of
 * voxcap_capacitance.  Does not enable voxcap_capacitance_grad unless the
 * range covers every conductor.
 */
int voxcap_capacitance_columns(voxcap_t* h, double tol, int j0, int j1, double* C_host, voxcap_stats* st);

/*
 * voxcap_capacitance_grad -- dL/d eps_r[label] for L = sum_s sum_ij
 * dL_dC[s][i][j] C_s,ij, by one batched adjoint solve A^T mu = W dL_dC that
 * reuses the FFT'd kernels (conjugated), the forward charges of the last
 * voxcap_capacitance call and the panel fields at every face.  Faces whose
 * two sides have equal permittivity contribute through the limit of the
 * dielectric row as I' -> infinity.
 *  dL_dC_host   host double, same layout as C_host.
 *  grad_host    host double [n_labels] (conductor labels get 0).
 * voxcap_capacitance must have been called on this handle first.
 */
int voxcap_capacitance_grad(voxcap_t* h, const double* dL_dC_host, double tol,
                            double* grad_host, voxcap_stats* st);

/*
 * voxcap_update_eps -- replace the permittivity table (host [n_labels]) and
 * rebuild the panels and the preconditioner; the FFT'd kernel tensors, which
 * do not depend on eps (Eqs. 5-6), are kept.
 */
int voxcap_update_eps(voxcap_t* h, const double* eps_r);

/*
 * voxcap_entries -- Galerkin integrals of single panel pairs, evaluated by
 * the device entry generator (FP64): kind 0 = P' (Eq. 5), 1 = E' (Eq. 6),
 * normalised units.  All arrays are device memory of n entries:
 *  kind, test_orient, src_orient  int32
 *  d                              double [n][3], test centre - source centre
 *                                 (each component an integer or half-integer
 *                                 as on the voxel lattice)
 *  out                            double [n]
 * The stream is the legacy default stream; the call synchronises it.
 */
int voxcap_entries(int n, const int32_t* kind, const int32_t* test_orient,
                   const int32_t* src_orient, const double* d, double* out);

/*
 * voxcap_tucker_expand -- X = S x1 U1 x2 U2 x3 U3 (Eq. 13) on the tensor cores
 * (tcgen05, TF32 hi/lo split, FP32 accumulation): the restoration step of
 * Sec. II.C.  Device arrays: core [r1][r2][r3] (last index fastest),
 * U1 [D1][r1], U2 [D2][r2], U3 [D3][r3] row-major, out [D3][D2][D1] (first
 * index fastest: out[i + D1 (j + D2 k)]).  Legacy default stream; synchronises.
 * Returns VOXCAP_ERR_CUDA if the tensor cores do not complete within a bound.
 */
int voxcap_tucker_expand(const double* core, int r1, int r2, int r3, const double* U1, int D1,
                         const double* U2, int D2, const double* U3, int D3, double* out);

/*
 * voxcap_canonical_tensors -- the four canonical Toeplitz tensors of
 * voxcap_tucker on a D x D x D index cube, generated in FP64 on the device
 * (Eqs. 5-6, Appendix A-B): the installation-stage input of the Tucker
 * compression.  Each output is device double [D][D][D] (first index fastest);
 * any pointer may be NULL.  Legacy default stream; synchronises.
 */
int voxcap_canonical_tensors(int D, double* ppar, double* epar, double* port, double* eort);

/*
 * voxcap_fft_length -- the padded FFT length the handle uses along each axis
 * (M_x, M_y, M_z >= 2 N + 1, Appendix B).  Any pointer may be NULL.
 */
int voxcap_fft_length(const voxcap_t* h, int* mx, int* my, int* mz);

/*
 * voxcap_toeplitz -- copy one FP64 block-Toeplitz tensor of the handle to
 * host memory (Appendix B).  Tensor index t: 0..5 = P^xx, P^yy, P^zz, P^xy,
 * P^xz, P^yz; 6..14 = E^xx, E^yy, E^zz, E^xy, E^xz, E^yz, E^yx, E^zx, E^zy
 * (superscript = test orientation, source orientation).  Entry (ex,ey,ez),
 * ex fastest, holds the integral for the centre difference whose absolute
 * value along each axis is e (integer axes) or e + 1/2 (the test normal axis
 * and the source normal axis of an orthogonal pair), the sign taken positive.
 * dims (may be NULL) receives the three extents; out may be NULL to query.
 */
int voxcap_toeplitz(const voxcap_t* h, int t, double* out_host, int* dims);

/*
 * voxcap_launch_count -- number of CUDA kernel launches this process has
 * issued through the library so far (a diagnostic counter with no
 * counterpart in the paper; benchmarks read it before and after a timed
 * region).
 */
int64_t voxcap_launch_count(void);

/*
 * voxcap_set_product_tiles -- choose the launch variant of the handle's FP32
 * products (an implementation choice with no counterpart in the paper; the
 * z pass is the z transform, spectral multiply-accumulate of Eqs. 11-12 and
 * inverse z transform of one product, the y passes the transforms along y).
 * z_order: 0 = the z transform's largest radix <= 9 last, 1 = its smallest
 * radix last (ignored when both orders coincide); z_tile_log2: log2 of the
 * z pass's columns per CTA, 0..4 (a width that does not fit falls back to
 * the widest that does); y_fwd_log2 / y_inv_log2: log2 of the forward /
 * inverse y passes' columns per CTA, 0..4, or -1 for the default width.
 * z_order = -1 re-runs the set-up autotuner, which times the variants on
 * this handle's own products and keeps the fastest (its choice is cached per
 * device, grid and batch); z_order = -2 changes nothing (query); the other
 * arguments are then ignored.
 * choice_out (may be NULL) receives {z_order, z_tile_log2, y_fwd_log2,
 * y_inv_log2} in force.  Forcing a variant (z_order >= 0) selects the
 * generic passes (product path 0, see voxcap_set_product_path).  Returns
 * VOXCAP_ERR_ARG for a NULL handle or an out-of-range argument.  Not safe
 * while another call on the same handle runs.
 */
int voxcap_set_product_tiles(voxcap_t* h, int z_order, int z_tile_log2, int y_fwd_log2, int y_inv_log2,
                             int* choice_out);

/*
 * voxcap_setup_times -- wall seconds of the phases of the handle's
 * voxcap_setup (the paper reports its set-up stages the same way, Table V):
 * seconds[0] input copies and FFT plans, [1] panels (Sec. II.A-B), [2] the
 * block-Toeplitz tensors, generated (Eqs. 5-6) or restored from Tucker
 * factors (Eq. 13), [3] circulant embedding and kernel spectra (Eqs. 11-12),
 * [4] preconditioner (Eq. 14), [5] autotuning of the products (zero when the
 * choice was cached).  seconds: host, 6 doubles.  Returns VOXCAP_ERR_ARG for
 * NULL arguments.
 */
int voxcap_setup_times(const voxcap_t* h, double* seconds);

/*
 * voxcap_set_product_path -- which kernels run the handle's FP32 products
 * (Eqs. 9-12; an implementation choice, same results to rounding).  The
 * FP64 products do not depend on it: they use the compiled persistent y
 * passes wherever the y length has a compiled plan and the generic passes
 * otherwise.
 *  path 0   the generic passes (any padded length);
 *  path 1   passes compiled for fixed radix plans wherever the padded length
 *           of an axis has one (x and y: 36, 72, 144, 288, 576, 1152; z: 36,
 *           72, 144; forward z pass only), the generic passes elsewhere, each
 *           in its default launch variant;
 *  path 1 + variant bits: 2 = the persistent z pass with asynchronous
 *           prefetch of the next tile (z length 144), 4 / 8 = the persistent
 *           forward / inverse y pass, double-buffered with asynchronous
 *           prefetch (compiled y lengths); a bit that does not apply to the
 *           handle's lengths changes nothing.
 *           The variants of path 1 differ in tiling only: every line is
 *           transformed with the same arithmetic, so they give the same bits;
 *  path -1  re-run the set-up autotuner, which times the generic variants,
 *           path 1 and its variant bits on this handle's own products and
 *           keeps the fastest (cached per device, grid and batch);
 *  path -2  change nothing (query).
 *  path_out (may be NULL) receives the path in force, with its variant bits.
 * Returns VOXCAP_ERR_ARG for a NULL handle or a path outside -2..15 or even
 * and above 1.  Not safe while another call on the same handle runs.
 */
int voxcap_set_product_path(voxcap_t* h, int path, int* path_out);

#ifdef __cplusplus
}
#endif
#endif /* VOXCAP_H */
