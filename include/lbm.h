/*
 * lbm.h -- C ABI of liblbm, a GB300 (sm_103a) implementation of the fused
 * stream-and-collide update of the recursive Hermite-regularized lattice
 * Boltzmann method (rrBGK) of Brogi, Malaspinas, Chopard and Bonadonna,
 * "Hermite regularization of the lattice Boltzmann method for open source
 * computational aeroacoustics", arXiv:1710.02065.
 *
 * The problem the library solves is the one of Sec. II: given a lattice
 * (D2Q9 or D3Q19), a box of cells, a relaxation time tau (or a viscosity
 * nu = c_s^2 (tau - 1/2), Sec. II.A) and the boundary treatment of Sec. III
 * (bounce-back walls, velocity inflow, zero-gradient outflow, absorbing
 * sponge layers of Sec. II.C), advance the populations f_i in time with
 *     f_i(x + xi_i, t + 1) = feqH_i(x, t) + (1 - 1/tau) fneqH_i(x, t)
 * (Eq. optimizedLB; Eq. spongeLB inside sponge layers).
 *
 * Conventions shared by every entry point
 *   - Lattice units: dx = dt = 1, c_s^2 = 1/3.
 *   - Cells are numbered x fastest: cell = x + nx * (y + ny * z); a 2D
 *     lattice has nz = 1.
 *   - Directions follow the order reported by lbm_lattice_table(): 0 is the
 *     rest velocity; directions 1..Q/2 and Q/2+1..Q-1 are opposite pairs
 *     (opp(i) = i + Q/2 for 1 <= i <= Q/2).
 *   - Population arrays exchanged with the caller are plain (unshifted) f_i
 *     in FP64, direction-major: f[i * ncell + cell].
 *   - The state held by a handle is the post-collision field after the last
 *     step (after lbm_set_state / lbm_set_populations: the field given).
 *     One step pulls f_i(x) = f*_i(x - xi_i), applies the boundary rules and
 *     collides.  Moments reported by lbm_moments / lbm_reduce / lbm_probe are
 *     those of this stored field.
 *   - Host buffers passed in are only read during the call; the caller keeps
 *     ownership.  Output buffers are caller-allocated.  Device memory is
 *     owned by the handle and released by lbm_destroy.
 *   - All work is enqueued on the CUDA stream given to lbm_create.  Calls that
 *     return data to the host synchronise that stream; lbm_step does not
 *     (launch errors are returned at once, execution errors at the next
 *     synchronising call).
 *   - Every function returns LBM_OK (0) or a negative LBM_E* code; the
 *     message of the last failure is available from lbm_last_error().
 *   - A handle must not be used from two host threads at once.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx *lbm_handle;

/* Return codes */
#define LBM_OK 0
#define LBM_EINVAL (-1)    /* invalid argument or unsupported combination      */
#define LBM_ENOMEM (-2)    /* device or host allocation failed                  */
#define LBM_ECUDA (-3)     /* a CUDA call failed (message has the CUDA error)   */
#define LBM_EUNSTABLE (-4) /* unstable cells found by lbm_reduce (non-finite, rho <= 0, |u| >= c_s) */
#define LBM_EIO (-5)       /* file error in lbm_save / lbm_load                 */

/* Lattices (Sec. II.A: D2Q9 in 2D, D3Q19 in 3D).  LBM_D3Q27, the tensor
 * product of D1Q3, carries the complete third-order Hermite set (the six
 * H_aab and H_xyz) that D3Q19 can only keep as pairs; general and two-cell
 * kernels, refinement patches and the solve server. */
#define LBM_D2Q9 0
#define LBM_D3Q19 1
#define LBM_D3Q27 2

/* Storage precision of the populations.  FP64 computes in FP64; the others
 * compute in FP32.  The *_SHIFTED formats store f_i - w_i (rho_0 = 1). */
#define LBM_FP64 0
#define LBM_FP32 1
#define LBM_FP16_SHIFTED 2
#define LBM_BF16_SHIFTED 3

/* Faces of the box */
#define LBM_FACE_XM 0
#define LBM_FACE_XP 1
#define LBM_FACE_YM 2
#define LBM_FACE_YP 3
#define LBM_FACE_ZM 4
#define LBM_FACE_ZP 5

/* Boundary kinds of a face (Sec. III) */
#define LBM_BC_PERIODIC 0 /* wrap-around; both faces of an axis must be periodic */
#define LBM_BC_VELOCITY 1 /* Dirichlet velocity inflow                          */
#define LBM_BC_OUTFLOW 2  /* zero-gradient outflow for all populations           */
#define LBM_BC_FREESLIP 3 /* free-slip wall (no normal flow, no shear)          */
#define LBM_BC_PRESSURE 4 /* constant pressure (density), see lbm_set_pressure */

/* Cell types for lbm_set_geometry */
#define LBM_CELL_FLUID 0
#define LBM_CELL_SOLID 1 /* halfway bounce-back wall */
#define LBM_CELL_FIXED 2 /* populations held fixed (set by the caller or by a
                            coupling step); streamed from like a fluid cell */

/*
 * lbm_lattice_table -- velocities and weights of a lattice (host only, no GPU
 * needed).  Sec. II.A, Eq. truncatedEq ("w_i ... specific to the lattice").
 *   q, d : out, number of directions and dimensions (may be NULL)
 *   xi   : out, q*3 ints, xi[3*i + a] (may be NULL)
 *   w    : out, q doubles (may be NULL)
 * Returns LBM_EINVAL for an unknown lattice.
 */
int lbm_lattice_table(int lattice, int *q, int *d, int *xi, double *w);

/*
 * lbm_create -- allocate a lattice of extents[0] x extents[1] x extents[2]
 * cells on the current CUDA device, fully periodic, every cell fluid and at
 * rest (rho = 1, u = 0).
 *   lattice     : LBM_D2Q9 (extents[2] must be 1), LBM_D3Q19 or LBM_D3Q27
 *                 (the tensor-product lattice with the complete third order)
 *   tau_or_nu   : relaxation time tau (> 1/2) or, if value_is_nu != 0, the
 *                 kinematic viscosity nu > 0, tau = nu / c_s^2 + 1/2
 *                 (Sec. II.A, below Eq. truncatedEq)
 *   Ma_ref      : reference Mach number, 0 <= Ma_ref <= 0.6 (the paper reports
 *                 stable runs up to Ma 0.6, Sec. V); informational, it sets
 *                 U_ref = Ma_ref c_s reported by lbm_info
 *   precision   : LBM_FP64, LBM_FP32, LBM_FP16_SHIFTED or LBM_BF16_SHIFTED
 *   cuda_stream : cudaStream_t to enqueue work on, or NULL for the legacy
 *                 default stream
 * Errors: LBM_EINVAL (extents < 1, extents[1] or extents[2] > 65535, more
 * than 2^31 - 1 cells; tau <= 1/2; bad lattice/precision; Ma_ref outside
 * [0, 0.6]; a non-periodic axis needs >= 3 cells, checked at lbm_step),
 * LBM_ENOMEM, LBM_ECUDA.  On error *out is NULL.
 */
int lbm_create(lbm_handle *out, int lattice, const int extents[3], double tau_or_nu,
               int value_is_nu, double Ma_ref, int precision, void *cuda_stream);

/* lbm_destroy -- free the handle and its device memory (NULL is ignored). */
void lbm_destroy(lbm_handle h);

/* lbm_last_error -- message of the last failed call on h (h may be NULL for
 * failures of lbm_create).  The string lives until the next call on h. */
const char *lbm_last_error(lbm_handle h);

/*
 * lbm_set_geometry -- cell types, ncell bytes (LBM_CELL_FLUID / LBM_CELL_SOLID /
 * LBM_CELL_FIXED), host memory; NULL removes all solids.  Solid cells are
 * walls with halfway bounce-back (Sec. III: the paper's cylinder and pipe
 * walls): a population that would stream out of a solid cell is replaced by
 * the receiving cell's own post-collision population in the opposite
 * direction.  Solid and fixed cells keep their stored populations unchanged;
 * fixed cells are streamed from like fluid cells.  lbm_reduce counts fluid
 * cells only.
 */
int lbm_set_geometry(lbm_handle h, const uint8_t *cell_type);

/*
 * lbm_set_boundary -- boundary rule of one face (Sec. III).
 *   face      : LBM_FACE_*
 *   kind      : LBM_BC_PERIODIC, LBM_BC_VELOCITY or LBM_BC_OUTFLOW.  Both faces
 *               of an axis are periodic or neither is; a non-periodic axis
 *               needs at least 3 cells.
 *   u_in      : velocity of a LBM_BC_VELOCITY face (3 doubles; may be NULL if
 *               u_profile is given)
 *   u_profile : optional per-face-cell velocity, 3 doubles per face cell,
 *               face cells numbered by the two tangential coordinates, the
 *               lower axis fastest (x faces: y + ny z; y faces: x + nx z;
 *               z faces: x + nx y).  Replaces u_in when given.
 * Velocity node: rho and Pi^neq are taken from the streamed populations of
 * the inward neighbour and the node is rebuilt as feqH(rho, u_in) +
 * fneqH(u_in, Pi^neq) before the collision.  Outflow node: takes all
 * streamed populations of the inward neighbour (zero gradient), then collides.
 * Free-slip node (Sec. III: lateral boundaries, zero gradient of the
 * tangential velocity): rho, u and Pi^neq of the inward neighbour with the
 * normal velocity and the normal-tangential Pi^neq set to zero, rebuilt the
 * same way.  A node on several faces takes the first non-outflow face in the
 * order -x, +x, -y, +y, -z, +z.
 */
int lbm_set_boundary(lbm_handle h, int face, int kind, const double u_in[3],
                     const double *u_profile);

/*
 * lbm_set_pressure -- constant-pressure face (Sec. IV: the jet's right
 * boundary): p = c_s^2 rho_out imposed; the node takes u and Pi^neq of its
 * inward neighbour (zero gradient) and is rebuilt as feqH(rho_out, u) +
 * fneqH(u, Pi^neq) before the collision.  rho_out > 0.
 */
int lbm_set_pressure(lbm_handle h, int face, double rho_out);

/*
 * lbm_set_inlet_noise -- seeded random perturbation of velocity-face nodes.
 * At step t, face cell k, component a < d, a node with prescribed velocity
 * u (|u| > 0) gets u_a + amplitude |u| (2 U - 1) with
 * U = (splitmix64(seed * 2^32 + (t * n_face_cells + k) * 3 + a) >> 11) * 2^-53
 * (splitmix64 of Steele, Lea and Flood 2014).  amplitude = 0 disables it.
 */
int lbm_set_inlet_noise(lbm_handle h, uint64_t seed, double amplitude);

/*
 * lbm_set_sponge -- absorbing layer of width cells along a face (Sec. II.C,
 * Eq. spongeLB with the damping term Eq. dampingLBM).  In the layer,
 * chi(x) = chi_max sigma(d), sigma(d) = 3125 (W - d) d^4 / (256 W^5), d the
 * distance of the cell from the layer's inner edge (W = width); overlapping
 * layers take the larger chi.  The damped moments are rho* = (rho + chi
 * rho_ref / 2) / (1 + chi / 2), rho* u* = (j + chi rho_ref u_ref / 2) /
 * (1 + chi / 2).  Stability needs chi_max < 4 tau (Sec. II.C); larger values
 * are rejected.  The reference state (rho_ref, u_ref) is shared by all
 * layers: a call with a reference different from an earlier layer's is
 * rejected.  width = 0 removes the layer.
 */
int lbm_set_sponge(lbm_handle h, int face, int width, double chi_max, double rho_ref,
                   const double u_ref[3]);

/*
 * lbm_set_radial_sponge -- circular (D2Q9) or spherical (D3Q19) absorbing
 * layer (Sec. III: the cylinder's sponge is circular and covers the corners
 * of the domain): with r the distance of a cell from center and d = r - r0,
 * chi = chi_max sigma(d) (the profile of lbm_set_sponge, width W = width) for
 * 0 <= d < 0.8 W, and chi = chi_max (the profile's maximum) for d >= 0.8 W, so
 * the corners beyond the circle are damped at full strength.  Combined with
 * planar layers by taking the larger chi; shares their reference state.
 * width = 0 removes it.  Errors as lbm_set_sponge.
 */
int lbm_set_radial_sponge(lbm_handle h, const double center[3], double r0, double width,
                          double chi_max, double rho_ref, const double u_ref[3]);

/*
 * lbm_set_state -- initialise every cell to feqH(rho, u) (Eq. eqH).
 *   rho : ncell doubles; u : 3*ncell doubles, per cell (ux, uy, uz) (host).
 * Resets the step counter to 0.  The values are checked on the device while
 * the field is written: LBM_EINVAL names the first cell whose rho is not
 * finite and > 0 (or, 2D, whose u_z is not 0), and the field is then
 * unspecified until it is set again.
 * Page-locked host arrays (cudaHostAlloc / cudaMallocHost, or registered with
 * cudaHostRegister, e.g. pinned torch tensors) are read by the kernel
 * directly over the host link in one pass; pageable arrays are copied through
 * the handle's staging buffer (lbm_set_transfer_staging).  Same values either
 * way.
 */
int lbm_set_state(lbm_handle h, const double *rho, const double *u);
/* The same with FP32 host arrays (half the host-link bytes), for FP32 and
 * 16-bit storage whose populations carry no more than FP32 precision. */
int lbm_set_state_f32(lbm_handle h, const float *rho, const float *u);

/* lbm_set_populations / lbm_get_populations -- the full stored field as plain
 * FP64 f_i, direction-major, q*ncell doubles (host).  set resets the step
 * counter to 0; get synchronises the stream. */
int lbm_set_populations(lbm_handle h, const double *f);
int lbm_get_populations(lbm_handle h, double *f);

/*
 * lbm_step -- advance n >= 0 time steps: stream (pull), apply the boundary
 * rules, collide with Eq. optimizedLB / Eq. spongeLB.  Asynchronous.
 */
int lbm_step(lbm_handle h, int64_t n);

/*
 * lbm_moments -- moments of the stored field (host outputs, any may be NULL):
 *   rho    : ncell doubles, sum_i f_i                       (Eq. moments)
 *   u      : 3*ncell doubles, (sum_i f_i xi_i) / rho        (Eq. moments)
 *   pi_neq : 6*ncell doubles, Pi - rho c_s^2 I - rho u u, Pi = sum_i f_i xi_i xi_i,
 *            per cell (xx, xy, xz, yy, yz, zz); z components are 0 in 2D.
 * Computed on the device from the stored populations in the compute type of
 * the storage: FP64 for LBM_FP64, FP32 for LBM_FP32 and the shifted 16-bit
 * formats (rho = 1 + sum_i (f_i - w_i) keeps the precision of the small
 * sum), and returned as FP64.  When every non-NULL output is page-locked
 * host memory (as for lbm_set_state), the kernel writes the outputs directly;
 * otherwise they pass through the staging buffer.
 */
int lbm_moments(lbm_handle h, double *rho, double *u, double *pi_neq);
/* The same with FP32 host arrays (half the host-link bytes; the values are
 * formed in the compute type and rounded once to FP32). */
int lbm_moments_f32(lbm_handle h, float *rho, float *u, float *pi_neq);

/*
 * lbm_reduce -- FP64 totals over fluid cells of level 0: *mass = sum rho,
 * momentum[0..2] = sum rho u (over the cells with finite populations); the
 * per-cell moments are formed in the storage's compute type (as for
 * lbm_moments) and summed in FP64 in a fixed order.
 * Returns LBM_EUNSTABLE if a fluid cell holds a non-finite population, a
 * non-positive density or a velocity at or above the lattice sound speed
 * c_s = 1/sqrt(3) (the totals are still written).
 */
int lbm_reduce(lbm_handle h, double *mass, double momentum[3]);

/*
 * lbm_probe -- acoustic pressure fluctuation p' = c_s^2 (rho - rho_ref)
 * (Sec. II.A: p = c_s^2 rho) at n cells (host list of cell indices);
 * rho_ref is the sponge reference density (1 if no sponge).
 */
int lbm_probe(lbm_handle h, int n, const int64_t *cells, double *p_prime);

/*
 * lbm_set_launch -- launch shape of the update kernel (a tuning knob; the
 * result does not depend on it beyond FP round-off order).
 *   block            : threads per block, a multiple of 32 in [32, 256], or 0
 *                      for the default (128 one cell per thread, else 64)
 *   cells_per_thread : 1 = one cell per thread (the general kernel); 2 or 4 =
 *                      vectorised kernel with that many consecutive x cells per
 *                      thread (FP64: 2; FP32, FP16, BF16: 2 or 4); 0 = default
 *                      (measured fastest on GB300: 2 for FP16 / BF16 on D3Q19
 *                      and D3Q27 and for FP32 on D3Q27, else 1).  The
 *                      vectorised kernel is used only when
 *                      there is no cell-type mask and nx is a multiple of it
 *                      (on D3Q27 only with 2 cells per thread); otherwise the
 *                      general kernel runs.  These kernels
 *                      run when the row-staged kernel (lbm_set_staging) is off
 *                      or not eligible.
 * lbm_get_launch reports the shape lbm_step will use now.
 */
int lbm_set_launch(lbm_handle h, int block, int cells_per_thread);
int lbm_get_launch(lbm_handle h, int *block, int *cells_per_thread);

/*
 * lbm_pressure_mean / lbm_pressure_fluctuation -- the fluctuating pressure
 * Delta p~ = Delta p - Delta p_mean of Sec. III (Inoue and Hatakeyama), with
 * Delta p = c_s^2 (rho - 1) and Delta p_mean its temporal mean, for every cell
 * of the single level / coarse level.
 *   lbm_pressure_mean(h, LBM_MEAN_RESET)       forget the samples
 *   lbm_pressure_mean(h, LBM_MEAN_ACCUMULATE)  add rho of the stored field to
 *       a device FP64 running sum (allocated on first use: 8 bytes per cell,
 *       freed with the handle); the caller chooses the sampling steps
 *   lbm_pressure_fluctuation(h, dp_tilde, dp_mean): host arrays of ncell
 *       doubles (either may be NULL): c_s^2 (rho - mean rho) of the stored
 *       field and c_s^2 (mean rho - 1).  LBM_EINVAL before any sample.
 */
#define LBM_MEAN_RESET 0
#define LBM_MEAN_ACCUMULATE 1
int lbm_pressure_mean(lbm_handle h, int op);
int lbm_pressure_fluctuation(lbm_handle h, double *dp_tilde, double *dp_mean);

/*
 * lbm_set_sponge_jet_reference -- reference field of the outflow sponge for a
 * round jet along +x (Sec. IV: the jet similarity solution of Pope 2000 as
 * the sponge's reference in the outflow region; D3Q19).  In the cells of the
 * +x face's sponge layer (lbm_set_sponge on face 1; x >= nx - width) the
 * reference velocity becomes the self-similar mean axial profile
 *   u_x = U_0(x) / (1 + a eta^2)^2,  U_0 = min(U_jet, B D U_jet / (x - x0)),
 *   eta = r / (x - x0),  r = |(y, z) - (yc, zc)|,  a = (sqrt 2 - 1) / S^2
 * (u_x = U_0 / 2 at the half-width r = S (x - x0)), u_y = u_z = 0; other
 * sponge cells keep the uniform u_ref.  Lattice units; B 5.8 and S 0.094
 * are the usual round-jet constants.  D = 0 removes it.  LBM_EINVAL for
 * D2Q9, D, B or S <= 0, U_jet < 0, or non-finite values.
 */
int lbm_set_sponge_jet_reference(lbm_handle h, double yc, double zc, double U_jet, double D, double x0,
                                 double B, double S);

/*
 * lbm_set_hermite_order -- expansion order N of the regularized equilibrium
 * and off-equilibrium parts (Sec. II.A; default 3).  4 exists for D2Q9,
 * whose velocity set also supports H_xxyy = (xi_x^2 - c_s^2)(xi_y^2 - c_s^2):
 * the term 20.25 w_i H_xxyy(i) a4_xxyy is added with a4_eq = rho u_x^2 u_y^2
 * (Eq. recursive1) and a4_neq = u_x^2 P_yy + u_y^2 P_xx + 4 u_x u_y P_xy
 * (Eq. recursive2 at n = 4 read as the symmetric sum over index pairs);
 * lbm_set_state then also starts from the order-4 equilibrium.  It applies
 * to the rrBGK collision and its rebuilt boundary nodes (plain BGK keeps its
 * quadratic equilibrium).  LBM_EINVAL for other orders, other lattices, or
 * with refinement patches.
 */
int lbm_set_hermite_order(lbm_handle h, int order);

/*
 * lbm_set_collision -- collision model of the single-level update (Sec. II.A).
 *   LBM_COLLISION_RR  (default) recursive Hermite-regularized rrBGK, order 3
 *                     (Eq. optimizedLB with Eq. eqH, Eq. neqH, Eq. recursive2).
 *   LBM_COLLISION_BGK plain LBM-BGK, f* = f - (f - f^eq)/tau with the
 *                     quadratic equilibrium of Eq. truncatedEq (Eq. standardLB):
 *                     the A/B baseline the paper improves on.  Sponge cells
 *                     take f^eq at rho*, u* and add chi (f^eq(rho_ref, u_ref) -
 *                     f^eq(rho*, u*)); velocity, free-slip and pressure nodes
 *                     are rebuilt to second order, f^eq + (1 - 1/tau) f^neq_2.
 *                     Runs on the general one-cell-per-thread kernel; not
 *                     available with a refinement patch (LBM_EINVAL either way
 *                     round) nor in the solve server.
 */
#define LBM_COLLISION_RR 0
#define LBM_COLLISION_BGK 1
int lbm_set_collision(lbm_handle h, int model);

/*
 * lbm_set_transfer_staging -- bound on the device memory that host transfers
 * use.  lbm_set_state, lbm_set_populations, lbm_get_populations and
 * lbm_moments (and their per-level forms) move fields through one device
 * staging buffer per handle, in chunks of whole cells (state and moments in
 * page-locked host memory skip it: the kernels access them directly); it is allocated on
 * first use, holds min(max_bytes, what one field needs) bytes and is freed
 * with the handle.  Default 256 MiB; max_bytes must be >= 1024.  Transfers
 * synchronise the stream once, at the end of the call.
 */
int lbm_set_transfer_staging(lbm_handle h, size_t max_bytes);

/*
 * lbm_set_staging -- the row-staged update kernel (a tuning knob; same update
 * as the other kernels, results equal up to FP round-off order).  A
 * persistent grid of CTAs walks over tiles of whole x rows; bulk asynchronous
 * copies bring, for every direction, the rows the tile's cells pull from into
 * shared memory (`stages` tiles in flight per CTA) while the CTA updates the
 * previous tile.  It exists for FP32, FP16 and BF16 storage and runs only on a
 * level without a cell-type mask whose rows are a multiple of 16 bytes (nx a
 * multiple of 4 for FP32, of 8 for FP16 / BF16); elsewhere lbm_step falls
 * back to the kernels of lbm_set_launch.
 *   mode   : -1 default (= off: on GB300 the register kernels of
 *            lbm_set_launch are faster for the D3Q19 jet), 0 off, 1 on
 *            where eligible
 *   stages : shared-memory stages per CTA, 0 (= 2) or 2..8
 *   block  : threads per CTA, 0 (one per cell of a tile, at most 384) or a
 *            multiple of 32 in [32, 384]
 * The kernel bounds each wait for a copy at 2 s; a copy that does not arrive
 * makes the next lbm_sync return LBM_ECUDA (and clears the condition).
 * lbm_get_staging reports whether lbm_step uses it now (*active) and its
 * plan: stages, threads per CTA, rows per tile and CTAs; zeros when inactive.
 * Any output pointer may be NULL.
 */
int lbm_set_staging(lbm_handle h, int mode, int stages, int block);
int lbm_get_staging(lbm_handle h, int *active, int *stages, int *block, int *rows_per_tile, int *grid);

/*
 * lbm_set_storage_shift -- the constant subtracted from the stored
 * populations.  By default a population is stored as f_i - w_i (the rest
 * equilibrium at rho = 1); with u_s != 0 it is stored as f_i - feqH_i(1, u_s),
 * the third-order Hermite equilibrium of Eq. eqH at rho = 1 and the mean flow
 * u_s.  On a mean flow the stored values are then the acoustic and
 * non-equilibrium parts only, so the 16-bit formats round p' (Sec. III: the
 * acoustic pressure on a mean flow) far less; for FP32 / FP64 storage it only
 * moves the rounding.  u_s = NULL or (0, 0, 0) restores the default.  The
 * stored field (both lattices) is re-expressed in the new shift on the
 * device.  The arithmetic is unchanged: a loaded value gets
 * feqH_i(1, u_s) - w_i added, a stored one subtracted.  Runs on the general
 * update kernel (the vectorised and row-staged kernels are not used); not with
 * the AA pattern or refinement patches (LBM_EINVAL); |u_s| < c_s.
 * Checkpoints record the shift and load only into a handle with the same one.
 */
int lbm_set_storage_shift(lbm_handle h, const double u_s[3]);

/*
 * lbm_set_streaming -- streaming pattern of the single level (the update of
 * Eq. optimizedLB is the same with either; Sec. II.A streams post-collision
 * populations along xi_i, and where they are stored between steps is free):
 *   LBM_STREAM_PULL (default): two lattices; every step pulls the populations
 *       streamed into a cell from one lattice and writes the other.
 *   LBM_STREAM_AA: one lattice updated in place (half the device memory),
 *       with two step types that alternate.  A gather-push step pulls as the
 *       pull update does and pushes each collided population o_i into the
 *       slot P_opp(i)[x + xi_i] the neighbour will read (or back to P_i[x]
 *       at a solid or outside a non-periodic face); the next, local step
 *       reads P_opp(i)[x], collides and writes P_i[x], which restores the
 *       standard layout.  Every cell reads exactly the slots it writes; a
 *       boundary node is updated by the thread of the inward neighbour whose
 *       populations it takes.  Results equal the pull update's to round-off.
 *       Calls that read or write the populations (moments, reduce, probes,
 *       forces, checkpoints, transfers) first bring an odd-step lattice back
 *       to the standard layout in place.  Not with refinement patches.
 * The state is kept.  Switching to AA frees the second lattice; switching
 * back allocates it (LBM_ENOMEM if that fails; the handle stays AA).
 * lbm_get_streaming reports the pattern in use.
 */
#define LBM_STREAM_PULL 0
#define LBM_STREAM_AA 1
int lbm_set_streaming(lbm_handle h, int pattern);
int lbm_get_streaming(lbm_handle h, int *pattern);

/*
 * lbm_set_staging_wait -- limit of each wait of the row-staged kernel for a
 * tile's bulk copies, in nanoseconds of device global time (default 2e9).
 * 0 makes each wait one non-blocking test: a tile whose copies are still in
 * flight at that instant counts as late, so the failure path (error word set,
 * the CTA awaits its remaining copies with the 2 s limit and returns,
 * lbm_sync reports LBM_ECUDA) can be exercised without any copy actually
 * failing.  The populations written by such a step are unspecified.  No paper
 * counterpart: failure detection of the runtime.
 */
int lbm_set_staging_wait(lbm_handle h, uint64_t limit_ns);

/*
 * lbm_force -- force on the solid cells of a level (0 coarse / single level, 1
 * fine), FP64 on the device: momentum exchange over the halfway bounce-back
 * links, F = sum over fluid cells x and directions i with x + xi_i solid of
 * 2 xi_i f*_i(x), f* the stored post-collision field (momentum per step in
 * that level's lattice units).  The paper reports lift and drag coefficients
 * of its cylinder (Sec. III) without stating how they are computed; this is
 * the standard estimate for the bounce-back wall.  Zero without solids.
 */
int lbm_force(lbm_handle h, int level, double F[3]);

/*
 * lbm_force_async / lbm_probe_async -- lbm_force and lbm_probe written to
 * caller-owned DEVICE memory in stream order, without synchronising the
 * stream: a time series of lift, drag and probe pressures can be recorded
 * every few steps and read back once, so that sampling does not stall the
 * stepping.
 *   lbm_force_async : F_dev = 3 doubles (device) of level `level`
 *   lbm_probe_async : cells_dev = n cell indices (device, int64), p_dev = n
 *                     doubles (device); p' = c_s^2 (rho - rho_ref) as in
 *                     lbm_probe.  Indices are not checked on the host (they
 *                     are device data): an index outside [0, ncell) is
 *                     skipped and its output set to NaN.
 * Both return launch errors at once and execution errors at the next
 * synchronising call.
 */
int lbm_force_async(lbm_handle h, int level, double *F_dev);
int lbm_probe_async(lbm_handle h, int n, const int64_t *cells_dev, double *p_dev);

/* lbm_sync -- wait for all work of h; returns any pending execution error,
 * including a bulk copy of the row-staged kernel that timed out and, in the
 * checked build of the library (built with LBM_BOUNDS_CHECK, every index of
 * the update kernels tested before use), an index outside the lattice
 * (LBM_ECUDA; the condition is cleared). */
int lbm_sync(lbm_handle h);

/*
 * lbm_info -- read-only facts about a handle (any pointer may be NULL):
 *   step           : steps taken since the last set_state / set_populations / load
 *   launches       : number of kernels this handle has launched so far
 *   bytes_per_cell : algorithmic bytes one cell update moves (2 Q s, + 1 with
 *                    a geometry mask)
 *   tau            : relaxation time in use
 */
int lbm_info(lbm_handle h, int64_t *step, int64_t *launches, double *bytes_per_cell,
             double *tau);

/*
 * Refined levels (Sec. II.B, multi-domain 2:1 refinement; D2Q9, D3Q19 and
 * D3Q27).
 *
 * lbm_add_refinement_patch -- add a level inside the finest existing level
 * (the first call refines level 0, the next one nests inside it, ...; at
 * most LBM_MAX_LEVELS levels in all).  The new level covers the parent-level
 * nodes origin[a]..origin[a]+extent[a] on every axis a of the lattice (x, y;
 * and z in 3D; extent >= 4, at least 2 cells from every face of the
 * parent).  It has 2 extent[a] + 1 nodes per axis, half the parent's spacing,
 * two steps per parent step (Eq. convective), tau = 2 tau_parent - 1/2 (same
 * physical viscosity), and starts at rest.  Coupling per parent step: the new
 * level's boundary ring (2D) / shell (3D) is rebuilt from the parent's rho,
 * u, Pi^neq interpolated in space (copy at coincident nodes; the 4-point
 * cubic (-1, 9, 9, -1)/16 along every axis on which the node falls between
 * parent nodes, their tensor product on the 3D interface planes) and linearly
 * in time (t + 1/2, t + 1), Eq. couplingFC; the parent's first ring / shell of
 * covered nodes is rebuilt from the coincident node's rho, u and its
 * full-weighted Pi^neq ((1,2,1)^2 / 16 in 2D, (1,2,1)^3 / 64 in 3D),
 * Eq. couplingCF.  f^neq is rescaled by tau_child / (2 tau_parent) parent ->
 * child and 2 tau_parent / tau_child child -> parent (the leading-order
 * Chapman-Enskog scaling of Sec. II.B).  Deeper covered parent cells are
 * frozen.  Solids of a refined level must stay 2 of its cells inside its
 * ring / shell and outside its child's box.
 *
 * Level-indexed variants (level 0 = coarse, the plain functions; level k =
 * the k-th refined level): extents and tau of a level; geometry (cell types
 * of a refined level; its ring and its child's covered box are managed by the
 * library); initial state and populations (set_*_level touches only that
 * level and refreshes the interface moments of the level it is the parent
 * of); populations and moments of the stored field.
 */
#define LBM_MAX_LEVELS 8
int lbm_add_refinement_patch(lbm_handle h, const int origin[3], const int extent[3]);
int lbm_level_info(lbm_handle h, int level, int extents[3], double *tau);
int lbm_set_geometry_level(lbm_handle h, int level, const uint8_t *cell_type);
int lbm_set_state_level(lbm_handle h, int level, const double *rho, const double *u);
int lbm_set_populations_level(lbm_handle h, int level, const double *f);
int lbm_get_populations_level(lbm_handle h, int level, double *f);
int lbm_moments_level(lbm_handle h, int level, double *rho, double *u, double *pi_neq);

/*
 * lbm_set_level_streams -- how the refined levels' part of a step is
 * scheduled (Sec. II.B: within one coarse step the fine levels read the
 * coarse interface moments, not the coarse update).
 *   concurrent = 1 (default): the levels below level 0 (their updates, ring
 *                fills and the restriction into level 0's covered ring) run
 *                on a second stream of the highest priority, concurrently
 *                with the level-0 update; the handle's stream waits for them
 *                at the end of each step.
 *   concurrent = 0: everything in order on the handle's stream.
 * The results are bitwise the same.  Errors: LBM_EINVAL (other values).
 */
int lbm_set_level_streams(lbm_handle h, int concurrent);

/*
 * lbm_save / lbm_load -- checkpoint and resume: write / read the stored
 * field of every level (raw storage format), the refined levels' interface
 * moments at the current time, the pressure-mean accumulator (if sampled)
 * and the step counter to a host file with a header.  A run resumed from
 * the file continues bit for bit as the run that wrote it.  lbm_load
 * requires a handle configured the same way: lattice, precision, extents and
 * the same refinement patches (else LBM_EINVAL, before any state changes);
 * boundary rules, geometry, sponges and options are not part of the file.
 */
int lbm_save(lbm_handle h, const char *path);
int lbm_load(lbm_handle h, const char *path);

/*
 * Solve server: continuous batching of independent solves (serving).
 *
 * A request is a fully periodic lattice with its own lattice type, extents,
 * tau, number of steps, storage precision and initial rho, u (Eq. eqH
 * populations).  lbm_server_submit queues it (the initial fields are copied).
 * Each lbm_server_run call is one round: queued requests are admitted in
 * arrival order, first fit, while their population lattices (two, or one
 * with the AA pattern) fit in the HBM budget and a slot is free; then every
 * active request advances by up to `steps` steps in one CUDA-graph replay of
 * batched updates (one persistent launch per (lattice, precision) group, plus
 * a per-request step counter), a request stopping exactly at its own step
 * count; finished requests are retired behind the round (rho and u of the
 * final post-collision field copied to pinned host memory, device memory
 * returned to the budget).  A round is enqueued without waiting for the GPU:
 * lbm_server_run returns once the round and its admissions and retirements
 * are on the stream, waiting only while two earlier rounds are still in
 * flight; a retired request turns LBM_REQ_DONE (or FAILED) when its result
 * copy has completed, seen by lbm_server_poll.  A request's arithmetic is
 * the single-lattice update's and does not depend on what it is batched
 * with.
 *   lbm_server_create : budget in bytes, max_slots concurrent requests, stream
 *                       (NULL: the server creates its own)
 *   lbm_server_run    : *completed (may be NULL) = requests whose results
 *                       completed since the previous call
 *   lbm_server_set_streaming : LBM_STREAM_PULL (default) or LBM_STREAM_AA for
 *                       requests admitted from now on (one lattice each, so
 *                       the budget holds twice the cells)
 *   lbm_server_set_launch : launch shape of the (lattice, precision) group's
 *                       batched update from the next round on: cells_per_lane
 *                       1 or 2 (0: 2; a request with an odd row length, or
 *                       whose direction arrays span 2 GB or more, takes 1) and
 *                       warps_per_block 1, 2, 4 or 8 (0: 2).  The arithmetic
 *                       of a request does not depend on it.
 *   lbm_server_get_launch : the group's current shape
 *   lbm_server_poll   : state LBM_REQ_* and steps done so far
 *   lbm_server_result : copies rho (ncell) and u (3 ncell) of a finished request
 *                       to host buffers (either may be NULL) and forgets it;
 *                       LBM_EUNSTABLE if the result is not finite
 *   lbm_server_stats  : queue length, running requests, budget in use, total
 *                       cell updates advanced
 *   lbm_server_gpu_time : device time of all rounds' graphs so far (ms, CUDA
 *                       events around each replay; waits for the stream)
 * Errors: LBM_EINVAL (bad request, a request larger than the whole budget,
 * unknown id, result of an unfinished request), LBM_ECUDA.
 */
typedef struct lbm_server *lbm_server_handle;

#define LBM_REQ_QUEUED 0
#define LBM_REQ_RUNNING 1
#define LBM_REQ_DONE 2
#define LBM_REQ_FAILED 3

typedef struct {
    int lattice;        /* LBM_D2Q9, LBM_D3Q19 or LBM_D3Q27 */
    int precision;      /* LBM_FP64 .. LBM_BF16_SHIFTED */
    int extents[3];     /* extents[2] = 1 for D2Q9 */
    double tau;         /* > 1/2 */
    int64_t steps;      /* >= 0 */
    const double *rho;  /* ncell, host, or NULL for 1 */
    const double *u;    /* 3 ncell, host, or NULL for 0 */
} lbm_request;

int lbm_server_create(lbm_server_handle *out, size_t hbm_budget_bytes, int max_slots, void *cuda_stream);
void lbm_server_destroy(lbm_server_handle s);
const char *lbm_server_last_error(lbm_server_handle s);
int lbm_server_submit(lbm_server_handle s, const lbm_request *req, int64_t *id);
int lbm_server_run(lbm_server_handle s, int64_t steps, int *completed);
int lbm_server_set_streaming(lbm_server_handle s, int pattern);
int lbm_server_set_launch(lbm_server_handle s, int lattice, int precision, int cells_per_lane, int warps_per_block);
int lbm_server_get_launch(lbm_server_handle s, int lattice, int precision, int *cells_per_lane, int *warps_per_block);
int lbm_server_poll(lbm_server_handle s, int64_t id, int *state, int64_t *steps_done);
int lbm_server_result(lbm_server_handle s, int64_t id, double *rho, double *u);
int lbm_server_stats(lbm_server_handle s, int *queued, int *running, size_t *bytes_in_use,
                     int64_t *cell_updates);
int lbm_server_gpu_time(lbm_server_handle s, double *ms);

/*
 * lbm_reduce_noalloc -- the totals of lbm_reduce for a population field the
 * caller owns, computed without allocating any memory.  (The paper has no
 * counterpart: this is an integration entry point.)
 *
 * For callers that cannot allocate device memory where they need the totals:
 * loops that must never enter an allocator (real-time or memory-accounted
 * code), or hosts that keep a fixed device-memory budget and lend the
 * library only their own buffers.
 * The per-block partial sums live in a static device array inside the
 * library, sized for at most LBM_NOALLOC_MAX_CELLS cells, which every GPU
 * that loads the library keeps until the process exits.  The call itself
 * allocates nothing and does not use a handle.
 *   lattice   : LBM_D2Q9, LBM_D3Q19 or LBM_D3Q27
 *   precision : LBM_FP64, LBM_FP32, LBM_FP16_SHIFTED or LBM_BF16_SHIFTED
 *   f         : device pointer to the field in the library's storage layout:
 *               q * ncell values of the precision's type, direction-major
 *               (f[i * ncell + cell]), each holding f_i - w_i
 *   ncell     : number of cells, 1 <= ncell <= LBM_NOALLOC_MAX_CELLS (larger
 *               fields are rejected with LBM_EINVAL)
 *   cell_type : device pointer to ncell cell types, or NULL (all fluid); only
 *               fluid cells are counted
 *   out       : device pointer to 6 doubles, written in stream order:
 *               [sum rho, sum rho ux, sum rho uy, sum rho uz, fluid cells,
 *               unstable cells (non-finite, rho <= 0 or |u| >= c_s)]
 *   cuda_stream : stream to enqueue on (NULL: legacy default stream)
 * Asynchronous: synchronise the stream before reading out.  The first call on
 * a device looks up the scratch array's device address on the host (once per
 * device, with that device current).  Every call reuses the same scratch, so
 * calls that overlap on the
 * GPU (other streams, other host threads) race; each call overwrites all the
 * scratch it reads, so nothing needs clearing between calls.  Errors are
 * reported by lbm_last_error(NULL).
 */
#define LBM_NOALLOC_MAX_CELLS 67108864LL
int lbm_reduce_noalloc(int lattice, int precision, const void *f, int64_t ncell,
                       const uint8_t *cell_type, double *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
