/*
 * clbm.h - C ABI of the GB300 cascaded thermal lattice Boltzmann library.
 *
 * The library advances the double-distribution-function cascaded LBM of
 * Fei & Luo ("Cascaded lattice Boltzmann method for incompressible thermal
 * flows with heat sources and general thermal boundary conditions"):
 * D2Q9 flow distributions f_i (Sec. 2.1, Eq. 3-12) and D2Q5 temperature
 * distributions g_i (Sec. 2.2, Eq. 13-22), coupled through the Boussinesq
 * force (Eq. 2), with the central-moment heat source (Sec. 2.3, Eq. 23-25),
 * half-way bounce-back for velocity (Sec. 3) and the general bounce-back
 * scheme for Dirichlet / Neumann / Robin temperature walls (Eq. 26-28).
 *
 * Conventions
 *   - Lattice units (dx = dt = 1).  Nodes are cell centres (x+1/2, y+1/2),
 *     x = 0..nx-1, y = 0..ny-1.  Every array crossing this ABI is row major
 *     [ny][nx] (x fastest), dense, without padding.
 *   - D2Q9 directions follow Eq. 3: ex = {0,1,0,-1,0,1,-1,-1,1},
 *     ey = {0,0,1,0,-1,1,1,-1,-1}; D2Q5 uses directions 0..4.
 *   - Walls of non-periodic box sides lie half a spacing outside the first
 *     and last node row/column.  Solid nodes (mask) are walls too.
 *   - Ownership: the library owns every device allocation it makes; caller
 *     arrays are only read (inputs) or written (outputs) during the call and
 *     are never retained.  Host pointers are plain host memory; "device"
 *     pointers are CUDA device pointers valid on the context's device.
 *   - Streams: all device work of a context is issued on its stream (the one
 *     passed to clbm_create, or a stream the library creates for NULL).
 *     clbm_step only enqueues work; calls that return a host value
 *     (clbm_moments to host, clbm_nusselt, clbm_residual, clbm_totals) synchronise the
 *     stream before returning.
 *   - Errors: no call throws or aborts.  Each returns a clbm_status; on a
 *     failure the context (when there is one) keeps a message readable with
 *     clbm_last_error().  CLBM_ECUDA means a CUDA runtime call failed.
 */
#ifndef CLBM_H_
#define CLBM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CLBM_OK = 0,
  CLBM_EINVAL = 1,     /* invalid argument or problem description        */
  CLBM_ENOMEM = 2,     /* device or host allocation failed               */
  CLBM_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed    */
  CLBM_EUNSTABLE = 4,  /* NaN or Inf found in the fields                 */
  CLBM_ETIMEOUT = 5,   /* a bounded device-side wait ran out             */
  CLBM_ENOTCONV = 6    /* iteration cap reached before convergence       */
} clbm_status;

/* Storage precision of the distributions.  Every format stores deviations
 * from the rest state (f_i - w_i rho0, g_i - w^T_i T0, with w the D2Q9
 * weights 4/9, 1/9, 1/36 and w^T = (1 - 2 cT2, cT2/2 x4)).  The collision is
 * computed in FP64 for CLBM_F64 and in FP32 for every other format.  The
 * 16-bit formats round either to nearest even or stochastically (params
 * `rounding`); stochastic rounding draws its bits from a counter-based hash of
 * (step, node, plane), so runs stay reproducible. */
typedef enum {
  CLBM_F64 = 0,
  CLBM_F32 = 1,
  CLBM_F16DEV = 2,   /* IEEE binary16 deviations                          */
  CLBM_BF16DEV = 3   /* bfloat16 deviations                               */
} clbm_precision;

/* Problem parameters (lattice units).
 *   s_nu  : shear rate, nu = (1/s_nu - 1/2)/3 (Eq. 8 text)
 *   s_b   : bulk rate, nu_b = (1/s_b - 1/2)/3 (Eq. 8 text)
 *   s_3   : rate of k~21, k~12; <= 0 selects s3 = (16 - 8 s_nu)/(8 - s_nu) (Sec. 3)
 *   s_4   : rate of k~22 (Eq. 8)
 *   lambda0, lambda1, lambda2 : S_T = diag(l0, l1, l1, l2, l2) (Sec. 2.2);
 *           alpha = (1/lambda1 - 1/2) cT2; lambda2 <= 0 selects
 *           lambda2 = 12 (lambda1 - 2)/(lambda1 - 12) (Sec. 3.1)
 *   rho0, T0 : reference density and temperature (Eq. 1-2)
 *   gbeta : g * beta; the buoyancy force density is rho0 gbeta (T - T0) along +y (Eq. 2)
 *   Fvx, Fvy : external body force density F_v (Eq. 2)
 *   Q     : uniform volumetric heat source (Eq. 23-25)
 *   cT2   : squared D2Q5 sound speed c_T^2 (Eq. 19; 2/5 in Sec. 3)
 *   viscous_heating : 1 adds the viscous dissipation source of Sec. 3.2 to Q at
 *           every node, Q_v = nu (D^2 + G^2) with D = dux/dx - duy/dy and
 *           G = duy/dx + dux/dy (= nu (du/dy)^2 in a channel), the strain read
 *           from the node's pre-collision non-equilibrium central moments
 *           (G = -3 s_nu k~11/rho, D = -3 s_nu (k~20 - k~02)/(2 rho)); the
 *           Boussinesq force then uses T without Q_v/2.  Adds one stored plane. */
typedef struct {
  int32_t nx, ny;
  int32_t periodic_x, periodic_y;
  int32_t precision; /* clbm_precision */
  int32_t rounding;  /* 16-bit formats: 0 = round to nearest even, 1 = stochastic rounding */
  double s_nu, s_b, s_3, s_4;
  double lambda0, lambda1, lambda2;
  double rho0, T0, gbeta, Fvx, Fvy, Q, cT2;
  int32_t viscous_heating;
  int32_t reserved1;
} clbm_params;

/* Thermal wall condition b1 dT/dn + b2 T = b3 (Sec. 2.3), n the unit normal
 * pointing out of the fluid.  Dirichlet: (0, 1, Tw); Neumann: (1, 0, flux). */
typedef struct {
  double b1, b2, b3;
} clbm_tbc;

/* One wall link of a fluid node into a solid node (Eq. 26-28): the link `dir`
 * leaves fluid node `node` = y*nx + x towards the wall (the e_i of Eq. 26).
 * D2Q5 directions 1..4: `n_dot_e` = n.e_i > 0 of Eq. 27-28 and `tbc` indexes
 * the condition table; every D2Q5 link into a solid node must be listed.
 * Curved walls are described by such links with the true normal.
 * `q` in (0, 1] is the fraction of the link from the fluid node to the wall.
 * q = 1/2 is the paper's half-way wall.  Any other q (no counterpart in the
 * paper) selects, for that link: for f the linear interpolated bounce-back of
 * Bouzidi, Firdaouss and Lallemand (2001) (q < 1/2 also reads f_i* at
 * x_f - e_i); for g Eq. 26 at the link midpoint with the temperature that the
 * wall profile has there (T_w from b1 dT/dn + b2 T_w = b3 with the gradient
 * of the quadratic through the wall and the fluid nodes at q and 1 + q).
 * Diagonal directions 5..8 may be listed to give their q (n_dot_e and tbc are
 * ignored there); unlisted wall directions are half-way. */
typedef struct {
  int32_t node, dir;
  double n_dot_e;
  int32_t tbc, reserved;
  double q;
} clbm_link;

typedef struct clbm_ctx clbm_ctx;

/* Create a solver for one lattice on the current CUDA device.  Allocates two
 * distribution buffers (ping-pong) and sets the state to the equilibrium at
 * rest (rho0, u = 0, T0).  `stream` is a cudaStream_t or NULL.  The lattice
 * has no walls until clbm_set_boundaries is called (all four box sides must
 * then be periodic or have a condition).
 * Errors: CLBM_EINVAL (sizes < 1, non-positive rates, unknown precision),
 * CLBM_ENOMEM, CLBM_ECUDA. */
clbm_status clbm_create(const clbm_params* params, void* stream, clbm_ctx** out);

/* Describe the walls (Sec. 2.3, Sec. 3).
 *   solid    : host uint8 [ny][nx], nonzero = solid node, or NULL (no obstacles)
 *   tbc      : host table of n_tbc conditions
 *   side_tbc : host int32[4], condition index of the box sides x0 (left),
 *              x1 (right), y0 (bottom), y1 (top); ignored on periodic axes
 *   links    : host array of n_links wall links (may be NULL when n_links = 0);
 *              every D2Q5 link from a fluid node into a solid node must be listed
 * All inputs are copied.  The distribution state is left unchanged.
 * Errors: CLBM_EINVAL for out-of-range indices, a missing link, a fluid node
 * with no fluid neighbour, or a non-periodic side without a condition. */
clbm_status clbm_set_boundaries(clbm_ctx* ctx, const uint8_t* solid, const clbm_tbc* tbc,
                                int32_t n_tbc, const int32_t* side_tbc, const clbm_link* links,
                                int32_t n_links);

/* Velocity (ux, uy) of box side `side` (0 = x0, 1 = x1, 2 = y0, 3 = y1), for
 * flows driven by a moving wall such as thermal Couette flow.  Not part of the
 * paper, whose walls are at rest: a population f_i* reflected at a moving side
 * returns as f_ibar = f_i* - 2 w_i rho0 (e_i . u_w) / cs^2 (the bounce-back of
 * Ladd, J. Fluid Mech. 271, 1994; e_i toward the wall, cs^2 = 1/3).  The
 * temperature rule (Eq. 26-28) is unchanged: for a wall moving along itself
 * the D2Q5 populations crossing it carry no velocity term.  A diagonal link
 * into a box corner takes the velocity of the x side when x is not periodic.
 * Periodic sides ignore their velocity.  All sides start at rest.
 * Errors: CLBM_EINVAL for side outside 0..3 or a non-finite velocity. */
clbm_status clbm_set_wall_velocity(clbm_ctx* ctx, int32_t side, double ux, double uy);

/* Set the state to the equilibrium distributions whose central moments are
 * Eq. 9 and Eq. 19 at the given fields, i.e. f(t=0) = f^eq(rho, u),
 * g(t=0) = g^eq(T, u), and reset the step counter.  Each pointer is an FP64
 * [ny][nx] array or NULL for the rest value (rho0, 0, 0, T0).  on_device
 * selects device (1) or host (0) pointers.  Host arrays: exactly nx * ny
 * doubles are read from each; page-locked memory mapped into the device's
 * address space (cudaHostAlloc, cudaHostRegister) is read by the kernel in
 * place, pageable memory is copied through a device scratch allocated on first
 * use.  With host pointers the call synchronises before it returns. */
clbm_status clbm_init_fields(clbm_ctx* ctx, const double* rho, const double* ux, const double* uy,
                             const double* T, int32_t on_device);

/* Enqueue nsteps time steps (collision Eq. 7/23, streaming Eq. 11/21, wall
 * rules Eq. 26-28) on the context stream.  Returns without synchronising;
 * CLBM_ECUDA reports a launch failure. */
clbm_status clbm_step(clbm_ctx* ctx, int64_t nsteps);

/* Macroscopic fields at the current time: rho = sum f (Eq. 12),
 * u = (sum f e + F/2)/rho (Eq. 12), T = sum g + Q/2 (Eq. 25), as FP64
 * [ny][nx] arrays; solid nodes report 0.  Any pointer may be NULL.
 * on_device selects device (1) or host (0) outputs; host outputs synchronise.
 * Each host output receives exactly nx * ny doubles: the kernel writes mapped
 * page-locked memory in place and pageable memory through the device scratch. */
clbm_status clbm_moments(clbm_ctx* ctx, double* rho, double* ux, double* uy, double* T,
                         int32_t on_device);

/* Nusselt number of one wall: (length/dT) * mean over its D2Q5 wall links of
 * dT/dn from Eq. 27 with T_w from Eq. 28, n pointing out of the fluid, so it
 * is positive where heat enters the fluid.  which = 0..3 selects a box side
 * (x0, x1, y0, y1); which = 4 + k selects the listed links with condition k.
 * Accumulated in FP64 in a fixed order (deterministic).  Synchronises.
 * Errors: CLBM_EINVAL when the selection has no links. */
clbm_status clbm_nusselt(clbm_ctx* ctx, int32_t which, double length, double dT, double* nu_out);

/* Steady-state residual over the last step: max over phi in {T, ux, uy} of
 * ||phi(t) - phi(t-1)||_2 / max(||phi(t)||_2, 1e-30) over fluid nodes,
 * accumulated in FP64 in a fixed order.  Needs at least one step since the
 * last initialisation (else CLBM_EINVAL).  Returns CLBM_EUNSTABLE (and
 * r_out = +inf) if any field value is NaN or Inf.  Synchronises. */
clbm_status clbm_residual(clbm_ctx* ctx, double* r_out);

/* Conservation sums (Eq. 7's conserved moments, Eq. 23's zeroth thermal
 * moment): FP64 sums over the fluid nodes of the stored post-collision
 * distributions, out[0] = sum f_i (mass), out[1] = sum f_i e_ix,
 * out[2] = sum f_i e_iy (momentum; = sum (rho u + F/2)), out[3] = sum g_j
 * (= sum (T + Q/2), plus half the viscous source where it is on).  On a
 * lattice without walls the mass is constant, the momentum grows by the summed
 * body force and out[3] by N Q per step.  `out` is a host array of 4 doubles.
 * Fixed-order reduction (same value on every call for the same state).
 * Returns CLBM_EUNSTABLE if a value is NaN or Inf.  Synchronises. */
clbm_status clbm_totals(clbm_ctx* ctx, double* out);

/* ---------------------------------------------------------------------
 * Domain decomposition into y-slabs.  The step needs, at every node, only the
 * post-collision populations of its eight neighbours (streaming, Eq. 11 and
 * Eq. 21) and, at a wall link, the temperature of the next node along the
 * link (Eq. 27-28), so a lattice splits into slabs of whole rows that each
 * keep one ghost row on each side: after every step (and after the
 * initialisation) each slab's first and last own rows, all planes, are copied
 * into its neighbours' ghost rows.  A slab reproduces the whole lattice's
 * values on its rows bit for bit.  Reductions are partial sums over the own
 * rows (clbm_reduce_sums), added across slabs and finished with
 * clbm_finish_sums.
 * ------------------------------------------------------------------- */

/* Create a solver for rows [y0, y0 + rows) of the lattice that `params`
 * describes (params->ny = the whole lattice's rows, params->periodic_y its y
 * axis).  Stores rows + 2 rows (a ghost row below and above).  Every other
 * call takes and returns the slab's own rows: clbm_init_fields and
 * clbm_moments arrays are [rows][nx]; clbm_set_boundaries takes the WHOLE
 * lattice's description (solid [ny][nx], links with whole-lattice node
 * numbers) and keeps the slab's part.  A box side y0 / y1 is a wall of the
 * slab only if the slab holds the first / last row of a non-periodic lattice.
 * The ghost rows start at zero: exchange halos before the first step.
 * Errors: CLBM_EINVAL (rows < 1, y0 < 0, y0 + rows > ny, or as clbm_create);
 * clbm_set_boundaries returns CLBM_EINVAL for an off-midpoint Dirichlet link
 * (q < 1/2) whose third node x_f - 2 e_i lies beyond the ghost row. */
clbm_status clbm_create_slab(const clbm_params* params, int32_t y0, int32_t rows, void* stream,
                             clbm_ctx** out);

/* Bytes of one packed halo row: planes (14, or 15 with the viscous source) x nx
 * elements of the storage format, laid out [plane][x]. */
clbm_status clbm_halo_bytes(const clbm_ctx* ctx, int64_t* bytes);

/* Copy the slab's first (side 0) or last (side 1) own row of the current
 * state, every plane, into the device buffer dst ([plane][x], clbm_halo_bytes
 * bytes), on the context stream.  For exchanges through a communication
 * library (one slab per process): side 0 goes to the slab below, side 1 to the
 * slab above. */
clbm_status clbm_halo_pack(clbm_ctx* ctx, int32_t side, void* dst);

/* Write a packed row (device buffer, as clbm_halo_pack) into the ghost row
 * below (side 0: the last own row of the slab below) or above (side 1: the
 * first own row of the slab above) of the current state, on the context stream. */
clbm_status clbm_halo_unpack(clbm_ctx* ctx, int32_t side, const void* src);

/* Copy `from`'s first (side 0) or last (side 1) own row, every plane, straight
 * into the ghost row above (side 0) or below (side 1) of `to` (the slab below /
 * above it), with one strided copy on `to`'s stream; if the two contexts have
 * different streams, events order the copy after `from`'s work and `from`'s
 * later work after the copy.  Both must be slabs of the same nx, format and
 * plane count, on one device or on peer-accessible devices. */
clbm_status clbm_halo_copy(clbm_ctx* from, int32_t side, clbm_ctx* to);

/* Exchange the halos of n slabs of one lattice held by this process, ordered
 * bottom to top (slabs[k + 1] above slabs[k]); periodic != 0 also joins the
 * last slab to the first. */
clbm_status clbm_slabs_exchange(clbm_ctx* const* slabs, int32_t n, int32_t periodic);

/* nsteps times: one step of every slab, then clbm_slabs_exchange. */
clbm_status clbm_slabs_step(clbm_ctx* const* slabs, int32_t n, int32_t periodic, int64_t nsteps);

/* Raw FP64 sums of one reduction over the context's own rows, into out[8]
 * (host), for adding across slabs before clbm_finish_sums:
 *   what = 0: residual over the last step: sum dT^2, T^2, dux^2, ux^2, duy^2,
 *             uy^2 (differences to the previous step), non-finite count, 0;
 *   what = 1: Nusselt selection `which` (as clbm_nusselt): sum of dT/dn over
 *             the selection's links held here, their count (0 allowed),
 *             non-finite count;
 *   what = 2: conservation: sum of the stored deviations d_i, d_i e_ix,
 *             d_i e_iy, h_j over the fluid nodes, fluid-node count,
 *             non-finite count.
 * Fixed-order sums; synchronises. */
clbm_status clbm_reduce_sums(clbm_ctx* ctx, int32_t what, int32_t which, double* out);

/* Finish summed reductions (the sums of every slab added element-wise):
 * what = 0 -> out[0] = the clbm_residual value; 1 -> out[0] = the Nusselt
 * number (length/dT x mean dT/dn); 2 -> out[0..3] = the clbm_totals values
 * (rho0, T0 from ctx).  CLBM_EUNSTABLE for non-finite sums, CLBM_EINVAL for a
 * Nusselt selection with no links. */
clbm_status clbm_finish_sums(const clbm_ctx* ctx, int32_t what, const double* sums, double length,
                             double dT, double* out);

/* Allocation-free variant of the residual reduction (the paper has no
 * counterpart; it is a service for callers of this library).
 *
 * For callers that cannot allocate device memory: applications that give all
 * device memory to their own pool allocator up front, host frameworks that
 * forbid allocations by embedded libraries, and time-critical loops that
 * cannot take the device synchronisation cudaFree implies.  It computes the
 * clbm_residual quantity, max over phi in {T, ux, uy} of
 * ||phi_now - phi_prev||_2 / max(||phi_now||_2, 1e-30), from caller-owned
 * FP64 device arrays of n values (for instance two clbm_moments snapshots one
 * step apart); `solid` is an optional device uint8 mask (nonzero = skip).
 * The result is written to the host double *r_out; the call synchronises
 * `stream` (a cudaStream_t, NULL = legacy default stream), which must belong
 * to the current device (else CLBM_EINVAL).  Because it copies the result to
 * the host and synchronises, it must not be called while any stream of the
 * process is being captured into a CUDA graph.
 *
 * It calls no cudaMalloc, cudaFree or allocating library routine: its
 * reduction scratch is a fixed 65,600-byte array in the library's device
 * data, held on every GPU that loads the library until the process exits.
 * The first call on a device looks that array's address up (once per device,
 * with the device current) and caches it; after a cudaDeviceReset of that
 * device the cached address is stale, so do not use this call after a reset.
 * All calls share the array, so calls that overlap on the GPU race and must be
 * serialised by the caller.  Limits: 1 <= n <= 2^31, else CLBM_EINVAL;
 * CLBM_EUNSTABLE (r_out = +inf) if a value is NaN or Inf. */
clbm_status clbm_residual_fields_noalloc(const double* T_now, const double* ux_now,
                                         const double* uy_now, const double* T_prev,
                                         const double* ux_prev, const double* uy_prev,
                                         const uint8_t* solid, int64_t n, void* stream,
                                         double* r_out);

/* ---------------------------------------------------------------------
 * Batched solves: many independent lattices (sizes, rates, walls may all
 * differ) advanced together by the same kernel launches.
 * ------------------------------------------------------------------- */
typedef struct clbm_batch clbm_batch;

/* One lattice of a batch.  params.precision and params.rounding must be the
 * same for every item.  solid / tbc / side_tbc / links follow
 * clbm_set_boundaries; rho, ux, uy, T are host FP64 [ny][nx] initial fields
 * (NULL = rest value), used as in clbm_init_fields.  All host data is copied
 * during clbm_batch_create. */
typedef struct {
  clbm_params params;
  const uint8_t* solid;
  const clbm_tbc* tbc;
  int32_t n_tbc;
  int32_t side_tbc[4];
  int32_t n_links;
  const clbm_link* links;
  const double* rho;
  const double* ux;
  const double* uy;
  const double* T;
} clbm_batch_item;

/* Create a batch of n lattices in one device arena (two ping-pong buffers).
 * Batched lattices run without the viscous source (viscous_heating must be 0).
 * autotune != 0 times the batched step with tile widths of 32, 64 and 128
 * nodes per warp for each class of row length (<= 48, <= 96, <= 192, > 192
 * nodes) and keeps the fastest; otherwise every lattice uses 128 (64 for
 * FP64).  `stream` as in clbm_create.  Errors as clbm_create and
 * clbm_set_boundaries. */
clbm_status clbm_batch_create(const clbm_batch_item* items, int32_t n, int32_t autotune,
                              void* stream, clbm_batch** out);

/* Advance every lattice until its steady-state residual falls below tol, or
 * until max_steps steps (the last check may overrun by less than
 * check_every).  The residual is checked every K = check_every steps
 * (rounded up to an even number) as max over phi in {T, ux, uy} of
 * ||phi(t) - phi(t - K)||_2 / (K ||phi(t)||_2) over fluid nodes: the mean
 * per-step change over the interval.  Comparing states an even number of
 * steps apart ignores the small period-2 oscillation that closed cavities can
 * sustain, which keeps the one-step quantity of clbm_residual above tight
 * tolerances.  Per-node values are formed in the collision's arithmetic
 * (FP32 below FP64 storage) and summed in FP64.  The first check of a solve
 * only takes the snapshot.  Each check_every block of steps is one replay of a
 * captured CUDA graph; converged lattices leave the device-side work list.
 * Outputs (host arrays of n, may be NULL): conv_steps[i] = step count at
 * which lattice i converged, -1 if it did not, -2 if it diverged (NaN/Inf);
 * residuals[i] = its last computed residual; *steps_run = steps taken.
 * The lattices keep their final state (read it through clbm_batch_lattice). */
clbm_status clbm_batch_solve(clbm_batch* b, double tol, int64_t max_steps, int32_t check_every,
                             int64_t* conv_steps, double* residuals, int64_t* steps_run);

/* Context view of lattice i (owned by the batch: do not destroy it) for
 * clbm_moments, clbm_nusselt, clbm_residual, clbm_init_fields or clbm_step. */
clbm_status clbm_batch_lattice(clbm_batch* b, int32_t i, clbm_ctx** view);

/* Nodes per warp tile chosen for lattice i (32, 64 or 128). */
clbm_status clbm_batch_tile_width(const clbm_batch* b, int32_t i, int32_t* nodes_per_warp);

/* Free the batch, its views and its arena (NULL is allowed). */
clbm_status clbm_batch_destroy(clbm_batch* b);

/* Message of the last failure on this batch ("" if none). */
const char* clbm_batch_last_error(const clbm_batch* b);

/* ---------------------------------------------------------------------
 * Surrogate network for warm starts (no counterpart in the paper): a
 * convolutional encoder-decoder (U-Net) on a G x G grid, trained and run
 * by the library's own kernels (implicit-GEMM convolutions, FP32
 * accumulation, BF16 weights with an FP32 master copy, Adam).
 *   levels L (2..6), base width B: widths B, 2B, ..., 2^(L-1) B; G must be
 *   divisible by 2^(L-1).  Input in_ch, output out_ch channels (NCHW FP32).
 * All tensors passed to these calls are FP32 device arrays.
 *
 * Convolution arithmetic (clbm_net_config.math):
 *   CLBM_NET_TENSOR  5th-generation tensor cores (tcgen05.mma): both GEMM
 *                    operands (activations or activation gradients, and
 *                    weights) rounded to BF16 (nearest even), products
 *                    accumulated in FP32 in tensor memory.
 *   CLBM_NET_FP32    FP32 CUDA cores: FP32 activations and gradients, BF16
 *                    weights, FP32 accumulation.
 * Bias, pooling, upsampling, ReLU, loss and Adam are FP32 in both.  A
 * tensor-core GEMM that waits more than about a second for its MMAs gives
 * up, and the next clbm_net_forward / clbm_net_gradients /
 * clbm_net_train_step returns CLBM_ETIMEOUT (sticky for the network).
 * ------------------------------------------------------------------- */
typedef struct clbm_net clbm_net;

typedef enum { CLBM_NET_TENSOR = 0, CLBM_NET_FP32 = 1 } clbm_net_math;

typedef struct {
  int32_t grid, in_ch, out_ch, base, levels, max_batch;
  int32_t math; /* clbm_net_math; any other value: CLBM_EINVAL */
} clbm_net_config;

/* Create a network with seeded He-uniform weights and zero biases. */
clbm_status clbm_net_create(const clbm_net_config* cfg, uint64_t seed, void* stream, clbm_net** out);

/* Number of parameters (weights and biases of every layer, in layer order;
 * each layer: weights [co][ci][k][k] then bias [co]). */
clbm_status clbm_net_param_count(const clbm_net* net, int64_t* count);

/* Copy the FP32 master parameters out / in (host or device array).  Setting
 * parameters also refreshes the BF16 copy and resets the Adam state. */
clbm_status clbm_net_get_params(const clbm_net* net, float* dst, int32_t on_device);
clbm_status clbm_net_set_params(clbm_net* net, const float* src, int32_t on_device);

/* y[N][out_ch][G][G] = net(x[N][in_ch][G][G]), 1 <= N <= max_batch (async).
 * x is copied into the network's input buffer and the output copied to y;
 * between the copies the forward pass runs as a CUDA graph captured on the
 * first call with this N (and replayed afterwards), unless the network's
 * stream cannot be captured (the legacy default stream), where it is
 * launched kernel by kernel. */
clbm_status clbm_net_forward(clbm_net* net, const float* x, int32_t n, float* y);

/* Loss and parameter gradients: loss = sum mask (y - t)^2 / (sum mask * out_ch)
 * with mask[N][G][G] (NULL = all ones; the sums are formed on the device, and
 * a mask that sums to zero returns CLBM_EINVAL with the gradients undefined).
 * grad (param_count floats, host or device, may be NULL) receives
 * dloss/dparams; *loss (may be NULL) the loss.  Synchronises once, at the end.
 * x, target and mask are copied into the network's own buffers first; the
 * pass (forward, loss, backward) then runs as a CUDA graph captured on the
 * first call with this N and mask-or-none, as for clbm_net_forward. */
clbm_status clbm_net_gradients(clbm_net* net, const float* x, const float* target,
                               const float* mask, int32_t n, float* grad, double* loss);

/* clbm_net_gradients followed by one Adam step (beta 0.9, 0.999, eps 1e-8). */
clbm_status clbm_net_train_step(clbm_net* net, const float* x, const float* target,
                                const float* mask, int32_t n, float lr, double* loss);

clbm_status clbm_net_destroy(clbm_net* net);
const char* clbm_net_last_error(const clbm_net* net);

/* Replace the current state by the mean of the current and the previous
 * post-collision states (both are kept by the ping-pong buffers), which
 * cancels exactly any component that flips sign from one step to the next.
 * The scheme on closed cavities has such a period-2 mode that does not
 * decay: a rest start barely excites it, but an initialisation from
 * predicted or interpolated fields can leave it at an amplitude that biases
 * every instantaneous quantity (for instance a wall Nusselt number that
 * alternates between two values).  Call after at least one step since the
 * initialisation (else CLBM_EINVAL); enqueued on the context stream.  Not
 * part of the paper's method. */
clbm_status clbm_damp_period2(clbm_ctx* ctx);

/* clbm_damp_period2 on every lattice of a batch (after a solve; synchronises). */
clbm_status clbm_batch_damp_period2(clbm_batch* b);

/* Number of time steps taken since the last initialisation. */
clbm_status clbm_time(const clbm_ctx* ctx, int64_t* t_out);

/* Shape of the fields clbm_init_fields reads and clbm_moments writes: nx
 * columns by the context's own rows (ny, or a slab's rows), i.e. each field
 * array holds nx * rows doubles.  Errors: CLBM_EINVAL for a NULL argument. */
clbm_status clbm_field_shape(const clbm_ctx* ctx, int64_t* nx_out, int64_t* rows_out);

/* Free every device and host resource of the context (NULL is allowed). */
clbm_status clbm_destroy(clbm_ctx* ctx);

/* Message of the last failure on this context ("" if none). */
const char* clbm_last_error(const clbm_ctx* ctx);

/* Static name of a status code. */
const char* clbm_status_string(clbm_status s);

#ifdef __cplusplus
}
#endif

#endif /* CLBM_H_ */
