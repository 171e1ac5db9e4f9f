/*
 * vlb.h -- C-ABI of the GB300 (sm_103a) volumetric lattice Boltzmann library
 * for general curvilinear meshes (H. Chen, "Volumetric Lattice Boltzmann
 * Models in General Curvilinear Coordinates: Theoretical Formulation").
 *
 * The paper's problem statement (section 2): given the node positions x(q)
 * of a structured mesh, indexed by the unit-spaced integer lattice q (section
 * 2.1), advance the cell-volume-weighted populations N_a = J f_a (Eq. 14) by
 *     N_a(q + c_a, t + 1) = N_a(q, t) + Omega_a(q, t) + deltaN_a(q, t)   (Eq. 12)
 * with BGK collision (Eq. 20), the curvilinear equilibrium (Eq. 33), the
 * discrete inertial force (Eqs. 27, 30, 31) and exact one-to-one advection
 * (Eq. 22), and map the result back to Euclidean fields (Eq. 34).
 *
 * Conventions shared by every entry point:
 *   - Status: every function returns VLB_OK (0) or a VLB_E* code; no C++
 *     exception crosses this boundary. vlb_last_error() returns a
 *     thread-local message describing the most recent failure.
 *   - Memory: all pointer arguments are HOST pointers owned by the caller
 *     and are only read or written during the call (inputs are copied).
 *     The library owns all device memory and frees it in the matching
 *     destroy call.
 *   - Layout: cell arrays are C-ordered [n0][n1][n2] (axis 2 fastest; n2 = 1
 *     in 2D); vector fields append a trailing [dim] axis. Population arrays
 *     are [q][n0][n1][n2] in the library's velocity order, which
 *     vlb_lattice() reports.
 *   - Streams: work is issued on params.stream (a cudaStream_t; NULL means
 *     the legacy default stream). vlb_step is asynchronous; calls that
 *     return host data synchronise the stream first.
 *   - Errors raised inside kernels (a fixed-point solve that hit its
 *     iteration cap) are sticky: they are reported by the next call that
 *     synchronises (vlb_sync, vlb_moments, vlb_get_state).
 */
#ifndef VLB_H
#define VLB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum vlb_status {
  VLB_OK = 0,
  VLB_EINVAL = 1,      /* bad argument, shape or unsupported combination */
  VLB_EGEOM = 2,       /* degenerate mesh: J <= 0 or |D_i - D_-i| = 0 (Eqs. 3, 5) */
  VLB_ENOCONV = 3,     /* the local implicit solve for F hit its iteration cap */
  VLB_ENOMEM = 4,      /* device or host allocation failed */
  VLB_ECUDA = 5,       /* a CUDA runtime call failed */
  VLB_ENONFINITE = 6   /* non-finite population or moment detected */
};

/* D3Q39: moment isotropy to 6th order (Eq. 10 in full, T0 = 2/3), so that the
 * equilibrium of Eq. 33 matches the third moment Q^eq of Eq. 32 exactly;
 * speeds up to 3. Periodic meshes only (every axis at least 3 cells, no
 * periodic rotation), FP64 populations, per-cell geometry; no batches and no
 * vlb_totals_noalloc. The paper names no velocity set with this property;
 * the weights are those of the published D3Q39 set. */
enum vlb_lattice_kind { VLB_D2Q9 = 9, VLB_D3Q19 = 19, VLB_D3Q39 = 39 };
enum vlb_bc { VLB_PERIODIC = 0, VLB_WALL = 1 };
enum vlb_precision { VLB_F64 = 0, VLB_F32 = 1, VLB_F16 = 2, VLB_BF16 = 3 };
enum vlb_reference { VLB_REF_UNIFORM = 0, VLB_REF_REST = 1 };
enum vlb_coef_mode { VLB_COEF_AUTO = 0, VLB_COEF_FULL = 1, VLB_COEF_PLANE = 2 };
enum vlb_wall_links { VLB_WALL_LINKS_ZERO = 0, VLB_WALL_LINKS_GHOST = 1 };

typedef struct vlb_mesh vlb_mesh; /* opaque, library-owned */
typedef struct vlb_sim vlb_sim;   /* opaque, library-owned */

/* Mesh description (section 2.1).
 *   x            host [n0][n1][n2][dim] node positions, copied by vlb_mesh_create
 *   bc[a]        VLB_PERIODIC or VLB_WALL for index axis a (axes >= dim ignored)
 *   period_shift periodic image across the +end of axis a:
 *   period_rot     x(q + n_a e_a) = R_a x(q) + shift_a, R_a row-major 3x3
 *                  (an all-zero matrix means identity; 2D uses its 2x2 block)
 *   dx           the representative spacing Delta x of Eq. 3; <= 0 means 1
 *   wall_links   Theta (Eq. 11) on links that cross a wall: VLB_WALL_LINKS_ZERO
 *                (the reflected particle never travels the link, Theta = 0) or
 *                VLB_WALL_LINKS_GHOST (Theta from the ghost nodes)
 * Behind a wall the ghost nodes needed by Eq. 1 are linear extrapolations of
 * the two nearest interior nodes along that axis. */
typedef struct {
  int32_t dim;      /* 2 or 3 */
  int32_t lattice;  /* VLB_D2Q9 with dim 2, VLB_D3Q19 or VLB_D3Q39 with dim 3 */
  int64_t n[3];     /* nodes per index axis, each >= 1 (>= 2 on a wall axis); n[2] = 1 in 2D */
  const double *x;
  int32_t bc[3];
  double period_shift[3][3];
  double period_rot[3][9];
  double dx;
  int32_t wall_links;
} vlb_mesh_desc;

/* Run parameters.
 *   tau          BGK relaxation time (Eq. 20), > 1/2
 *   precision    VLB_F64: FP64 populations and arithmetic;
 *                VLB_F32: FP32 populations, FP32 arithmetic, FP32 coefficients
 *                rounded from the FP64 precompute;
 *                VLB_F16 / VLB_BF16: populations stored in 16 bits (IEEE half
 *                or bfloat16) as deviations from a reference (see reference),
 *                FP32 arithmetic and coefficients as for VLB_F32. Storage
 *                rounding is not mass-conserving: each stored deviation is
 *                rounded to 11 (half) or 8 (bfloat16) significant bits
 *   reference    what a 16-bit population is stored relative to:
 *                VLB_REF_UNIFORM: N_a - w_a n_ref with one n_ref for the mesh
 *                (the scheme FP32/FP64 always use);
 *                VLB_REF_REST: N_a minus the rest state of Eq. 33 (rho = 1,
 *                U = 0) on the metric of the storage location's cell, which
 *                leaves only the flow in the stored value. Needs plane mode
 *                (the references of a column's neighbours are then
 *                per-column constants). Ignored for VLB_F32 and VLB_F64
 *   coef_mode    VLB_COEF_FULL streams one coefficient record per cell;
 *                VLB_COEF_PLANE stores one record per column of the fastest
 *                axis and is only accepted when the mesh geometry does not
 *                vary along that axis (checked to 1e-12 relative);
 *                VLB_COEF_AUTO picks PLANE when allowed, else FULL
 *   body_force   Euclidean acceleration G; adds rho G.g^i to F^i
 *   wall_u, wall_omega
 *                rigid motion of the wall on axis a, side s (0: index 0,
 *                1: index n-1): u_wall = wall_u + wall_omega x x_wall, with
 *                x_wall halfway between the boundary node and its ghost
 *   max_iter     iteration cap of the local fixed-point solve for F (0: 100)
 *   tol          its tolerance, max|dF| <= tol * max(rho, |F|)
 *                (0: 1e-14 in FP64, 1e-6 with FP32 arithmetic; never below 64 ulp of |F|)
 *   stream       cudaStream_t for all work of the simulation (NULL: default) */
typedef struct {
  double tau;
  int32_t precision;
  int32_t coef_mode;
  double body_force[3];
  double wall_u[3][2][3];
  double wall_omega[3][2][3];
  int32_t max_iter;
  double tol;
  void *stream;
  int32_t reference;
} vlb_params;

/* Per-mesh diagnostics filled by vlb_mesh_info. */
typedef struct {
  double J_min, J_max;          /* cell volume range (Eq. 5) */
  double feq_rest_min;          /* min over cells and directions of f^eq_a(rho = 1, U = 0) / w_a;
                                   negative means the mesh is outside the range where the
                                   rest state of Eq. 33 is a positive distribution */
  double ginv_diag_min, ginv_diag_max;
  int32_t invariant_fast_axis;  /* 1 when the geometry does not vary along the fastest axis */
  int64_t ncell;
} vlb_mesh_stats;

/* Velocity set used by the library: c[q][3] (zero-padded) and w[q] (host
 * outputs, either may be NULL). Section 2.1 lists D3Q19; D2Q9 is its planar
 * restriction. Weights are the standard ones with T0 = 1/3 (Eq. 10 to 4th order). */
int vlb_lattice(int32_t lattice, int32_t *c, double *w);

/* Build the mesh and run the FP64 geometry precompute on the current device:
 * D_{+-i} (Eq. 1), g_i with beta_i (Eq. 3), J (Eq. 5), g^i (Eq. 7), g^ij
 * (Eq. 8) and the contracted link coefficients
 *     K^i_a(q) = sum_j c^j_a Theta^i_j(q + c_a, q)     (Eq. 11)
 * (zero on links that cross a wall). Errors: VLB_EINVAL (shape, lattice,
 * bc), VLB_EGEOM (degenerate cell), VLB_ENOMEM, VLB_ECUDA. On failure *out is
 * NULL. Blocks until the precompute is done. */
int vlb_mesh_create(const vlb_mesh_desc *desc, vlb_mesh **out);
int vlb_mesh_info(const vlb_mesh *mesh, vlb_mesh_stats *out);
/* FP64 geometry read-back (host outputs, each may be NULL):
 * J [ncell], g_low [ncell][dim][dim] (row i = g_i), ginv [ncell][dim][dim],
 * K [ncell][q][dim] (row a = K_a). */
int vlb_mesh_geometry(const vlb_mesh *mesh, double *J, double *g_low, double *ginv, double *K);
void vlb_mesh_destroy(vlb_mesh *mesh);

/* Create a simulation on a mesh and set N_a = J f^eq_a(rho, U, U~ = U)
 * (Eqs. 14, 33) with U^i = u . g^i. rho [ncell] and u [ncell][dim] are host
 * arrays (Euclidean velocity). The mesh must outlive the simulation.
 * Errors: VLB_EINVAL (tau <= 1/2, bad precision, coef_mode or reference,
 * VLB_REF_REST without plane mode, moving walls on a cell touching two
 * walls, a D3Q39 mesh with a precision other than VLB_F64 or with
 * VLB_COEF_PLANE), VLB_ENOMEM, VLB_ECUDA. */
int vlb_init(const vlb_mesh *mesh, const vlb_params *params, const double *rho, const double *u,
             vlb_sim **out);
/* Re-initialise the populations from host fields as vlb_init does (no allocation). */
int vlb_reset(vlb_sim *sim, const double *rho, const double *u);

/* Advance nsteps time steps (Eq. 12 with Eq. 22), one fused pull-collide-push
 * kernel launch per step, alternating the two in-place A-A layouts. Returns
 * after queueing the launches. */
int vlb_step(vlb_sim *sim, int64_t nsteps);

/* Synchronise the stream and report any sticky kernel error. */
int vlb_sync(vlb_sim *sim);

/* Moments at the current time (host outputs, each may be NULL):
 *   rho [ncell]                 rho = sum_a N_a / J           (Eq. 15)
 *   u [ncell][dim]              u  = U^i g_i                  (Eq. 34)
 *   u_tilde [ncell][dim]        u~ = U~^i g_i, U~ = U + F/(2 rho) (text after Eq. 32)
 *   totals[7]                   mass = sum N, P = sum e_a(q) N_a (dim values),
 *                               M = sum 1/2 [e_a(q) + e_a(q - c_a)] N_a (dim values),
 *                               laid out [mass, P0, P1, P2, M0, M1, M2], reduced in FP64
 * F is the converged solution of the same local fixed point the step solves.
 * Synchronises; returns VLB_ENONFINITE if a moment is not finite. */
int vlb_moments(vlb_sim *sim, double *rho, double *u, double *u_tilde, double *totals);

/* Arrived populations N_a(q, t) as FP64 [q][ncell] (host), whatever the
 * in-place layout of the current step parity; and the inverse. */
int vlb_get_state(vlb_sim *sim, double *N);
int vlb_set_state(vlb_sim *sim, const double *N);

/* Steps taken since vlb_init / vlb_reset / vlb_set_state. */
int64_t vlb_time(const vlb_sim *sim);
/* Bytes per cell of the coefficient record and whether it is one per column
 * (plane mode); for reporting. */
int vlb_sim_layout(const vlb_sim *sim, int32_t *coef_per_cell, int32_t *plane_mode,
                   int64_t *coef_records);

void vlb_destroy(vlb_sim *sim);
const char *vlb_last_error(void);

/* ---- Batches: many simulations advanced by one kernel launch per time step.
 * Each member's time step is the same fused stream-and-collide of Eq. 12 /
 * Eq. 22 as vlb_step (the per-cell arithmetic is identical, so a batch gives
 * bit-for-bit the populations of stepping each member alone). The members'
 * tiles (128 or, after vlb_batch_tune, possibly 64 cells along the fastest
 * axis) are cut into runs and every run is one block of a single launch; a member's work thus never waits for a launch
 * of its own, which is what pays for many small meshes.
 *   sims    nsims >= 1 simulations on the current device with the same
 *           lattice, precision (VLB_F32 or VLB_F64), coefficient mode (all
 *           plane or all full), time parity and stream, each with fewer than
 *           2^31 / q cells; they must outlive the batch and are not copied
 * Errors: VLB_EINVAL (mismatch, 16-bit storage, D3Q39 members, NULL),
 * VLB_ENOMEM, VLB_ECUDA. */
typedef struct vlb_batch vlb_batch;
int vlb_batch_create(vlb_sim *const *sims, int32_t nsims, vlb_batch **out);
/* Advance every member nsteps steps (asynchronous on the members' stream;
 * errors raised by kernels are sticky per member, see vlb_sync). Whole runs
 * of 32 steps replay a CUDA graph of 32 launches built on first use. */
int vlb_batch_step(vlb_batch *b, int64_t nsteps);
/* Pick the block shape and the run length (tiles per block) by timing. The
 * shapes are the tile width (threads per block, cells along the fastest
 * axis: 128 or 64; narrow tiles waste fewer threads at the ragged end of
 * short rows) with the resident blocks per SM that the registers are cut
 * for (four shapes for VLB_F32 members, two for VLB_F64); with each shape,
 * run lengths of about 1, 2, 4 and 8 runs per resident block. Every
 * candidate runs `steps` steps on the members, so the simulations advance by
 * the count vlb_batch_tune_steps gives. Blocks until done. run_length_out
 * may be NULL. */
int vlb_batch_tune(vlb_batch *b, int32_t steps, int64_t *run_length_out);
/* The number of steps vlb_batch_tune(b, steps, ...) advances every member by. */
int vlb_batch_tune_steps(const vlb_batch *b, int32_t steps, int64_t *advanced);
/* Use block shape `shape` with its default run length, about two runs per
 * resident block. VLB_F32 members: 0 .. 3 = 128 threads cut for 3, 6 or 8
 * resident blocks per SM (the first is the single-mesh step's budget), then
 * 64 threads cut for 12; VLB_F64 members: 0 .. 1 = 128 threads for 2 blocks,
 * 64 threads for 4. EINVAL outside that range. */
int vlb_batch_set_shape(vlb_batch *b, int32_t shape);
/* The block shape in use: threads per block (= tile width) and the resident
 * blocks per SM its kernel's registers were cut for. Either may be NULL. */
int vlb_batch_shape(const vlb_batch *b, int32_t *threads, int32_t *min_blocks);
/* Blocks (tile runs) per launch and tiles per run; for reporting. */
int vlb_batch_layout(const vlb_batch *b, int64_t *blocks, int64_t *run_length, int64_t *cells);
void vlb_batch_destroy(vlb_batch *b);

/* The paper has no counterpart to this call: it is a service for callers that
 * cannot allocate device memory -- code whose device memory comes from a fixed
 * budget or from a pool allocator it does not own, and latency-bound
 * monitoring loops in which an allocation, which can synchronise the device,
 * is not acceptable. vlb_moments allocates its staging buffers on first use;
 * this call computes the same totals[7] (mass, P, M) and allocates nothing.
 *   d_totals  DEVICE pointer to 7 doubles owned by the caller, written
 *             asynchronously on the simulation's stream (layout as in
 *             vlb_moments; unused components of 2D runs are zero).
 * Its per-block partial sums live in a fixed device array of 4096 x 7 doubles
 * (224 KiB) that every device which loads the library holds until the process
 * exits; meshes of more than 4096 x 16384 = 67,108,864 cells are rejected
 * with VLB_EINVAL. The kernels are those of vlb_moments' totals; they run on
 * the mesh's device (the call makes it current for the launches and restores
 * the caller's device). The first call on a device looks up that array's
 * device address; make the first call before any stream capture. All calls share the
 * array, so calls that overlap on the GPU (for example on two streams) race
 * and give wrong totals; every call writes each slot it reads before reading
 * it, so nothing needs clearing. D2Q9 and D3Q19 simulations only (D3Q39:
 * VLB_EINVAL, use vlb_moments). Errors: VLB_EINVAL, VLB_ECUDA. Kernel-raised
 * errors are not checked here (no synchronisation). */
int vlb_totals_noalloc(vlb_sim *sim, double *d_totals);

#ifdef __cplusplus
}
#endif
#endif
