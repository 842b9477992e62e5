/*
 * pic.h -- C ABI of libpic.so, the GB300 (sm_103a) particle hot path of the
 * particle-in-cell method of Gassmoeller, Heien, Puckett & Bangerth,
 * "Flexible and scalable particle-in-cell methods for massively parallel
 * computations" (arXiv 1612.03369).
 *
 * What the library computes, per call:
 *   - particle generation from local coordinates  (Sec. 2.2, Remark "local generation")
 *   - evaluation of the Q2 velocity u_h at stored reference coordinates
 *     x-hat = Phi_K^{-1}(x)                        (Sec. 2.3, Remark 2.1)
 *   - forward Euler / RK2 / RK4 advection          (Sec. 2.3)
 *   - location of every stage point and of the new position: inverse of the
 *     (bi/tri)linear cell map by Newton, then the vertex-neighbour walk, then
 *     a search over all cells                      (Sec. 2.4)
 *   - re-binning into a store sorted by (cell, id), lost particles removed
 *                                                  (Sec. 2.1 data structure, Sec. 2.4 listing)
 *   - arithmetic per-cell averages of a property   (Sec. 2.7, scheme (ii))
 *
 * Conventions
 *   - Every call that takes a `stream` (a cudaStream_t, 0 = legacy default)
 *     is asynchronous on it, unless its comment says it synchronises.
 *   - Arguments are checked on the host before anything is enqueued; a bad
 *     argument returns PIC_ERR_ARG and enqueues nothing.  pic_last_error()
 *     gives a message for the last failure on the calling thread.
 *   - Conditions found on the device (Newton non-convergence in a cell that
 *     is then treated as not containing the point, capacity overflow, an
 *     out-of-range index caught by a bounds check) are latched in a device
 *     status word that pic_get_state() returns; the kernels never trap.
 *   - Lost particles (a stage point or the new position in no cell, option 3
 *     of the Sec. 2.4 listing) are not errors: they are removed and counted.
 *   - Handles are not thread-safe; use one stream per particle handle.
 *   - Coordinates are FP64.  Layouts are structure-of-arrays, component
 *     major: an array documented as [dim][n] holds component a of item i at
 *     a*n + i.
 *   - Mesh topology is structured: n_cells[0] x n_cells[1] (x n_cells[2])
 *     cells, cell (i,j,k) has index i + nx*(j + ny*k); vertex (i,j,k) has
 *     index i + (nx+1)*(j + (ny+1)*k); Q2 node (I,J,K) has index
 *     I + (2nx+1)*(J + (2ny+1)*K), and node (2i+a, 2j+b, 2k+c), a,b,c in
 *     {0,1,2}, is node (a,b,c) of cell (i,j,k).  Vertex positions are free
 *     (any non-degenerate (bi/tri)linear cells).
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_mesh_s *pic_mesh;           /* owned by the library; pic_destroy_mesh */
typedef struct pic_particles_s *pic_particles; /* owned by the library; pic_destroy_particles */
typedef struct pic_tape_s *pic_tape;           /* owned by the library; pic_destroy_tape */
typedef struct pic_ensemble_s *pic_ensemble;   /* owned by the library; pic_ensemble_destroy */

typedef enum {
  PIC_OK = 0,
  PIC_ERR_ARG = 1,           /* invalid argument; nothing was enqueued */
  PIC_ERR_OOM = 2,           /* device allocation failed */
  PIC_ERR_CAPACITY = 3,      /* more particles than the store's capacity */
  PIC_ERR_CUDA = 4,          /* a CUDA runtime call failed (message in pic_last_error) */
  PIC_ERR_NOT_CONVERGED = 5, /* reserved for callers that treat Newton failure as fatal */
  PIC_ERR_TIMEOUT = 6,       /* a bounded device wait ran out */
  PIC_ERR_STATE = 7          /* call not valid in the handle's current state */
} pic_status;

typedef enum { PIC_EULER = 1, PIC_RK2 = 2, PIC_RK4 = 4 } pic_integrator;
typedef enum { PIC_FP64 = 0, PIC_FP32_BASIS = 1, PIC_FP32_BASIS_STAGE_DF = 2 } pic_precision;
typedef enum { PIC_AVG_ARITHMETIC = 0, PIC_AVG_GEOMETRIC = 1, PIC_AVG_HARMONIC = 2 } pic_average;

/* Bits of the device status word (pic_get_state). */
#define PIC_STATUS_NEWTON_NONCONV 0x1u /* Newton hit its iteration cap in some candidate cell */
#define PIC_STATUS_CAPACITY 0x2u       /* a store or list overflowed; data past capacity dropped */
#define PIC_STATUS_GLOBAL_SEARCH 0x4u  /* the all-cells search ran for some point */
#define PIC_STATUS_BOUNDS 0x8u         /* a bounds check caught an out-of-range index; access skipped */
#define PIC_STATUS_TIMEOUT 0x10u       /* a bounded device wait ran out; the kernel carried on without it */

/* Mesh of (bi/tri)linear cells with a Q2 velocity field (Sec. 2.1, 2.3).
 *   dim       2 or 3
 *   n_cells   [dim] cells per axis, each >= 1; total cells < 2^31, Q2 nodes < 2^32
 *   vertices  [dim][nverts] FP64 positions, nverts = prod(n_cells[a]+1);
 *             on the device if vertices_on_device, else host memory
 *   stream    stream for the upload and the per-cell set-up kernels
 *   out       receives the handle
 * The library copies the vertices; the caller keeps ownership of its array.
 * Synchronises `stream` before returning (the handle is usable at once).
 * Errors: PIC_ERR_ARG, PIC_ERR_OOM, PIC_ERR_CUDA. */
pic_status pic_create_mesh(int dim, const int *n_cells, const double *vertices, int vertices_on_device, void *stream,
                           pic_mesh *out);
pic_status pic_destroy_mesh(pic_mesh mesh);

/* Q2 nodal velocity u_h (Sec. 2.3: the finite-element field; evaluating it at
 * the particle positions is where the paper says the advection spends most).
 *   U       [dim][nnodes] FP64, device or host, nnodes = prod(2*n_cells[a]+1):
 *           the field at the start of a time step, u_h^n
 *   U_next  NULL for a steady field, or the field at the end of the step,
 *           u_h^{n+1}: every step of pic_advect then evaluates stage s at
 *           t^n + c_s dt with u-tilde_h = (1 - c_s) u_h^n + c_s u_h^{n+1}
 *           (Sec. 2.3, eq. position-ode-approx; c = 0, 1/2, 1/2, 1 for RK4,
 *           0, 1/2 for RK2, 0 for Euler).  Not supported by the adjoint.
 * The library copies the fields (stream-ordered); the caller may reuse them.
 * Errors: PIC_ERR_ARG, PIC_ERR_CUDA. */
pic_status pic_set_velocity_dofs(pic_mesh mesh, const double *U, const double *U_next, void *stream);

/* Staged upload of the next field, so that its copy overlaps the current
 * step (a flow solver hands over u_h^{n+1} while the particles take step n).
 * pic_stage_velocity_dofs copies U ([dim][nnodes] FP64, host (pinned for an
 * asynchronous copy) or device) into a staging buffer on copy_stream; the
 * caller keeps U unchanged until the copy has run (copy_stream order).
 * pic_commit_velocity_dofs makes the staged field the field of the mesh on
 * `stream`: `stream` waits for the copy, then the FP32 and double-float
 * copies are rebuilt there.  A staging buffer is allocated on first use; a
 * later stage waits (on the device) until the previous commit's conversions
 * have released it.  U_next, if set, is unchanged.
 * Errors: PIC_ERR_ARG; PIC_ERR_STATE (no first field set, a stage while one
 * is pending, a commit with nothing staged); PIC_ERR_OOM; PIC_ERR_CUDA. */
pic_status pic_stage_velocity_dofs(pic_mesh mesh, const double *U, void *copy_stream);
pic_status pic_commit_velocity_dofs(pic_mesh mesh, void *stream);

/* Generation from local coordinates (Sec. 2.2, Remark "local generation"):
 * cells are visited in index order and n_K particles created in cell K with
 * reference coordinates x-hat uniform in [0,1)^dim, position x = Phi_K(x-hat),
 * id = first_id + (number of particles created before it).  x-hat_j of the
 * g-th particle is (r >> 11) * 2^-53 with r output number g*dim + j (0-based)
 * of SplitMix64 (Steele, Lea & Flood 2014) seeded with `seed`.
 *   per_cell       [n_cells] u32 on the device, or NULL for uniform_count per cell
 *   n_props        properties per particle (0..16), initialised to 0
 *   capacity       store capacity (>= number created); 0 = exactly the number created
 *   out            receives the handle; the store is sorted by (cell, id)
 * Synchronises `stream` (reads the total count).  Errors: PIC_ERR_ARG,
 * PIC_ERR_CAPACITY, PIC_ERR_OOM, PIC_ERR_CUDA. */
pic_status pic_seed_particles(pic_mesh mesh, const uint32_t *per_cell, uint32_t uniform_count, uint64_t seed,
                              uint64_t first_id, int n_props, size_t capacity, void *stream, pic_particles *out);
pic_status pic_destroy_particles(pic_particles parts);

/* Generation with a density rho(x) (Sec. 2.2, the listing for N particles
 * and the Metropolis-Hastings paragraph).  rho is given by its values at the
 * mesh vertices, [nverts] FP64 device, >= 0; rho_h is its (bi/tri)linear
 * interpolant.
 *
 * pic_cell_weights: w[K] = int_K rho_h dx ([n_cells] FP64 device), by the
 * tensor 2-point Gauss rule on the reference cell, exact for these fields.
 * Errors: PIC_ERR_ARG, PIC_ERR_CUDA. */
pic_status pic_cell_weights(pic_mesh mesh, const double *rho, double *w, void *stream);

/* pic_draw_cell_counts: particles per cell for n_particles draws.  The
 * accumulated weights acc_K = w_0 + .. + w_K form one left fold; draw i takes
 * u_i = (SplitMix64 output i of `seed`) >> 11 times 2^-53 and goes to the
 * first cell with acc_K > W u_i, W = acc_{n_cells-1} (or to the last cell of
 * positive weight if W u_i rounded up to W).  Zero-weight cells get none.
 *   w       [n_cells] FP64 device, finite and >= 0, positive sum
 *   counts  [n_cells] u32 device (overwritten); usable as pic_seed_particles'
 *           or pic_seed_particles_mh's per_cell
 * The fold runs on one warp (one-time set-up cost, about 5 ns per cell).
 * Synchronises `stream` to check the weights.
 * Errors: PIC_ERR_ARG (bad weights), PIC_ERR_CAPACITY (n_particles >= 2^32),
 * PIC_ERR_OOM, PIC_ERR_CUDA. */
pic_status pic_draw_cell_counts(uint32_t n_cells, const double *w, uint64_t n_particles, uint64_t seed,
                                uint32_t *counts, void *stream);

/* pic_seed_particles_mh: like pic_seed_particles, but the reference
 * coordinates in cell K come from a Metropolis-Hastings chain with target
 * rho-hat(x-hat) = rho_h(Phi_K(x-hat)) |det grad-hat Phi_K(x-hat)| and
 * uniform proposals on the reference cell, started at its centre; the chain
 * runs thinning * per_cell[K] steps and every thinning-th state becomes a
 * particle.  Step s of cell K's chain is global step g = thinning * (particles
 * of the cells before K) + s and uses SplitMix64 outputs g (dim+1) + a for
 * proposal coordinate a and g (dim+1) + dim for the acceptance uniform u; the
 * proposal y is accepted when u rho-hat(current) < rho-hat(y).  rho-hat is a
 * fixed sequence of correctly rounded operations (documented in
 * csrc/generate.cu), so the chains do not depend on the device.
 * Ids first_id + creation index; properties 0.  Synchronises `stream`.
 *   per_cell  [n_cells] u32 device;  rho  [nverts] FP64 device;  thinning >= 1
 * Errors: PIC_ERR_ARG, PIC_ERR_CAPACITY, PIC_ERR_OOM, PIC_ERR_CUDA. */
pic_status pic_seed_particles_mh(pic_mesh mesh, const uint32_t *per_cell, const double *rho, uint32_t thinning,
                                 uint64_t seed, uint64_t first_id, int n_props, size_t capacity, void *stream,
                                 pic_particles *out);

/* Prescribed particle locations (Sec. 2.2, second listing): every point is
 * located by the all-cells search of pic_locate_points (lowest index on
 * shared faces); points in no cell are skipped.  The k-th point found, in
 * input order, gets id first_id + k; the store is sorted by (cell, id).
 *   x          [dim][n] FP64 device positions
 *   capacity   store capacity (0 = the number found)
 *   n_outside  receives the number skipped (may be NULL)
 * Synchronises `stream`.  Errors: PIC_ERR_ARG, PIC_ERR_CAPACITY, PIC_ERR_OOM,
 * PIC_ERR_CUDA. */
pic_status pic_import_particles(pic_mesh mesh, size_t n, const double *x, uint64_t first_id, int n_props,
                                size_t capacity, void *stream, pic_particles *out, size_t *n_outside);

/* Property p of every particle from values [N] (device, store order).
 * Sec. 2.6: a run-time number of scalars per particle. */
pic_status pic_set_properties(pic_particles parts, int prop, const double *values, void *stream);

/* n_steps time steps (Sec. 2.3 and the Sec. 2.4 listing), each:
 *   - every particle advances with the integrator; the first stage uses the
 *     stored (cell, x-hat); every later stage point and the new position are
 *     located (Newton in the hint cell, vertex-neighbour walk, all-cells
 *     search; the lowest cell index owns points on shared faces)
 *   - a particle with a stage point or new position in no cell is lost
 *   - the store is rebuilt sorted by (cell, id) with lost particles removed
 * The particle data move to their sorted slots inside the next step's
 * advect.  After the last step of a call the new order is computed but left
 * pending: the next pic_advect applies it inside its first advect, and
 * pic_interpolate_to_cells reads through it; every other call on the store
 * applies it first (one gather on that call's stream).  Every call thus sees
 * the store sorted by (cell, id); pic_get_state and pic_cell_offsets already
 * describe the new order.
 * Integrators (classical forms, reading of the garbled printed formulas):
 *   PIC_EULER x + dt u(x);  PIC_RK2 midpoint x + dt u(x + dt/2 u(x));
 *   PIC_RK4 x + (k1 + 2 k2 + 2 k3 + k4)/6, k1 = dt u(x), k2 = dt u(x + k1/2),
 *   k3 = dt u(x + k2/2), k4 = dt u(x + k3).
 *   precision  PIC_FP64: FP64 storage, arithmetic in double-float on the FP32
 *              pipe (~2^-48 relative; within 1e-12 of the FP64 oracle);
 *              PIC_FP32_BASIS: the Q2 basis and contraction in FP32 on
 *              reference coordinates; positions accumulate in double-float
 *              and are stored in FP64; the new position of each step is
 *              located with the double-float residual and convergence test
 *              (its stored x-hat good to ~1e-14), the stage points with the
 *              FP32 Newton alone (x-hat to ~1e-7, all an FP32 basis can use);
 *              PIC_FP32_BASIS_STAGE_DF: the same with the double-float
 *              residual and convergence test at the stage points too
 * Errors: PIC_ERR_ARG (mesh/store mismatch, dt not finite, n_steps < 0,
 * velocity not set), PIC_ERR_CUDA. */
pic_status pic_advect(pic_particles parts, pic_mesh mesh, double dt, pic_integrator integrator,
                      pic_precision precision, int n_steps, void *stream);

/* Property ODEs integrated along the particle paths (Sec. 2.6):
 *   damage               d' = alpha |eps-dot| - beta d,  eps-dot = (G + G^T)/2,
 *                        |.| the Frobenius norm
 *   deformation gradient F' = G F  (start from F = I with pic_set_properties)
 * with G = grad u_h at the particle.  Both ride on the position as one
 * system, stepped by the same integrator over the same located stage points,
 * so positions, cells and order are exactly those of pic_advect (FP64 form);
 * G is evaluated in double-float arithmetic (~2^-44 relative) at every stage.
 *   damage       property slot of d, or -1
 *   alpha, beta  material parameters of the damage law (finite)
 *   deformation  first of dim*dim consecutive property slots holding F
 *                row-major (F_ij in slot deformation + i*dim + j), or -1 */
typedef struct {
  int damage;
  double alpha, beta;
  int deformation;
} pic_property_odes;

/* n_steps of pic_advect (FP64 form) that also advance the properties of
 * `odes` (host struct, read during the call).  Other properties ride along.
 * Scratch: 4 (4 + 8 dim + 8 dim^2) bytes per particle of capacity (stage
 * records and gradients), allocated with the store on the first call.
 * Errors: PIC_ERR_ARG (as pic_advect; a slot outside the store's properties;
 * damage overlapping the deformation slots), PIC_ERR_STATE (the mesh carries
 * a second velocity field: the property ODEs take the steady field),
 * PIC_ERR_OOM (the scratch), PIC_ERR_CUDA. */
pic_status pic_advect_properties(pic_particles parts, pic_mesh mesh, double dt, pic_integrator integrator,
                                 int n_steps, const pic_property_odes *odes, void *stream);

/* Adjoint (gradients with respect to the velocity field).
 * pic_advect_record: n_steps of pic_advect (FP64 form) that also keep, for
 * every step, each particle's stage records (the located cell and the
 * reference coordinates of every stage point, as the step used them) and the
 * rebin's permutation; the store ends where pic_advect would leave it, bit
 * for bit.  Memory: (20 + 32 dim) bytes per particle of capacity per step,
 * plus work arrays.
 * The mesh and its velocity must not change until the tape is used.
 * Errors: PIC_ERR_ARG, PIC_ERR_OOM, PIC_ERR_CUDA. */
pic_status pic_advect_record(pic_particles parts, pic_mesh mesh, double dt, pic_integrator integrator, int n_steps,
                             void *stream, pic_tape *out);

/* What a tape keeps per step.
 *   PIC_TAPE_STAGES       the stage records above, read back by the sweep:
 *                         (20 + 32 dim) bytes per particle of capacity
 *   PIC_TAPE_CHECKPOINTS  the store at the start of the step (x, x-hat, cell)
 *                         and the permutation: (8 + 16 dim) bytes per particle
 *                         of capacity; the sweep replays each step from its
 *                         checkpoint with the forward's own particle step, so
 *                         the gradient is the same bit for bit, at the cost of
 *                         one more advect per step.
 * pic_advect_record is pic_advect_record_tape with PIC_TAPE_STAGES.
 * Errors: those of pic_advect_record; an unknown kind is PIC_ERR_ARG. */
typedef enum { PIC_TAPE_STAGES = 0, PIC_TAPE_CHECKPOINTS = 1 } pic_tape_kind;
pic_status pic_advect_record_tape(pic_particles parts, pic_mesh mesh, double dt, pic_integrator integrator,
                                  int n_steps, pic_tape_kind kind, void *stream, pic_tape *out);

/* Reverse sweep of a recorded run (adjoint of the Sec. 2.3 integrators over
 * located stages; a stage's cell is held fixed, where u_h is continuous):
 *   dL_dxfinal [dim][N_final] device: dL/dx of the particles alive at the end,
 *              in the store order at the end (pic_export order)
 *   dL_dU      [dim][nnodes] device, overwritten with dL/dU
 *   dL_dx0     [dim][N_0] device or NULL: dL/dx at the start, store order at
 *              the start (0 for particles lost during the run)
 * The velocity gradients at the recorded stage points and the adjoint
 * variables are carried in double-float arithmetic (~2^-44 relative).
 * Per-stage contributions are summed per cell in (cell, stage, particle slot)
 * order and the cells into the nodes in cell order: the result is
 * reproducible bit for bit.  Errors: PIC_ERR_ARG, PIC_ERR_CUDA. */
pic_status pic_tape_adjoint(pic_tape tape, const double *dL_dxfinal, double *dL_dU, double *dL_dx0, void *stream);
pic_status pic_destroy_tape(pic_tape tape);

/* Ensemble of independent problems advanced together (the imbalance
 * discussion of Sec. 2.5 is the motivation: problems of uneven size share
 * one device).  All problems have the same dimension; problem p uses
 * meshes[p] (with its velocity set) and its own time step.
 *   per_cell        [n_problems] pointers to device [n_cells_p] u32 counts, or
 *                   NULL (then uniform_counts[p] particles in every cell)
 *   seeds           [n_problems] generator seeds (ids count from 0 per problem)
 * Problem p is seeded exactly as pic_seed_particles would seed it alone, and
 * advances with the same per-particle arithmetic: each problem matches its
 * solo run bit for bit.  Synchronises.  At most 128 problems; steady fields
 * only (the views of the meshes are taken at creation).
 * Errors: PIC_ERR_ARG, PIC_ERR_OOM, PIC_ERR_CUDA. */
pic_status pic_ensemble_create(int n_problems, const pic_mesh *meshes, const uint32_t *const *per_cell,
                               const uint32_t *uniform_counts, const uint64_t *seeds, int n_props, void *stream,
                               pic_ensemble *out);
pic_status pic_ensemble_destroy(pic_ensemble ens);

/* Time step of every problem ([n_problems] host doubles).  Synchronises. */
pic_status pic_ensemble_set_dt(pic_ensemble ens, const double *dts, void *stream);

/* n_steps of every problem (advect with located stages + rebin).
 *   mode 0: per step, the ensemble advect kernel and the rebin kernels
 *   mode 1: one persistent cooperative kernel for all n_steps; phases are
 *           separated by a grid barrier whose waits give up after a time
 *           limit (then PIC_ERR_TIMEOUT); synchronises to read that status
 *   In both modes the advect's warps take tiles of particles (32 unless the
 *   autotuner chose another size) from a work counter.
 *   use_graph: capture the launches once (per n_steps, mode, integrator and
 *           buffer parity) into a CUDA graph and replay it
 * Errors: PIC_ERR_ARG, PIC_ERR_TIMEOUT, PIC_ERR_CUDA. */
pic_status pic_ensemble_run(pic_ensemble ens, pic_integrator integrator, int n_steps, int mode, int use_graph,
                            void *stream);

/* Autotuner of the persistent kernel: times one step for every (blocks per
 * SM from 1 to the occupancy limit, tile of 32, 128 or 512 particles claimed
 * by a warp at a time) candidate on a snapshot of the store, keeps the
 * fastest for later runs of both modes (the per-step mode takes the tile
 * size) and restores the store.  Any out pointer may be NULL.  Synchronises.
 * Errors: PIC_ERR_ARG, PIC_ERR_OOM, PIC_ERR_TIMEOUT, PIC_ERR_CUDA. */
pic_status pic_ensemble_tune(pic_ensemble ens, pic_integrator integrator, int *blocks_per_sm, int *tile,
                             double *best_ms, void *stream);

/* Totals over all problems (as pic_get_state).  Synchronises. */
pic_status pic_ensemble_state(pic_ensemble ens, size_t *n_alive, size_t *n_lost, uint32_t *status_word);

/* Problem `problem`'s particles in (cell, id) order: x, xhat [dim][n] FP64,
 * id [n], cell [n] (cells of that problem's mesh); *n_out = n.  Any output
 * may be NULL; device or host memory; size the arrays from a first call with
 * all outputs NULL.  Synchronises. */
pic_status pic_ensemble_export(pic_ensemble ens, int problem, double *x, double *xhat, uint64_t *id, uint32_t *cell,
                               size_t *n_out, void *stream);

/* Failure-detection self-test of the bounded grid barrier: runs it with one
 * arrival fewer than it expects, so every wait must run out after timeout_s
 * (0 < timeout_s <= 10).  Returns PIC_ERR_TIMEOUT when the barrier reported
 * the timeout (the expected outcome); the context stays usable. */
pic_status pic_barrier_selftest(double timeout_s, void *stream);

/* Re-locate every particle at its current position, using its current cell
 * as the hint (Sec. 2.4), then rebuild the store as pic_rebin does.
 * Errors: PIC_ERR_ARG, PIC_ERR_CUDA. */
pic_status pic_locate(pic_particles parts, pic_mesh mesh, void *stream);

/* Rebuild the store sorted by (cell, id), dropping particles marked lost
 * (Sec. 2.1 "sorted by their containing cells", Sec. 2.4 batched
 * re-insertion).  Uses the cells found by the last locate.
 * Errors: PIC_ERR_ARG, PIC_ERR_CUDA. */
pic_status pic_rebin(pic_particles parts, void *stream);

/* Stateless point location (Sec. 2.4, and Sec. 2.2 prescribed positions):
 *   x        [dim][n] device positions
 *   hint     [n] device start cells, or NULL (then cell 0's neighbourhood is
 *            skipped and every point goes to the all-cells search)
 *   cell_out [n] device owner cells (lowest index on shared faces), or
 *            0xFFFFFFFF if no cell contains the point
 *   xhat_out [dim][n] device reference coordinates in the owner (0 if none)
 * Errors: PIC_ERR_ARG, PIC_ERR_CUDA. */
pic_status pic_locate_points(pic_mesh mesh, size_t n, const double *x, const uint32_t *hint, uint32_t *cell_out,
                             double *xhat_out, void *stream);

/* Stateless form of the rebin (Sec. 2.1 "sorted by their containing cells",
 * Sec. 2.2 "first put cell-particle pairs into a linear array ... then fill
 * the multi-map"): the order of n items by (cell, id).
 *   cell      [n] u32 device; items with cell >= n_cells (0xFFFFFFFF = lost)
 *             are left out
 *   id        [n] u64 device, unique among the items kept
 *   perm      [n] u32 device: perm[0 .. kept-1] = item indices in (cell, id)
 *             order; entries past `kept` are not written
 *   cell_off  [n_cells + 1] u32 device: items of cell K are
 *             perm[cell_off[K] .. cell_off[K+1]-1]; cell_off[n_cells] = kept
 * Allocates its scratch (about 12 B per item + 8 B per cell) on `stream`
 * with cudaMallocAsync and frees it there.  Errors: PIC_ERR_ARG, PIC_ERR_CUDA. */
pic_status pic_sort_by_cell(size_t n, const uint32_t *cell, const uint64_t *id, uint32_t n_cells, uint32_t *perm,
                            uint32_t *cell_off, void *stream);

/* pic_sort_by_cell without any device allocation.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory
 * where they sort (an application pool that has reserved the device, an
 * embedder whose allocator owns every byte, or a loop that must not enter the
 * driver's allocator, which can synchronise or fail).  Arguments, outputs and
 * results are those of pic_sort_by_cell.
 *   Limits: n <= 524288 items and n_cells <= 131072 cells; larger requests
 *   return PIC_ERR_ARG with a message and enqueue nothing.
 *   Scratch: a fixed device array of 7,340,800 bytes inside the library
 *   (the scratch of one sort at both limits).  Under CUDA's lazy module
 *   loading (the default) a device receives the array on this entry point's
 *   first call there, which looks up its address (cudaGetSymbolAddress): make
 *   that first call (n = 0 is enough) before the application reserves the
 *   device's memory for itself, and outside any stream capture.  The device
 *   then holds the array until the process exits.  Calls outside a capture
 *   look the address up again (no allocation once loaded; correct after a
 *   cudaDeviceReset); a call on a capturing stream uses the address of the
 *   device's last call outside capture, and fails with PIC_ERR_STATE if
 *   there was none.
 *   All calls share the array, and it keeps the last call's contents (each
 *   call clears what it needs at zero), so calls whose work overlaps on the
 *   GPU (on different streams, or from host threads without ordering) race;
 *   order them, for example on one stream.
 * Calls no allocation routine.  Errors: PIC_ERR_ARG, PIC_ERR_STATE, PIC_ERR_CUDA. */
pic_status pic_sort_by_cell_noalloc(size_t n, const uint32_t *cell, const uint64_t *id, uint32_t n_cells,
                                    uint32_t *perm, uint32_t *cell_off, void *stream);

/* Particle -> cell transfer (Sec. 2.7, scheme (ii)): over the particles of
 * cell K, in store order (deterministic),
 *   PIC_AVG_ARITHMETIC  sum v / n_K
 *   PIC_AVG_GEOMETRIC   exp(sum log v / n_K)  (NaN if the cell holds a v <= 0)
 *   PIC_AVG_HARMONIC    n_K / sum(1 / v)      (NaN if the cell holds a v <= 0)
 * count[K] = n_K; empty cells get empty_fill.
 *   avg    [n_cells] FP64 device;  count  [n_cells] u32 device (may be NULL)
 * Errors: PIC_ERR_ARG, PIC_ERR_CUDA. */
pic_status pic_interpolate_to_cells(pic_particles parts, pic_mesh mesh, int prop, pic_average kind, double *avg,
                                    uint32_t *count, double empty_fill, void *stream);

/* Particle -> field transfer (Sec. 2.7, scheme (iv)): shape-function-weighted
 * averages at the mesh vertices,
 *   avg[v] = sum_i phi_v(x_i) p_i / sum_i phi_v(x_i)
 * over the particles i of the cells around vertex v, phi_v the (bi/tri)linear
 * nodal basis function of v (in a particle's cell: the map weight of v's
 * corner at the stored x-hat).  Each cell's particles are summed in store
 * order, then the cells' sums in increasing cell index (deterministic).  The
 * value at a quadrature point is the Q1 interpolation of avg.  The first
 * call allocates 2^(dim+4) bytes per cell of scratch, kept with the store.
 *   avg     [nverts] FP64 device, vertex (i,j,k) at i + (n0+1)(j + (n1+1)k)
 *   weight  [nverts] FP64 device, the sum of the weights, or NULL
 * A vertex whose weights sum to 0 gets empty_fill.
 * Errors: PIC_ERR_ARG, PIC_ERR_OOM, PIC_ERR_CUDA. */
pic_status pic_interpolate_to_vertices(pic_particles parts, pic_mesh mesh, int prop, double *avg, double *weight,
                                       double empty_fill, void *stream);

/* Particle -> field transfer (Sec. 2.7, scheme (v)): per cell, the linear
 * least-squares fit in reference coordinates,
 *   f(x-hat) = c_0 + sum_j c_{j+1} (x-hat_j - 1/2)
 * minimising sum over the cell's particles of (f(x-hat_i) - p_i)^2.  Solved
 * from the normal equations (folded in store order) by Gaussian elimination
 * with partial pivoting.  A cell with at most dim particles, or a pivot
 * <= 1e-12 times the largest diagonal entry, gets the mean (c_0 = mean,
 * slopes 0); an empty cell gets c_0 = empty_fill.
 *   coef   [dim+1][n_cells] FP64 device;  count  [n_cells] u32 device or NULL
 * Errors: PIC_ERR_ARG, PIC_ERR_CUDA. */
pic_status pic_project_linear(pic_particles parts, pic_mesh mesh, int prop, double *coef, uint32_t *count,
                              double empty_fill, void *stream);

/* Synchronises the particle stream and reads the state: alive particles,
 * particles lost since seeding, and the device status word (bits above).
 * Any output pointer may be NULL. */
pic_status pic_get_state(pic_particles parts, size_t *n_alive, size_t *n_lost, uint32_t *status_word);

/* Per-call counters since seeding: particle-steps advanced, points that
 * needed the neighbour walk, points that needed the all-cells search, Newton
 * iterations.  Synchronises. */
pic_status pic_get_stats(pic_particles parts, uint64_t *particle_steps, uint64_t *walks, uint64_t *global_searches,
                         uint64_t *newton_iterations);

/* All device counters since seeding, in this order (up to n_values of them):
 * particle-steps, neighbour walks, all-cells searches, Newton iterations,
 * particles lost, particle-steps where some cell needed the FP64 Newton
 * fallback, particle-steps whose walk went past the predicted neighbour,
 * particle-steps that pic_advect redid on its full path because the fast
 * path needed a rare one (FP64 Newton, lowest-index test across a nearby
 * facet, neighbour walk, all-cells search).  Synchronises. */
#define PIC_N_COUNTERS 8
pic_status pic_get_counters(pic_particles parts, uint64_t *values, int n_values);

/* Copy the store out in (cell, id) order.  Synchronises `stream` first to
 * read the particle count.  Any pointer may be NULL; host or device memory.
 *   x, xhat [dim][N] FP64;  id [N] u64;  cell [N] u32;  props [n_props][N] FP64 */
pic_status pic_export(pic_particles parts, double *x, double *xhat, uint64_t *id, uint32_t *cell, double *props,
                      void *stream);

/* Particles leaving a process's part of the mesh (Sec. 2.4, parallel
 * transport: a particle that left a process's cells is sent to the owner of
 * its new cell together with that cell, so that the receiver does not search
 * for it).  With the mesh split into slabs of whole cell layers, the sorted
 * store holds the particles that moved below its own layers at its start and
 * those that moved above at its end, each a contiguous range.
 *
 * pic_export_range copies `count` particles of the sorted store from slot
 * `first` on:  x, xhat [dim][count] FP64 (xhat device memory; the store's
 * double-float pair converted exactly);  id [count] u64;  cell [count] u32,
 * each the store's cell + cell_shift (for example into a global numbering;
 * a nonzero shift needs device memory);  props [n_props][count] FP64.  Any
 * pointer may be NULL; x, id, props device or host.  Synchronises `stream`
 * (reads the particle count).
 * Errors: PIC_ERR_ARG (range past the store, host xhat), PIC_ERR_CUDA. */
pic_status pic_export_range(pic_particles parts, size_t first, size_t count, long long cell_shift, double *x,
                            double *xhat, uint64_t *id, uint32_t *cell, double *props, void *stream);

/* Keep the store's particles whose cell lies in [keep_lo, keep_hi), add n_in
 * particles with known cells (cell_in[i] + cell_shift in this store's mesh;
 * out of range: dropped, PIC_STATUS_BOUNDS), then sort the store by
 * (cell, id).  Inputs in device memory, laid out as pic_export_range writes
 * them (props_in may be NULL: zeros).  Dropped particles are not counted as
 * lost (they were handed to another store).  Synchronises `stream`.
 * Errors: PIC_ERR_ARG, PIC_ERR_CAPACITY (kept + received > capacity),
 * PIC_ERR_CUDA. */
pic_status pic_merge_particles(pic_particles parts, uint32_t keep_lo, uint32_t keep_hi, size_t n_in, const double *x_in,
                               const double *xhat_in, const uint64_t *id_in, const uint32_t *cell_in,
                               long long cell_shift, const double *props_in, void *stream);

/* Cell offsets of the sorted store: off[K]..off[K+1] are the particles of
 * cell K.  off is [n_cells + 1] u32, device or host. */
pic_status pic_cell_offsets(pic_particles parts, uint32_t *off, void *stream);

/* Where pic_advect's kernel reads the cells' map and coefficient blocks
 * (Sec. 2.3: every particle evaluates the field of its cell).  on != 0: each
 * warp stages the blocks of the cells its 32 particles start in into shared
 * memory with bulk copies (at most three cells, double-buffered; other cells
 * from the mesh arrays); 0 (the default): all through the read-only cache.
 * Applies to 3D meshes with a single field; the results are bit-identical
 * either way.  Synchronous, enqueues nothing.  Errors: PIC_ERR_ARG. */
pic_status pic_set_advect_staging(pic_particles parts, int on);

/* Instrumentation (no counterpart in the paper).
 * pic_timing_enable: while on, pic_advect records CUDA events on its stream
 * around the advect kernel and around the rebin of every step.
 * pic_timing_read synchronises, returns the summed milliseconds and the
 * number of timed steps since the last read, and resets the sums. */
pic_status pic_timing_enable(pic_particles parts, int on);
pic_status pic_timing_read(pic_particles parts, double *advect_ms, double *rebin_ms, uint64_t *steps);

/* Number of kernels this library has launched in this process. */
uint64_t pic_kernel_launches(void);

/* Message describing the last failure on the calling thread ("" if none). */
const char *pic_last_error(void);

/* Library version string. */
const char *pic_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PIC_H */
