/* libdtt -- constrained DTT/FFT-based elasticity solver on one B300 GPU (sm_103a).
 *
 * The method is the displacement-based accelerated fixed point of Gelebart &
 * Amouzou-Adoun, "Constrained minimization problems and FFT-based solvers: application
 * to local Dirichlet boundary conditions and contact mechanics": per iteration, the
 * stress and its discrete divergence (Eq. 3), the projections proj_P / proj_U of local
 * kinematic constraints (Eq. 9, 11, 14, 17) or of frictionless sphere contact (Eq. 28),
 * depth-4 Anderson acceleration (Section 4.1.1), and the Green-operator step
 * DT -> Green -> iDT with per-face, per-component discrete trigonometric transforms
 * (Section 3.2, Tables 1-3, Eq. 7) -- Algorithm 1 and Algorithm 2.
 *
 * Conventions (every entry point):
 *   - Grid: nvox = {nx, ny, nz} voxels of size h.  Nodes at h*(i, j, k); nn_d = n_d + 1
 *     nodes along a non-periodic axis, n_d along a periodic one.  Flat node index
 *     n = i + nn_x * (j + nn_y * k) (x fastest).  Voxel index v = i + nx * (j + ny * k).
 *   - Nodal vector fields are component-major: f[c * n_nodes + n], c = 0, 1, 2.
 *   - Boundary conditions bc[18] = bc[axis][face][component] (axis 0..2 = x, y, z;
 *     face 0 at x_axis = 0, face 1 at x_axis = n_axis), codes DTT_BC_*.  Periodic must be
 *     set on both faces of an axis for all three components (Section 3.2.1).
 *   - u* = eps* . x is an affine lift; the unknown is the fluctuation u~, u = u* + u~.
 *   - Every call returns a dtt_status; on error, dtt_last_error() returns a message
 *     (thread-local).  No C++ exception crosses this interface.
 *   - Host pointers are read or written synchronously; the library copies what it keeps
 *     (the caller keeps ownership of its arrays).  Where a flag ptr_is_device is given,
 *     1 means the pointer is a CUDA device pointer on the grid's device.
 *   - Work is issued on the stream given at creation; with NULL the grid creates its own
 *     stream (the iteration is captured into a CUDA graph, which the legacy default
 *     stream does not allow).  Calls that return host data synchronise that stream.
 */
#ifndef DTT_H
#define DTT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dtt_grid dtt_grid;

typedef enum {
  DTT_OK = 0,
  DTT_ERR_ARG = 1,            /* invalid argument (size, pointer, index, value) */
  DTT_ERR_BC = 2,             /* inconsistent boundary conditions */
  DTT_ERR_OVERLAP = 3,        /* constraint rows with overlapping supports */
  DTT_ERR_CUDA = 4,           /* a CUDA call failed (message has the CUDA error) */
  DTT_ERR_OOM = 5,            /* device allocation failed */
  DTT_ERR_NOT_CONVERGED = 6,  /* iteration cap reached; the last iterate stays readable */
  DTT_ERR_DIVERGED = 7,       /* residual non-finite or grown by 1e6 */
  DTT_ERR_STATE = 8,          /* call out of order (e.g. solve before set_material) */
  DTT_ERR_NULLMODE = 9        /* constraint on a component whose Green symbol has null modes */
} dtt_status;

enum { DTT_BC_PERIODIC = 0, DTT_BC_DIRICHLET = 1, DTT_BC_NEUMANN = 2 };
enum { DTT_SCHEME_TETRA2 = 0, DTT_SCHEME_HEX1 = 1 };
enum { DTT_PREC_FP64 = 0, DTT_PREC_MIXED = 1 };
enum { DTT_INIT_ZERO = 0, DTT_INIT_PREVIOUS = 1, DTT_INIT_GUESS = 2 };
enum { DTT_ACV_U = 0, DTT_ACV_P = 1 };
enum { DTT_SMALL_STRAIN = 0, DTT_FINITE_STRAIN = 1 };
enum { DTT_MEDIUM_PAUX = 0, DTT_MEDIUM_ISOTROPIC = 1 };

/* Create a grid (Section 3.2.1 problem statement: cell, per-face per-component BCs, FD
 * scheme of Section 3.1.1).  precision: DTT_PREC_FP64 = every nodal field and every
 * transform in float64; DTT_PREC_MIXED = transforms, Green multiply, stress and the
 * Anderson ring in float32, u~ kept as a float-float pair, and float64 for norms, Gram
 * matrix, multipliers, reactions and the contact gap test.  stream: a cudaStream_t (or
 * NULL).  Allocates all device buffers of the grid (about 13 nodal vector fields).
 * Errors: DTT_ERR_ARG (sizes < 2, h <= 0, bad codes), DTT_ERR_BC, DTT_ERR_OOM, DTT_ERR_CUDA. */
dtt_status dtt_grid_create(dtt_grid** out, const int32_t nvox[3], double h, const int32_t bc[18],
                           int32_t scheme, int32_t precision, void* stream);
void dtt_grid_destroy(dtt_grid* grid);

/* Number of nodes and voxels of the grid (for sizing caller buffers). */
dtt_status dtt_grid_sizes(const dtt_grid* grid, int64_t* n_nodes, int64_t* n_voxels, int32_t nn[3]);

/* Material (Eq. 1: sigma = C : eps, isotropic per phase, Section 5.4 convention
 * sigma = lambda tr(eps) 1 + 2 mu eps).  phase: n_voxels uint8 ids (< nphase <= 256).
 * lambda, mu: host arrays of nphase values (>= 0).  Errors: DTT_ERR_ARG.  New values for
 * the same nphase are taken in place and keep the captured iteration graph; another
 * nphase invalidates it. */
dtt_status dtt_set_material(dtt_grid* grid, const uint8_t* phase, int32_t nphase,
                            const double* lambda, const double* mu, int32_t phase_is_device);

/* Reference medium of the Green operator, Paux form (Section 3.2.3):
 * R0 : grad u = lambda0 (grad u (.) I) + 2 mu0 grad u.  Requires mu0 > 0, lambda0 >= 0. */
dtt_status dtt_set_reference(dtt_grid* grid, double lambda0, double mu0);

/* Kind of reference medium (Section 3.2.3).  DTT_MEDIUM_PAUX (default): the Paux medium
 * above, which decouples the components and works with every boundary condition.
 * DTT_MEDIUM_ISOTROPIC: R0 : grad u = lambda0 tr(grad u) 1 + mu0 (grad u + grad u^T), whose
 * Green operator (Eq. 4 for HEX1, with the scheme's own symbols for TETRA2) couples the
 * components through a 3 x 3 solve per wave vector; usable only with normal mixed
 * conditions on every face -- the normal component Dirichlet and the tangential ones
 * Neumann, or the reverse -- and no periodic axis (else DTT_ERR_BC).  The Green step then
 * runs unfused (forward DTTs of the three components, the solve, inverse DTTs).  Other
 * values: DTT_ERR_ARG.  A change invalidates the captured iteration graph. */
dtt_status dtt_set_reference_medium(dtt_grid* grid, int32_t medium);

/* Prescribed strain eps* (3x3 row-major, symmetric part used), Eq. 1.  In finite strain
 * it is the prescribed displacement gradient: F = 1 + eps* + grad u~. */
dtt_status dtt_set_load(dtt_grid* grid, const double eps_star[9]);

/* Kinematics of the stress step (Section 5.2, Eq. 29, Algorithm 3).  DTT_SMALL_STRAIN
 * (default): sigma = C : (eps* + sym grad u~).  DTT_FINITE_STRAIN: the divergence acts on
 * the first Piola-Kirchhoff stress Pi = F.S of a St Venant-Kirchhoff material (the
 * paper's example law: S = C : E, E = (F^T F - 1)/2, F = 1 + eps* + grad u~); Pi also
 * replaces sigma in the Eq. 5 norm and in the contact reaction.  The Green operator, the
 * projections and the contact logic are unchanged.  Other values: DTT_ERR_ARG.  A change
 * invalidates the captured iteration graph. */
dtt_status dtt_set_kinematics(dtt_grid* grid, int32_t kinematics);

/* Local kinematic constraints as rows of the matrices A and B (Section 4.3, Eq. 20-23).
 * Row r has entries e in [row_ptr[r], row_ptr[r+1]): DOF (node[e], comp[e]) with
 * kinematic weight a[e] and reaction weight b[e] (b == NULL: b = a), and prescribes
 *     sum_e a[e] * u_{comp[e]}(node[e]) = value[r]       (u = total displacement).
 * Strong conditions (Eq. 21): one entry, a = b = 1.  Weak conditions (Eq. 10, 22): 8 (or
 * 4 on a face) entries a = b = 1/8 (1/4).  Smooth conditions (Eq. 15-17): a = 1 on the
 * node, b = neighbour weights.  Ties (Section 4.2.3): a = b = 1/|V*|.
 * Supports must be pairwise disjoint (DTT_ERR_OVERLAP), must not contain DOFs eliminated
 * by a Dirichlet face (DTT_ERR_ARG), and must not use a component whose Green symbol has
 * null modes, i.e. whose transforms keep q = 0 (or the TETRA2 checkerboard / a HEX1
 * hourglass) on every axis -- such a component needs a Dirichlet face, e.g. behind a void
 * buffer layer as in Section 4.1.2 (DTT_ERR_NULLMODE).  n_rows = 0 clears the rows.
 * Rows with the same count and total number of entries as the current ones reuse their
 * device buffers and keep the captured iteration graph; other rows invalidate it. */
dtt_status dtt_set_constraints(dtt_grid* grid, int32_t n_rows, const int32_t* row_ptr,
                               const int32_t* node, const int8_t* comp, const double* a,
                               const double* b, const double* value);

/* Rigid frictionless sphere (Section 5, Eq. 24): potential contact surface = all nodes of
 * face `face` (0/1) of axis `axis`; centre and radius in length units.  Components of the
 * face nodes must not have Green null modes (DTT_ERR_NULLMODE). */
dtt_status dtt_set_indenter(dtt_grid* grid, int32_t axis, int32_t face, const double center[3],
                            double radius);
/* Move the sphere centre for the next load increment (Algorithm 2). */
dtt_status dtt_move_indenter(dtt_grid* grid, const double center[3]);
dtt_status dtt_clear_indenter(dtt_grid* grid);

/* Initial fluctuation u~ (3 x n_nodes float64).  Values on Dirichlet-face DOFs are
 * ignored.  A component's null-mode content (if it has null modes) is kept unchanged by
 * the solver. */
dtt_status dtt_set_initial(dtt_grid* grid, const double* u, int32_t ptr_is_device);

/* Initial contact zone of the next increment (Algorithm 2 starts from C = {g < 0} at the
 * starting field, Section 5.1.3; this replaces that rule for one solve): active[q] != 0
 * puts surface node q (the order of dtt_get_contact) in C.  Host or device array of
 * n_surface bytes.  The zone update rule of Algorithm 2 then corrects it as usual.
 * DTT_ERR_STATE without an indenter. */
dtt_status dtt_set_initial_contact(dtt_grid* grid, const uint8_t* active, int32_t ptr_is_device);

typedef struct {
  double tol;          /* Eq. 5 tolerance (RMS norms): h ||p|| / ||sigma|| < tol */
  int32_t max_iter;    /* cap on Green steps (the paper declares failure at 2000) */
  int32_t acv_mod;     /* accelerate every acv_mod iterations after the first four (2 or 3);
                          0 disables acceleration */
  int32_t acv_on;      /* DTT_ACV_P (accelerate p~, default) or DTT_ACV_U (FP64 only) */
  int32_t init;        /* DTT_INIT_ZERO, DTT_INIT_PREVIOUS (current u~: previous step or
                          dtt_set_initial) or DTT_INIT_GUESS: the current u~ is a guess (e.g.
                          dtt_net_predict); the solve evaluates the Eq. 5 residual at it and at
                          u~ = 0 (both after the initial projections) and starts from the
                          lower one, so a guess never starts worse than the plain start */
  double update_tol;   /* contact-zone update threshold on the residual (paper: 1e-2) */
  int32_t graph_iters; /* iterations per captured CUDA-graph launch (0: default 8) */
  double acv_pivot;    /* Anderson is skipped when a pivot of the 4x4 Gram elimination is
                          <= acv_pivot * max_k G_kk (0: default, 1e-14) */
} dtt_solve_opts;

typedef struct {
  int32_t iterations;          /* Green steps performed */
  int32_t accelerations;       /* Anderson combinations applied */
  int32_t active_set_updates;  /* contact-zone changes (Algorithm 2) */
  int32_t status;              /* dtt_status of the solve */
  double residual;             /* Eq. 5 residual of the returned iterate */
  double seconds;              /* wall time of the solve (host clock, synchronised) */
  int32_t start_from_guess;    /* DTT_INIT_GUESS: 1 if the guess was kept, 0 if u~ = 0 won */
  double start_residual;       /* Eq. 5 residual of the starting iterate (DTT_INIT_GUESS) */
} dtt_report;

/* One solve (Algorithm 1), or one load increment (Algorithm 2) when an indenter is set:
 * the active set starts as the surface nodes with negative gap for the current sphere
 * position.  Returns DTT_OK on convergence, DTT_ERR_NOT_CONVERGED / DTT_ERR_DIVERGED
 * otherwise (report filled in every case). */
dtt_status dtt_solve_step(dtt_grid* grid, const dtt_solve_opts* opts, dtt_report* report);

/* Residual history of the last solve (Eq. 5 per iteration); *n in: capacity, out: count. */
dtt_status dtt_get_history(const dtt_grid* grid, double* hist, int32_t* n);

/* u~ (3 x n_nodes, float64) and optionally the stress at the integration points
 * (sigma: n_voxels x n_ip x 6, order xx yy zz yz xz xy; n_ip = 2 TETRA2, 1 HEX1): the
 * Cauchy stress in small strain, the second Piola-Kirchhoff stress S in finite strain. */
dtt_status dtt_get_fields(dtt_grid* grid, double* u, double* sigma, int32_t ptr_is_device);

/* The stress that the divergence acts on, at the integration points, all nine values
 * (tensor: n_voxels x n_ip x 9, row c, column d, float64, caller-owned, host or device):
 * sigma in small strain, the first Piola-Kirchhoff Pi = F.S in finite strain (Section 5.2;
 * Section 5.4 takes the reaction force from its volume average).  DTT_ERR_STATE without
 * a material. */
dtt_status dtt_get_stress_tensor(dtt_grid* grid, double* tensor, int32_t ptr_is_device);

/* Smallest det F over the integration points, F = 1 + eps* + grad u~ of the current u~
 * (Section 5.2's deformation gradient; meaningful in either kinematics).  A value <= 0
 * means an inverted point: a St Venant-Kirchhoff solve (Section 5.4's law) can converge to
 * such a branch when a load increment is too large, and it is then not a physical
 * solution.  *det_min: host double. */
dtt_status dtt_get_min_jacobian(dtt_grid* grid, double* det_min);

/* Reactions of the constraint rows after the last solve: per_row[r] = h^3 f_r
 * sum_e W_e b_e (face DOFs halved, edge DOFs quartered, Section 4.1.3), f_r the
 * multiplier; total = vector sum.  per_row may be NULL. */
dtt_status dtt_get_reactions(dtt_grid* grid, double* per_row, double total[3]);

/* Contact state after the last solve: active[q], gap[q], normal reaction fn[q] for the
 * n_face surface nodes (order: flat node index), and the total contact force vector.
 * Any pointer may be NULL; *n_face returns the count. */
dtt_status dtt_get_contact(dtt_grid* grid, int32_t* n_face, uint8_t* active, double* gap,
                           double* fn, double force[3]);

/* ---- single-pass operators (one step of the hot path on caller data) ---- */

/* Eq. 3, Algorithm 1 stress/divergence step: for u~ (3 x n_nodes float64) returns
 * p = div_D sigma and p~ = p - div_D(R0 : grad_D u~) (both 3 x n_nodes, float64, either
 * may be NULL) and norms[0] = sum w sigma:sigma, norms[1] = sum p^2 over all DOFs.  No
 * constraint projection is applied.  Computed in the grid's precision. */
dtt_status dtt_apply_residual(dtt_grid* grid, const double* u, double* p, double* ptilde,
                              double norms[2], int32_t ptr_is_device);

/* Green step (Algorithm 1, DT -> G -> iDT): u = G_D(ptilde), null modes set to zero. */
dtt_status dtt_apply_green(dtt_grid* grid, const double* ptilde, double* u, int32_t ptr_is_device);

/* Allocation-free variant of dtt_apply_green (the paper has no counterpart: this is an
 * interface for callers that cannot allocate device memory while they run -- services
 * with a fixed device-memory budget, latency-critical loops that cannot afford the
 * synchronisation an allocation implies, hosts whose allocator belongs to another
 * framework).  ptilde_dev and u_dev are caller-owned float64 device arrays (3 x n_nodes,
 * component-major) on the grid's device; they may be the same array.  The grid's device
 * (the one current at dtt_grid_create) must be the current device, else DTT_ERR_ARG.
 * The intermediate spectra use a fixed 64 MiB device array inside the library, held by
 * every GPU that loads it until the process exits, so grids above 2,796,202 nodes are
 * rejected with DTT_ERR_ARG.  The call allocates nothing.  It synchronises the grid's
 * stream before it returns, so it cannot itself be recorded into a CUDA graph.  The first
 * call on a device looks up that array's device address, which a capture in global mode
 * on another stream would not allow: make that first call before such a capture.  All
 * calls share the array: calls that overlap on the GPU race. */
dtt_status dtt_apply_green_noalloc(dtt_grid* grid, const double* ptilde_dev, double* u_dev);

/* Forward (inverse = 0) or inverse (inverse = 1) transform of one nodal component array
 * (n_nodes float64) with that component's per-axis DTT types; the spectrum is stored on
 * the node grid, spectral index k of an axis at position k (unused positions zero). */
dtt_status dtt_transform(dtt_grid* grid, int32_t component, int32_t inverse, const double* in,
                         double* out, int32_t ptr_is_device);

/* Kernel-group timing of the iteration (tracing aid): runs `iters` iterations of the
 * current problem launch by launch (no graph), with CUDA events on the grid's stream
 * around each group, from the state left by the last solve, and returns the mean
 * milliseconds per iteration of each group in ms[DTT_NPROF]:
 *   0 stress/divergence/reference (a1), 1 projections + contact + control, 2 Anderson,
 *   3 forward transforms (3 axis passes), 4 Green multiply, 5 inverse transforms,
 *   6 increment update of u~.
 * Solver state (u~, rings) is modified; call it after the timed solves. */
#define DTT_NPROF 7
dtt_status dtt_profile_iteration(dtt_grid* grid, const dtt_solve_opts* opts, int32_t iters, double* ms);

/* ---- Batched solves and kernel tuning (no counterpart in the paper: its cells are
 * solved one at a time; these serve many independent cells of uneven sizes on one GPU). */

/* Kernel tile choices of one grid:
 *   residual_zchunk: node planes per CTA of the stress/divergence kernel (0: built-in
 *                    choice; otherwise 2..64);
 *   fft_generic:     1 keeps every transform length on the generic Stockham kernels,
 *                    0 lets power-of-two lengths take the register-radix kernels;
 *   z_route:         the fused z pass (forward DTT along z, Green multiply, inverse DTT):
 *                    0 = FFT (or dense) pass, 1 = two split-TF32 tensor-core contractions
 *                    against the z DTT matrices (mixed precision, z operand <= 256
 *                    nodes; elsewhere ignored);
 *   fft_warp:        1 (default) runs the mixed-precision Green step as five warp-register
 *                    sweeps that each read contiguous rows and write the next sweep's rows
 *                    transposed, where every axis is non-periodic with 2n = 32 R,
 *                    R in {2, 3, 4, 6, 8, 12, 16, 24, 32} (fft_generic = 0, z_route = 0 only);
 *                    0 keeps the shared-memory Stockham passes;
 *   ms_per_iteration: (dtt_autotune output) measured time of one iteration with them. */
typedef struct {
  int32_t residual_zchunk;
  int32_t fft_generic;
  int32_t z_route;
  int32_t fft_warp;
  double ms_per_iteration;
} dtt_tuning;

/* Times `iters` iterations of the current problem (launch by launch, CUDA events on the
 * grid's stream) for each candidate tiling -- the FFT routes (warp-register sweeps,
 * register-radix or generic Stockham) and the z route first, then the residual
 * kernel's z chunk in {built-in, 2, 4, 8, 16, 32, 64} -- keeps the fastest on the grid
 * and returns it in *best (may be NULL).  u~ and the solver rings are reset to zero
 * afterwards; call it before a solve.  iters < 1 is DTT_ERR_ARG. */
dtt_status dtt_autotune(dtt_grid* grid, const dtt_solve_opts* opts, int32_t iters, dtt_tuning* best);

/* Applies a tiling (e.g. one tuned on another grid of the same size); a zchunk outside
 * {0, 2..64}, fft_generic, z_route or fft_warp outside {0, 1}, or z_route 1 on a grid that cannot
 * take it (FP64, or more than 256 nodes along z) is DTT_ERR_ARG. */
dtt_status dtt_set_tuning(dtt_grid* grid, const dtt_tuning* tuning);

/* Solves ncell independent grids at once: every cell is prepared as dtt_solve_step
 * would (same opts for all), then the iterations of all cells are captured as parallel
 * branches of one CUDA graph (each cell on its own stream) that one launch advances by
 * opts->graph_iters iterations of every cell; cells that have finished return at once.
 * The host polls one status word per cell between launches.  reports[ncell] receives
 * each cell's report (as dtt_solve_step).  Returns DTT_OK when every cell converged,
 * else the first failing cell's status.  Cells must be distinct grids on the current
 * device; the captured graph is cached and reused while the same grids, unchanged, are
 * solved again with the same opts.  Not thread-safe (one batch at a time per process). */
dtt_status dtt_batch_solve(int32_t ncell, dtt_grid* const* cells, const dtt_solve_opts* opts,
                           dtt_report* reports);

const char* dtt_last_error(void);

/* Library version string. */
const char* dtt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DTT_H */
