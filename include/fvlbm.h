/*
 * fvlbm.h -- C ABI of the GB300 (sm_103a) implementation of the time step of the simplified
 * finite-volume lattice Boltzmann method on unstructured 2-D grids with k-omega SST eddy
 * viscosity and a three-stage second-order IMEX Runge-Kutta integrator
 * (Wang, Zhong, Cao, Zhuo, arXiv 1812.00394, Part II).
 *
 * Method (the passages each entry point implements):
 *   - D2Q9 discrete-velocity BGK equation, Eq. (bgkeq), semi-discretised in finite volumes as
 *     df/dt = Gamma^a + Gamma^c, Eq. (semibgk).
 *   - Convection Gamma^a_alpha = -(1/A) sum_m [(e_alpha . n) f_{alpha,bc} Delta l]_m,
 *     Eq. (advection), with a least-squares cell gradient and upwind linear face values (Sec. 3.2,
 *     Step 2).
 *   - Collision Gamma^c_alpha = -(f_alpha - f^eq_alpha)/tau, Eq. (collision), with
 *     tau = (nu + nu_t)/c_s^2, Eq. (turbtau).
 *   - IMEX stages, Eqs. (imexone), (imextwo) and the tableau of Sec. 3.1; the implicit collision
 *     is solved in closed form per cell through the collision invariants,
 *     Eqs. (sumimeximplicitnew) and (fnewstage).
 *   - k-omega SST (Sec. 2) in finite volumes, Eq. (SSTequint), solved once per step before the
 *     stages (Sec. 3.2, Step 1 and the coupling paragraph).
 *
 * Conventions for every entry point:
 *   - All pointers passed in are HOST pointers unless stated otherwise.  The library copies
 *     whatever it needs during the call; the caller keeps ownership of its arrays.
 *   - Cell arrays are in the caller's (mesh input) cell order.  Distribution arrays are
 *     cell-major: f[cell * 9 + alpha], alpha ordered rest, +x, +y, -x, -y, (+1,+1), (-1,+1),
 *     (-1,-1), (+1,-1).
 *   - Return 0 on success or a negative FVLBM_ERR_* code.  No entry point aborts the process.
 *   - A handle is used by one host thread at a time.  All device work is issued on the
 *     handle's stream.
 */
#ifndef FVLBM_H
#define FVLBM_H

#ifdef __cplusplus
extern "C" {
#endif

#define FVLBM_OK 0
#define FVLBM_ERR_BAD_MESH (-1)    /* connectivity inconsistent, non-positive area, > 4 nodes */
#define FVLBM_ERR_BAD_BC (-2)      /* boundary edge not on the mesh boundary, open edge left */
#define FVLBM_ERR_BAD_PARAM (-3)   /* nu <= 0, no dt and no cfl, bad precision, bad index */
#define FVLBM_ERR_OOM (-4)         /* device allocation failed */
#define FVLBM_ERR_CUDA (-5)        /* a CUDA runtime call failed */
#define FVLBM_ERR_DIVERGED (-6)    /* NaN or Inf in the state (watchdog) */
#define FVLBM_ERR_NOT_SUPPORTED (-7)
#define FVLBM_ERR_TIMEOUT (-8)     /* a bounded wait inside a kernel gave up; the steps since the
                                      last stats step are not valid (restore a saved state) */

/* boundary-edge types */
#define FVLBM_BC_WALL 0       /* no-slip wall moving at (u_b, v_b) */
#define FVLBM_BC_INLET 1      /* velocity inlet (u_b, v_b), turbulence (k_b, omega_b) */
#define FVLBM_BC_OUTLET 2     /* pressure outlet at rho_b */
#define FVLBM_BC_FARFIELD 3   /* characteristic far field (rho_b, u_b, v_b, k_b, omega_b) */
#define FVLBM_BC_PERIODIC 4   /* glued to its partner by fvlbm_bc.periodic_pairs */

/* storage precision of the distribution functions */
#define FVLBM_FP64 0          /* f and all arithmetic in double */
#define FVLBM_FP32_DEV 1      /* f - w_alpha rho0 stored and computed in float; reductions FP64 */
#define FVLBM_FP64_TANGENT 2  /* FP64 plus the forward-mode tangent: every stored and computed
                                 number is a pair (value, derivative with respect to one scalar
                                 parameter p); see fvlbm_tangent_seed.  Runs the two-pass
                                 kernels at about twice the FP64 cost. */

/* Unstructured 2-D mesh: triangles and quadrilaterals, nodes counter-clockwise. */
typedef struct {
    int n_nodes;
    const double *xy;          /* [2 * n_nodes] x0, y0, x1, y1, ... */
    int n_cells;
    const int *cell_ptr;       /* [n_cells + 1] CSR offsets into cell_nodes */
    const int *cell_nodes;     /* 3 or 4 node ids per cell, counter-clockwise */
} fvlbm_mesh;

/* Boundary conditions, one record per boundary edge.  Every boundary edge of the mesh must be
 * listed exactly once. */
typedef struct {
    int n_bedges;
    const int *bedge_nodes;    /* [2 * n_bedges] the two end nodes (any order) */
    const int *bedge_type;     /* [n_bedges] FVLBM_BC_* */
    const double *bedge_val;   /* [5 * n_bedges] rho_b, u_b, v_b, k_b, omega_b */
    int n_periodic;
    const int *periodic_pairs; /* [2 * n_periodic] boundary-edge indices (a, b) */
    const double *periodic_shift; /* [2 * n_periodic] edge b = edge a + shift */
} fvlbm_bc;

typedef struct {
    double nu;                 /* kinematic viscosity (> 0) */
    double rho0;               /* reference density (deviation offset, force normalisation) */
    double dt;                 /* time step; if <= 0, dt = cfl / (max upwind outflow rate) */
    double cfl;
    int sst;                   /* 1: k-omega SST eddy viscosity; 0: laminar */
    int precision;             /* FVLBM_FP64, FVLBM_FP32_DEV or FVLBM_FP64_TANGENT */
    double uref, lref;         /* reference speed and length (C_D, C_L, Cp, omega floor) */
    double alpha_deg;          /* free-stream angle for C_D / C_L */
    const double *rho_init;    /* [n_cells] or NULL (rho0) */
    const double *u_init;      /* [n_cells] or NULL (0) */
    const double *v_init;      /* [n_cells] or NULL (0) */
    const double *k_init;      /* [n_cells] or NULL (0) */
    const double *omega_init;  /* [n_cells] or NULL (1) */
    int kernel_path;           /* 0: fused stage kernels with shared-memory halo staging
                                  (default); 1: two-pass kernels (gradient array in HBM);
                                  2: fused stage kernels in the face-value form (each cell
                                  publishes its upwind face values once per face; the
                                  autotuner may still pick any fused form).
                                  FVLBM_FP32_DEV handles run the face-value form for 0 and 2
                                  (two-pass where its items do not fit): the 256- and
                                  128-cell forms derive the least-squares weights on chip,
                                  which in FP32 leaves wall cells of high aspect ratio with
                                  few correct digits; the face-value and two-pass kernels
                                  read weights formed in FP64 on the host.
                                  A handle with a periodic pair whose edges are translates only
                                  to the gluing tolerance (not to 1e-12 of the edge length)
                                  runs the two-pass kernels: they give both sides of the glued
                                  face side A's normal and length, as the oracle does. */
    int scheme;                /* 0: three-stage IMEX Runge-Kutta of Sec. 3.1 (default);
                                  1: explicit Euler f^{n+1} = f^n + dt (Gamma^a + Gamma^c), the
                                  original scheme that Sec. 3.1 and Sec. 4.1 compare against
                                  (stable only for dt < 2 tau).  All instances of a batch share
                                  it. */
    int local_dt;              /* 1: local time stepping (not in the paper; for steady runs):
                                  every cell advances with its own dt_i = cfl * its convective
                                  limit 1 / max_alpha sum_m max(e_alpha . n_m, 0) dl_m / A_i,
                                  in the stages, the implicit collision and the SST update.
                                  Not time accurate; the steady state moves with the steps at
                                  the level of the scheme's own dt dependence.  Needs cfl > 0
                                  (dt is ignored); fvlbm_info reports the smallest dt_i.
                                  0: one dt per instance (default). */
    int variant;               /* readings of points the paper leaves open, as a bit mask
                                  (0, the default, is the reading the oracle pins):
                                  1: Venkatakrishnan limiter on the least-squares gradient of f
                                     before the upwind reconstruction (Sec. 3.2 Step 2 states
                                     none); runs the two-pass kernels;
                                  2: non-orthogonal correction of the SST diffusion flux,
                                     grad phi . n = (phi_j - phi_i)/|d| + mean grad phi .
                                     (n - d/|d|), instead of the two-point difference alone;
                                  4: the SST solved again before stages 2 and 3 from k, omega,
                                     nu_t of t^n with the macros of f^(1), f^(2) (Sec. 3.2
                                     Step 5 read as "repeat Steps 1-4" per stage); stage J
                                     relaxes with its own tau^(J); the last solve gives
                                     t^{n+1}.  Runs the two-pass kernels; all instances of a
                                     batch must agree on this bit;
                                  8: Menter's production limiter P_k <= 10 beta* omega k, which
                                     the paper's SST (Sec. 2) does not list. */
} fvlbm_params;

typedef struct {
    long long steps;           /* steps taken since create */
    double residual;           /* max over instances of |u^{n+1}-u^n|_2 / |u^{n+1}|_2 (FP64) */
    double mass;               /* sum over instances of sum_i rho_i A_i (FP64) */
    int diverged;              /* 1 if a NaN / Inf was seen */
} fvlbm_stats;

typedef struct fvlbm_handle fvlbm_handle;

/* Build one solver instance on `device` (the current device when < 0), issuing work on
 * `stream` (a cudaStream_t; NULL creates a private non-blocking stream).  Step 0 of Sec. 3.2:
 * f = f^eq(rho_init, u_init); k, omega initialised; nu_t = k / omega.  Mesh geometry, the
 * least-squares matrices, wall distance and a locality-preserving (Hilbert) renumbering are
 * computed on the host; the handle owns all device memory it allocates.
 * Errors: BAD_MESH, BAD_BC, BAD_PARAM, OOM, CUDA. */
int fvlbm_create(const fvlbm_mesh *mesh, const fvlbm_bc *bc, const fvlbm_params *params,
                 int device, void *stream, fvlbm_handle **out);

/* Build one handle that advances n independent instances (meshes of any size, each with its
 * own parameters, laminar or SST) together: every kernel launch of a step covers all
 * instances.  All instances must share params[*].precision.  Instance indices below run
 * 0..n-1 in the given order. */
int fvlbm_create_batch(int n, const fvlbm_mesh *meshes, const fvlbm_bc *bcs,
                       const fvlbm_params *params, int device, void *stream,
                       fvlbm_handle **out);

/* Validate one (mesh, bc, params) triple on the host alone: no GPU, no CUDA call, nothing
 * allocated on a device.  It runs the host preprocessing of fvlbm_create, then checks the
 * result.
 *
 * What the preprocessing validates:
 *   - the mesh and boundary records;
 *   - periodic pairs: edge b must be edge a moved by the shift, to 1e-4 of its length;
 *   - the geometry and the least-squares stencils;
 *   - the renumbering and the time step.
 *
 * What the checks on its result cover.  fvlbm_create runs the same checks on every instance.
 *   - Every index the kernels gather through is in range: neighbours, back slots, boundary
 *     faces and their owners.
 *   - The face links are mutual.
 *   - The padding cells are inert.
 *   - Every geometry array agrees with the node positions and, across each face, with the
 *     neighbour's: n dl, face midpoints, centroid offsets, 1/|d|.
 *   - The least-squares weights satisfy sum_m W_m d_m^T = I.
 *
 * Arguments:
 *   - dt (may be NULL) receives the instance's time step: the given dt, or the CFL step.
 *   - why (may be NULL) receives a NUL-terminated message, at most why_len bytes: empty on
 *     success.
 *
 * Returns FVLBM_OK, or the code fvlbm_create would return for the same input: BAD_MESH,
 * BAD_BC or BAD_PARAM. */
int fvlbm_check_mesh(const fvlbm_mesh *mesh, const fvlbm_bc *bc, const fvlbm_params *params,
                     double *dt, char *why, int why_len);

/* Advance n_steps time steps (Steps 1-7 of Sec. 3.2 each), asynchronously on the handle's
 * stream.  The steps are replayed from a captured CUDA graph.  When `stats` is non-NULL the
 * call synchronises and fills it (FP64 residual of the last step, mass, NaN watchdog) and
 * returns FVLBM_ERR_DIVERGED if the state is not finite.  It also reads the device flag that
 * the fused stage kernels set when a staging wait gave up: FVLBM_ERR_TIMEOUT then (the flag is
 * cleared, so the next step starts clean; the state of the failed steps is not valid). */
int fvlbm_step(fvlbm_handle *h, int n_steps, fvlbm_stats *stats);

/* Diagnostic for the error path above (not in the paper): the number of polls the first
 * staging wait of the fused stage kernels (both fused forms: kernel_path 0 with 256- and
 * 128-cell blocks, and the face-value form of kernel_path 2) makes before giving up; default
 * 2^26, 0 gives up at once, without polling.  Only that wait changes: before a block returns it
 * still waits, with the full bound, for its own copies in flight, so that no copy lands in
 * shared memory after the block has left.  Drops the captured step graphs.
 * Errors: BAD_PARAM. */
int fvlbm_set_wait_limit(fvlbm_handle *h, long long polls);

/* Diagnostic (not in the paper): the work items of the face-value stages (kernel_path 2).
 * *nitem: items (256-cell blocks, or their halves / quarters); *n_split: 256-cell blocks split
 * because their ring-1 + ring-2 halo did not fit the shared memory; *n_overflow: items whose
 * halo has more than 192 cells (its ids continue in a second table).  All 0 when the handle
 * has no face-value items.  Lets a test check that a mesh exercises those paths.
 * Errors: BAD_PARAM (null pointer). */
int fvlbm_fv_items(fvlbm_handle *h, int *nitem, int *n_split, int *n_overflow);

/* Force on the wall faces of `instance`: F = sum over wall faces of sum_alpha e_alpha
 * (e_alpha . n) f_{alpha,bc} Delta l (momentum flux of the Eq. (advection) face values, FP64).
 * out[4] = {Fx, Fy, C_D, C_L}, coefficients along / normal to alpha_deg, normalised by
 * 0.5 rho0 uref^2 lref.  cp (NULL or [n_bedges]) receives (c_s^2 rho_P - c_s^2 rho0) /
 * (0.5 rho0 uref^2) on wall edges and 0 elsewhere, in boundary-edge input order.
 * Synchronises the stream. */
int fvlbm_forces(fvlbm_handle *h, int instance, double *out, double *cp);

/* Host copies of the state of `instance` in input cell order (absolute f, FP64 on output).
 * instance = FVLBM_ALL_INSTANCES (-1) addresses every instance at once: arrays are the
 * instances' arrays concatenated in instance order (one copy and one kernel per call).
 * Any pointer of get_fields may be NULL.  Synchronise the stream. */
#define FVLBM_ALL_INSTANCES (-1)
int fvlbm_get_f(fvlbm_handle *h, int instance, double *f);
int fvlbm_set_f(fvlbm_handle *h, int instance, const double *f);
int fvlbm_get_fields(fvlbm_handle *h, int instance, double *rho, double *u, double *v,
                     double *k, double *omega, double *nut);

/* ---------------------------------------------------------------------------------------------
 * Partitioned meshes (no counterpart in the paper, whose Sec. 4 only states that its code runs
 * in parallel).  One mesh is split into parts, each part a handle (one GPU per part) over its
 * own cells plus the cells within a fixed number of face rings of them (ghosts), with the
 * faces cut by the split as outlet edges.  After every step each part overwrites its ghosts
 * with the state their owners computed; a step of Sec. 3.2 reaches 8 rings (2 for the SST
 * update, 2 per IMEX stage), so with 8 ghost rings the owned cells step exactly as in the
 * whole mesh.  The time step (fvlbm_params.dt) and the wall distance are those of the whole
 * mesh.  These calls move the per-cell state of a list of cells and set the wall distance.
 *
 * fvlbm_get_cells / fvlbm_set_cells: n cells of `instance`, ids in the instance's input cell
 * order (0 <= cells[j] < n_cells, else BAD_PARAM and nothing changes).  f [n * 9] cell-major
 * like fvlbm_get_f; k, omega, nut [n] (current values).  get: any output may be NULL.  set: f
 * may be NULL (f unchanged), and k, omega, nut are all given or all NULL; setting f also
 * recomputes the cells' macros (as fvlbm_set_f).  Both synchronise.  Errors: BAD_PARAM, OOM,
 * CUDA.
 *
 * fvlbm_set_wall_distance: d [n_cells] (> 0, input cell order) replaces the distance to the
 * nearest wall that create computed from the instance's own wall edges (it enters the SST
 * blending functions and the wall value of omega).  Synchronises.  Errors: BAD_PARAM, CUDA.
 *
 * fvlbm_cell_geometry (host only, no CUDA call): area [n_cells] and the wall distance
 * [n_cells] (1e30 without wall edges) of a (mesh, bc, params) triple as create computes them,
 * in input cell order; either may be NULL.  Errors: those of fvlbm_check_mesh.
 *
 * fvlbm_forces_edges: the wall force of fvlbm_forces per boundary edge, fxy [2 * n_bedges] =
 * (Fx, Fy) in boundary-edge input order, 0 on edges that are not walls; a partitioned mesh
 * sums the edges of the cells it owns.  Synchronises.  Errors: BAD_PARAM, CUDA. */
int fvlbm_get_cells(fvlbm_handle *h, int instance, int n, const int *cells, double *f, double *k,
                    double *omega, double *nut);
int fvlbm_set_cells(fvlbm_handle *h, int instance, int n, const int *cells, const double *f,
                    const double *k, const double *omega, const double *nut);
int fvlbm_set_wall_distance(fvlbm_handle *h, int instance, const double *d);
int fvlbm_cell_geometry(const fvlbm_mesh *mesh, const fvlbm_bc *bc, const fvlbm_params *params,
                        double *area, double *wdist);
int fvlbm_forces_edges(fvlbm_handle *h, int instance, double *fxy);

/* The ghost exchange on DEVICE buffers (for NCCL send / receive between GPUs, no host copy).
 *
 * fvlbm_set_exchange_list: registers n cells of `instance` (host array, input cell order, each
 * in [0, n_cells), else BAD_PARAM and nothing is registered) as one list and returns its id in
 * *list_id.  Lists live as long as the handle.  Synchronises.  Errors: BAD_PARAM, OOM, CUDA.
 *
 * fvlbm_pack_cells_dev: vals (DEVICE pointer, n * 12 doubles, row j for cell j of the list)
 * receives f (9, absolute as fvlbm_get_f), k, omega, nu_t of the list's cells.
 * fvlbm_unpack_cells_dev: the reverse, as fvlbm_set_cells with all four fields (the macros
 * follow f).  Both are enqueued on the handle's stream and do not synchronise: vals must stay
 * valid until that work has run, and a caller that moves vals on another stream orders it
 * against the handle's stream.  Errors: BAD_PARAM (unknown list, NULL vals), CUDA. */
/* FP64 arithmetic peak of `device` (the current device when < 0), measured (no counterpart in
 * the paper): the rate of double-precision fused multiply-adds of a kernel that runs
 * independent FMA chains on every SM and reads no memory, in TFLOP/s (2 flops per FMA), the
 * best of three timed launches.  The roofline of the FP64 path, which the FP64 pipe bounds.
 * Synchronises.  Errors: BAD_PARAM, OOM, CUDA. */
int fvlbm_fp64_peak(int device, double *tflops);

int fvlbm_set_exchange_list(fvlbm_handle *h, int instance, int n, const int *cells, int *list_id);
int fvlbm_pack_cells_dev(fvlbm_handle *h, int list_id, double *vals);
int fvlbm_unpack_cells_dev(fvlbm_handle *h, int list_id, const double *vals);

/* Pipelined variants of fvlbm_set_f and fvlbm_get_fields that do not synchronise, so that host
 * transfers overlap the steps (no counterpart in the paper).  Each call stages its data in one
 * of two device slots per direction (alternating), copies on a transfer stream of the handle
 * (a copy engine, concurrent with kernels when the host buffers are pinned), and orders itself
 * after the work already issued on the handle's stream:
 *   fvlbm_set_f_async: host f -> slot (transfer stream), then the handle's stream waits for
 *     it and scatters it into the state (work issued later sees the new state);
 *   fvlbm_get_fields_async: the fields as of the work issued so far are gathered into a slot
 *     on the handle's stream and copied to the host pointers on the other transfer stream.
 * The host buffers must stay valid and unchanged (set) or unread (get) until fvlbm_wait(h)
 * returns.  Any number of calls may be issued: a call whose slot is still in use waits for it
 * on the device, not on the host (a slot that must grow synchronises once).  fvlbm_wait blocks
 * until the handle's stream and both transfer streams are idle.  Errors: BAD_PARAM, OOM,
 * CUDA. */
int fvlbm_set_f_async(fvlbm_handle *h, int instance, const double *f);
int fvlbm_get_fields_async(fvlbm_handle *h, int instance, double *rho, double *u, double *v,
                           double *k, double *omega, double *nut);
int fvlbm_wait(fvlbm_handle *h);

/* FP32 deviation I/O: the state as f - w_alpha rho0 in float, cell-major [cells][9] in input
 * order (instance -1: all instances concatenated).  For FVLBM_FP32_DEV handles this is their
 * storage format, so values pass unchanged, at half the bytes of the double interface; other
 * precisions convert.  fvlbm_get_fdev_f32 synchronises; fvlbm_set_fdev_f32_async is pipelined
 * like fvlbm_set_f_async (same slots, streams and fvlbm_wait). */
int fvlbm_get_fdev_f32(fvlbm_handle *h, int instance, float *fdev);
int fvlbm_set_fdev_f32_async(fvlbm_handle *h, int instance, const float *fdev);

/* Sizes and the time step actually used (instance -1: totals over all instances, dt = 0). */
int fvlbm_info(fvlbm_handle *h, int instance, int *n_cells, int *n_bedges, double *dt);

/* Bytes of device memory the handle holds, and the number of kernel launches one step issues. */
int fvlbm_footprint(fvlbm_handle *h, long long *device_bytes, int *launches_per_step);

/* Per-kernel device time over n_steps un-captured steps, measured with CUDA events recorded
 * on the handle's stream around each launch (for roofline reporting).  names receives up to
 * max_kernels entries of 32 chars; ms and launches the summed milliseconds and launch counts.
 * Returns the number of kernels reported (>= 0) or an error. */
int fvlbm_profile_kernels(fvlbm_handle *h, int n_steps, int max_kernels, char *names,
                          double *ms, int *launches);

/* Kernel autotuner (not in the paper).  Times trial_steps steps of each kernel configuration the
 * handle supports -- 0: fused stages with 256-cell blocks, 1: fused stages with 128-cell blocks,
 * 2: two-pass kernels, 3: fused stages in the face-value form -- on a snapshot of the current
 * state, restores the state exactly, and keeps the fastest for all later steps.  *chosen (may
 * be NULL) receives the configuration and ms_per_step[4] (may be NULL) the measured
 * milliseconds per step, -1 for configurations not
 * available (a block's halo too large for shared memory, kernel_path 1, the explicit
 * scheme, or configurations 0 and 1 on FVLBM_FP32_DEV handles, see kernel_path).  Allocates a temporary snapshot of the state (about 28 words per cell) and
 * synchronises the stream.  Errors: BAD_PARAM, OOM, CUDA. */
int fvlbm_autotune(fvlbm_handle *h, int trial_steps, int *chosen, double *ms_per_step);

/* ---------------------------------------------------------------------------------------------
 * Forward-mode tangent (no counterpart in the paper's Part II; the shape-design use of the solver
 * that its conclusion points to needs derivatives of C_D and C_L).  Valid on handles created with
 * precision FVLBM_FP64_TANGENT, else FVLBM_ERR_NOT_SUPPORTED.
 *
 * Such a handle advances, with every step, the values of the FP64 step AND their derivatives
 * with respect to one scalar parameter p, by the chain rule through each operation of the
 * discrete step (Steps 1-7 of Sec. 3.2: gradient, upwind face values, boundary values, the
 * closed-form implicit collision, the SST update and tau = (nu + nu_t) / c_s^2).  Where the step
 * is not differentiable (upwind switch on e.n = 0, limiter and clip branches, the nu_t limiter's
 * min), the derivative of the branch the value takes is carried.  The values equal those of an
 * FVLBM_FP64 handle with kernel_path 1 up to rounding (the compiler may fuse multiply-adds
 * differently).
 *
 * fvlbm_tangent_seed sets dp of the inputs p acts on, for `instance` (FVLBM_ALL_INSTANCES is not
 * accepted):
 *   dbedge_val  [5 * n_bedges] in boundary-edge input order: d(rho_b, u_b, v_b, k_b, omega_b)/dp,
 *               e.g. for p = free-stream angle alpha (radians) with u_b = U cos alpha,
 *               v_b = U sin alpha: (0, -v_b, u_b, 0, 0) on far-field edges.  NULL = unchanged.
 *   df          [n_cells * 9] cell-major like fvlbm_set_f: df/dp of the current state.  NULL =
 *               unchanged.  fvlbm_set_f resets the derivative of f it writes to 0.
 * The derivatives of k, omega and nu_t start at 0 at create.
 *
 * fvlbm_get_f_tangent: df/dp of the current state, layout of fvlbm_get_f.
 * fvlbm_forces_tangent: out[4] as fvlbm_forces and dout[4] = d(Fx, Fy, C_D, C_L)/dp.  dalpha is
 *   d(alpha)/dp in radians (1 when p is alpha in radians, 0 when alpha does not depend on p): it
 *   adds the derivative of the projection of (Fx, Fy) onto the drag and lift directions.
 * All three synchronise the stream.  Errors: BAD_PARAM, NOT_SUPPORTED, CUDA. */
int fvlbm_tangent_seed(fvlbm_handle *h, int instance, const double *dbedge_val, const double *df);
int fvlbm_get_f_tangent(fvlbm_handle *h, int instance, double *df);

/* Shape derivatives: dxy [2 * n_nodes] = d(x, y)/dp of every mesh node of `instance` (for example
 * a wall-normal displacement of one wall node).  Recomputes the instance's geometry on the host
 * with these derivatives (areas, normals and face lengths, centroids, least-squares weights,
 * face offsets, wall distance d) and stores d(geometry)/dp beside the values; the values and
 * the cell order do not change (FVLBM_ERR_NOT_SUPPORTED if the perturbed preprocessing would
 * reorder cells).  The time step stays the one fixed at create, so the derivative is the one at
 * fixed dt: for a dt derived from cfl it omits dt's own dependence on the geometry.  dxy = 0
 * clears the shape seed.  Synchronises.  Errors: BAD_PARAM, NOT_SUPPORTED, BAD_MESH, CUDA. */
int fvlbm_tangent_seed_nodes(fvlbm_handle *h, int instance, const double *dxy);
int fvlbm_forces_tangent(fvlbm_handle *h, int instance, double dalpha, double *out, double *dout);

/* ---------------------------------------------------------------------------------------------
 * Discrete adjoint (reverse mode; no counterpart in the paper, which its conclusion's design use
 * of the solver motivates like the tangent above).  One call gives the gradient of one scalar
 * objective with respect to every cell's initial distributions, every boundary value and every
 * node position, where the tangent needs one run per input direction.
 *
 *   J = w[0] C_D + w[1] C_L of `instance` after n_steps steps from the handle's current state,
 *
 * C_D, C_L as fvlbm_forces.  The step differentiated is the handle's step (Sec. 3.1-3.2, Steps
 * 1-7: the k-omega SST solve on SST instances, then the IMEX stages, or the explicit Euler
 * update), with one dt per instance or local time steps, as the two-pass kernels run it in FP64
 * (the fused kernels give the same values up to rounding).
 * Where the step is not differentiable (the upwind switch on e.n = 0, the SST's limiter, clip
 * and blending branches) the derivative of the branch the value takes is used, as in the
 * tangent.
 * Outputs (host, each may be NULL):
 *   J              the objective's value;
 *   dJ_df          [n_cells * 9] dJ/df of the current state, cell-major like fvlbm_get_f;
 *   dJ_dbedge_val  [5 * n_bedges] dJ/d(rho_b, u_b, v_b, k_b, omega_b) in boundary-edge input
 *                  order, the layout of fvlbm_tangent_seed (k_b, omega_b: 0 on laminar
 *                  instances; periodic edges: 0);
 *   dJ_dxy         [2 * n_nodes] dJ/d(x, y) of every mesh node at fixed dt and fixed initial
 *                  state, through the preprocessed geometry (areas, face normals and lengths,
 *                  centroids, face offsets, least-squares weights, the wall normals and lengths
 *                  of the force): the gradient whose inner product with a node displacement is
 *                  what fvlbm_tangent_seed_nodes gives for it; on SST instances also through
 *                  1/|d| and the wall distance d, and with the limiter on grad f through the
 *                  cell areas.  Not for meshes with periodic pairs (FVLBM_ERR_NOT_SUPPORTED).
 * The initial k, omega and nu_t of SST instances are held fixed (their adjoints are not output).
 * Neither the state nor the step count of the handle changes.  The call runs n_steps forward
 * steps that keep their stage values (99 doubles per cell and step, 119 with SST, 153 under the
 * per-stage SST reading) and n_steps adjoint steps.
 * Where the stage values of all steps do not fit the adjoint budget (fvlbm_set_adjoint_budget;
 * default half the free device memory), the run is cut into units of K steps whose stage values
 * fit in half the budget; the other half holds c state snapshots (9 doubles per cell, 15 with
 * SST), and the units are reversed on the binomial (revolve) schedule: with r the least number
 * with C(c + r, c) >= the number of units, no unit runs forward more than r + 1 times (2 when
 * there is a snapshot for every unit start).  The device memory is allocated for the call and
 * freed before it returns (about 60 doubles per cell plus the stage values and snapshots, 32
 * more with dJ_dxy); dJ_dxy adds one pass over the cells on the host (SST: and a nearest-wall
 * search per cell).
 * Valid on FVLBM_FP64 handles, with either scheme (IMEX or the explicit Euler comparison
 * scheme) and every reading variant; else FVLBM_ERR_NOT_SUPPORTED.  Synchronises.
 * Errors: BAD_PARAM (w NULL, n_steps < 0, bad instance), NOT_SUPPORTED, OOM, CUDA. */
int fvlbm_adjoint(fvlbm_handle *h, int instance, int n_steps, const double *w, double *J, double *dJ_df,
                  double *dJ_dbedge_val, double *dJ_dxy);
/* Parameter-level gradient of J = w[0] C_D + w[1] C_L (Sec. 4.3's force coefficients) after
 * n_steps FP64 steps from the handle's current state, with respect to the three parameter
 * kinds of the airfoil study: one fvlbm_adjoint solve, then the chain rule through
 *   alpha  the free-stream angle in radians.  It turns the velocity (u_b, v_b) of every
 *          FVLBM_BC_FARFIELD edge, d(u_b, v_b)/d alpha = (-v_b, u_b), and the drag and lift
 *          axes of fvlbm_forces, dC_D/d alpha = C_L, dC_L/d alpha = -C_D;
 *   ratio  the inflow eddy-viscosity ratio r = nu_t / nu, entering as omega_b = k_b / (nu r)
 *          on every FVLBM_BC_FARFIELD and FVLBM_BC_INLET edge with k_b > 0 (Sec. 3.2's Menter
 *          inflow values; r is read off each edge as k_b / (nu omega_b));
 *   s_j    the displacement of mesh node wall_nodes[j] along the direction
 *          wall_normals[2 j], wall_normals[2 j + 1] (the caller's choice, e.g. the outward unit
 *          normal of the wall there), through the mesh geometry as in fvlbm_adjoint's dJ_dxy.
 * The initial state and dt stay fixed, as in fvlbm_adjoint.
 * Inputs: w [2] (host); n_wall >= 0; wall_nodes [n_wall] node ids of the input mesh;
 * wall_normals [2 n_wall] (host).  Outputs (host, NULL to skip): J; cdcl [2] = C_D, C_L after
 * the n_steps steps; dJ_dalpha; dJ_dratio (0 on laminar instances); dJ_dwall [n_wall] (needed
 * when n_wall > 0).  Same device memory, schedule and synchronisation as fvlbm_adjoint; the
 * handle's state is unchanged.
 * Errors: BAD_PARAM (NULL w, bad instance, n_wall < 0, a NULL wall array with n_wall > 0, a
 * node id out of range); NOT_SUPPORTED (not FVLBM_FP64; n_wall > 0 on a mesh with periodic
 * pairs); OOM; CUDA. */
int fvlbm_adjoint_params(fvlbm_handle *h, int instance, int n_steps, const double *w, int n_wall,
                         const int *wall_nodes, const double *wall_normals, double *J, double *cdcl,
                         double *dJ_dalpha, double *dJ_dratio, double *dJ_dwall);
/* The device memory fvlbm_adjoint may use for stage values, in bytes (0: half the free device
 * memory at the time of the call, the default).  Errors: BAD_PARAM. */
int fvlbm_set_adjoint_budget(fvlbm_handle *h, long long bytes);

/* ---------------------------------------------------------------------------------------------
 * Checkpoint / resume and divergence rollback (no counterpart in the paper).
 *
 * The state of a handle -- f^n, f^(1) of the coming step, the macros, tau, k / omega / nu_t and
 * their ping-pong parity, and the step count -- as one opaque host blob in the handle's internal
 * cell order.  fvlbm_state_bytes gives its size; fvlbm_save_state writes it into buf (bytes at
 * least that size); fvlbm_load_state restores it into this handle or into any handle created
 * from the same meshes and parameters (the preprocessing is deterministic).  The blob's header
 * carries the precision, the sizes and a checksum of the cell order; a blob of another
 * configuration returns FVLBM_ERR_BAD_PARAM and changes nothing.  Both synchronise.
 *
 * fvlbm_set_rollback(h, every): with every > 0, the handle keeps one device copy of its state
 * (fvlbm_state_bytes of device memory), refreshed at the end of an fvlbm_step call with stats
 * that finds the state finite, at most once per `every` steps.  When an fvlbm_step with stats
 * finds a NaN / Inf, it restores that copy before returning FVLBM_ERR_DIVERGED, and
 * stats->steps is the restored step.  every = 0 frees the copy.
 * Errors: BAD_PARAM, OOM, CUDA. */
int fvlbm_state_bytes(fvlbm_handle *h, long long *bytes);
int fvlbm_save_state(fvlbm_handle *h, void *buf, long long bytes);
int fvlbm_load_state(fvlbm_handle *h, const void *buf, long long bytes);
int fvlbm_set_rollback(fvlbm_handle *h, int every);

void fvlbm_destroy(fvlbm_handle *h);
const char *fvlbm_strerror(int code);

/* ---------------------------------------------------------------------------------------------
 * Allocation-free FP64 step statistics (no counterpart in the paper).
 *
 * For callers that cannot call cudaMalloc -- for example code that runs while a framework's
 * caching allocator or a start-up memory pool owns all device memory, or real-time loops that
 * must never block in the allocator.  Computes the same FP64 reduction fvlbm_step reports
 * with stats (its velocity residual and mass), from caller-owned DEVICE arrays, without
 * allocating anything: the per-block partial sums live in a fixed file-scope device array of
 * FVLBM_STATS_STATIC_MAX_CELLS / 256 x 4 doubles (512 KiB), which every GPU that loads the
 * library holds until the process exits.
 *
 * Inputs (device pointers, n doubles each): the velocity before (u_old, v_old) and after
 * (u_new, v_new) a step, the density rho and the cell areas.  Output: `out`, a device pointer
 * to 4 doubles = {sum |u_new - u_old|^2, sum |u_new|^2, sum rho * area, number of non-finite
 * cells}; the residual of fvlbm_stats is sqrt(out[0]) / sqrt(out[1]).  Work is issued on
 * `stream` (a cudaStream_t, NULL = legacy default stream) on the current device and is
 * asynchronous; read `out` after synchronising that stream.
 *
 * The first call on a device looks up the device address of the scratch array
 * (cudaGetSymbolAddress); make that first call before any stream capture.  Later calls look
 * it up again unless `stream` is being captured, so a call after cudaDeviceReset (which
 * unloads the module, and with it the array) finds the array's new address; a call under
 * capture uses the address of the last lookup, so do not capture the first call after a
 * reset.  Every call shares
 * the one scratch array, so calls that overlap on the GPU (several streams or host threads)
 * race; serialise them.  Each call overwrites all the scratch it reads, so no clearing is
 * needed between calls.
 *
 * Errors: FVLBM_ERR_BAD_PARAM for a NULL pointer, n < 0, or n > FVLBM_STATS_STATIC_MAX_CELLS
 * (message on stderr); FVLBM_ERR_CUDA if the symbol lookup or a launch fails. */
#define FVLBM_STATS_STATIC_MAX_CELLS 4194304
int fvlbm_stats_reduce_static(const double *u_old, const double *v_old, const double *u_new,
                              const double *v_new, const double *rho, const double *area, int n,
                              double *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FVLBM_H */
