/*
 * felbm.h -- C ABI of the GB300 FE-LBM contact-line step.
 *
 * One time step of the characteristic-based finite-element lattice Boltzmann
 * method for the free-energy two-phase model with wetting walls
 * (Matin, Misztal, Hernandez-Garcia, Mathiesen, arXiv:1708.04678), written
 * for two D2Q9 distribution sets -- g (pressure/momentum) and h (composition)
 * -- on unstructured linear triangles.  Every step of the update runs in CUDA
 * kernels for sm_103a; the host only preprocesses the mesh once and enqueues.
 *
 * Conventions shared by every call:
 *  - Return value: FELBM_OK (0) or a negative FELBM_ERR_* code; the message of
 *    the last error of the calling thread is felbm_last_error().  No call
 *    throws across the ABI.
 *  - Host arrays are owned by the caller and only read (or written) during
 *    the call.  Node numbering is the caller's: the library reorders nodes
 *    internally (compact tiles of at most 1024 nodes by recursive coordinate
 *    bisection, reverse Cuthill-McKee order inside a tile) and converts back
 *    on every exchange.
 *  - Device memory: the library never allocates it.  The caller allocates one
 *    workspace of felbm_workspace_bytes() bytes (any allocator, 256-byte
 *    aligned) and keeps it alive until felbm_state_destroy().
 *  - Streams: all device work of a state is enqueued on the cudaStream_t given
 *    to felbm_init (passed as void*; NULL = legacy default stream).  Calls
 *    that return host data synchronise that stream; felbm_step does not.
 *  - Environment: FELBM_PDL=0 launches the solve sweeps without programmatic
 *    dependent launch (read at felbm_init; default on).  FELBM_ORDER=rcm
 *    (read at mesh creation) keeps the plain reverse Cuthill-McKee order.
 *  - Distribution layout on the host: double [9][n_nodes], direction-major,
 *    D2Q9 order e_0 = (0,0), e_1..e_4 = (1,0),(0,1),(-1,0),(0,-1),
 *    e_5..e_8 = (1,1),(-1,1),(-1,-1),(1,-1); weights 4/9, 1/9, 1/36.
 */
#ifndef FELBM_H
#define FELBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FELBM_OK 0
#define FELBM_ERR_INVALID_ARG (-1)
#define FELBM_ERR_BAD_MESH (-2)     /* inverted/degenerate triangle, open edge that is no wall, ... */
#define FELBM_ERR_CUDA (-3)         /* a CUDA runtime call failed */
#define FELBM_ERR_WORKSPACE (-4)    /* workspace missing, misaligned or too small */
#define FELBM_ERR_NONFINITE (-5)    /* NaN or Inf found in the state */
#define FELBM_ERR_UNSUPPORTED (-6)  /* option not available in this build */
#define FELBM_ERR_NOT_CONVERGED (-7) /* the checked solve's residual is above its tolerance (felbm_solver_check) */

#define FELBM_MAX_WALL_IDS 256

/* Patch Laplacian of C (eqn:lapl_int_mp): V = 2/3 |patch| (equals the lumped
 * P1 Laplacian) or V = |patch| (the literal patch area). */
#define FELBM_LAP_CONSISTENT 0
#define FELBM_LAP_PAPER 1

/* Storage/arithmetic of the distributions.
 * FP64:     g, h stored and updated in FP64.
 * FP32_DEV: the fields C (FP64), p, u (FP32) plus the FP32 deviations of g, h
 *           from their equilibria; FP32 arithmetic except the chemical
 *           potential (double well and Laplacian of C) and the C update, which
 *           stay FP64; the mass solve runs in FP32 (solver_rounds must be 0/1). */
#define FELBM_FP64 0
#define FELBM_FP32_DEV 1

/* Consistent-mass solve (Sec. II.C: M11 with the lumped-mass preconditioner).
 * MIXED: iterative refinement -- FP32 corrections (Richardson steps at the
 *        reciprocal Chebyshev roots of the spectrum [1/4, 1], which give the
 *        Chebyshev error bound), residual carried in FP64 (default; reaches
 *        FP64 round-off with solver_rounds = 3).
 * FP64:  Chebyshev sweeps in FP64 throughout. */
#define FELBM_SOLVER_MIXED 0
#define FELBM_SOLVER_FP64 1

/* Element Laplacian of mu in the h-force M lap(mu) Gamma (eq:H).
 * FACE:  Sec. II.D -- flux of the face-averaged element gradients of mu,
 *        wall faces zero (eqn:bc1).  The paper's form (default).
 * NODAL: the patch Laplacian of eqn:lapl_int_mp applied to mu with the zero
 *        wall flux of eqn:bc1 (the lumped P1 Laplacian), averaged over the
 *        element's vertices.  Not in the paper: the FACE form fed to the
 *        nodes through M11^-1 M10 has eigenvalues with positive real part on
 *        jittered meshes (an anti-diffusive Cahn-Hilliard mode that makes
 *        long runs diverge at rate ~ M dt max Re); this one has none.
 *        The adjoint (felbm_adjoint_*) supports FACE only. */
#define FELBM_LAPMU_FACE 0
#define FELBM_LAPMU_NODAL 1

/* Model constants (Sec. II of the paper, lattice units).
 *  dt              time step (characteristic step eqn::integrated)
 *  tau_l, tau_v    relaxation times of liquid and vapour; 1/tau = C/tau_l + (1-C)/tau_v
 *  rho_l, rho_v    bulk densities; rho = C rho_l + (1-C) rho_v
 *  kappa, beta     gradient and bulk free-energy constants (eqn:FE_func_b)
 *  mobility        Cahn-Hilliard mobility M (eqn:mp_che)
 *  phi_c[id]       wetting potential of wall id (eqn:bc2); cos(theta) = -phi_c / sqrt(2 kappa beta)
 *  lap_mode        FELBM_LAP_CONSISTENT or FELBM_LAP_PAPER
 *  precision       FELBM_FP64 or FELBM_FP32_DEV
 *  solver_mode     FELBM_SOLVER_MIXED or FELBM_SOLVER_FP64
 *  solver_iters    sweeps per correction (MIXED, 0 = 14, error
 *                  bound 2*3^-14 per correction; FP32_DEV, 0 = 10, bound
 *                  2*3^-10) or in total (FP64, 0 = 32, bound 2*3^-32); >= 2
 *  solver_rounds   corrections of the MIXED solve (0 = 3 for FP64 storage,
 *                  1 for FP32_DEV)
 *  lapmu_mode      FELBM_LAPMU_FACE (default) or FELBM_LAPMU_NODAL          */
typedef struct felbm_params {
    double dt;
    double tau_l, tau_v;
    double rho_l, rho_v;
    double kappa, beta;
    double mobility;
    double phi_c[FELBM_MAX_WALL_IDS];
    int32_t n_wall_ids;
    int32_t lap_mode;
    int32_t precision;
    int32_t solver_mode;
    int32_t solver_iters;
    int32_t solver_rounds;
    int32_t lapmu_mode;
} felbm_params;

typedef struct felbm_mesh felbm_mesh;
typedef struct felbm_state felbm_state;

typedef struct felbm_mesh_info {
    int32_t n_nodes, n_tri, n_wall_edges;
    int32_t n_groups;         /* connected components (independent droplets of a batch) */
    int32_t nnz;              /* entries of the node-node sparsity pattern */
    int32_t max_degree;       /* largest row of that pattern */
    int32_t bandwidth;        /* largest |i - j| of the pattern in the internal order */
    double min_area, total_area;
    int32_t n_tiles;          /* node tiles of the internal order (at most 1024 nodes each) */
    int32_t max_tile_halo;    /* most nodes outside a tile that its rows reference */
} felbm_mesh_info;

/* What felbm_diagnostics measures beside the global sums. */
typedef struct felbm_diag_request {
    double centre[2];         /* droplet centre for the interface band */
    double radius;            /* droplet radius R; band = nodes with |r - R| <= band */
    double band;              /* half width of the band (the paper uses xi) */
    int32_t substrate_wall_id;/* wall id on which contact angle is measured; <0: none */
} felbm_diag_request;

typedef struct felbm_diag {
    int64_t step;
    double mass;              /* sum_i m_i C_i, m_i = lumped mass (= |patch_i|/3) */
    double mass0;             /* the same at felbm_init */
    double mass_drift_rel;    /* (mass - mass0) / mass0 */
    double kinetic_energy;    /* <T> = 1/2 sum_i rho_i |u_i|^2 / N (Fig. 5 caption) */
    double max_u;             /* max_i |u_i| (spurious-current magnitude) */
    double interface_rho_uu;  /* area-weighted mean of rho |u|^2 over the band (Table I) */
    double p_in, p_out;       /* area-weighted mean p over C >= 0.95 / C <= 0.05 */
    double delta_p;           /* p_in - p_out (Laplace jump) */
    double wetted_length;     /* length of substrate wall edges with C >= 1/2 (linear in C) */
    double height;            /* max height of the C = 1/2 contour above the mean substrate height */
    double theta_deg;         /* contact angle from height and base, circular cap (Sec. III.B) */
    int32_t status;           /* FELBM_OK, FELBM_ERR_NONFINITE or FELBM_ERR_NOT_CONVERGED */
    int32_t solver_sweeps;    /* steps of one mass solve (all corrections) */
    double solver_residual;   /* felbm_solver_check on: ||b - M x|| / ||b|| of the last solve before its
                                 last step (all 18 right-hand sides); NaN when off */
} felbm_diag;

/* Text of the calling thread's last error ("" if none). */
const char* felbm_last_error(void);

/* Fill kappa, beta and phi_c[0..n_wall_ids) of *p from the surface tension
 * sigma, the interface width xi and the contact angles (degrees):
 * xi = sqrt(8 kappa/beta), sigma = sqrt(2 kappa beta)/6 (Sec. II, planar
 * profile) and cos(theta) = -phi_c/sqrt(2 kappa beta) (Sec. II.B, Young). */
int felbm_params_derive(double sigma, double xi, const double* theta_deg,
                        int32_t n_wall_ids, felbm_params* p);

/* Build a mesh (host only; Sec. II.C, linear elements).
 *  xy          double [n_nodes][2] node coordinates
 *  tri         int32 [n_tri][3] node ids, counter-clockwise after minimum image
 *  wall_edges  int32 [n_wall_edges][2] node pairs lying on solid walls
 *  wall_id     int32 [n_wall_edges] index into felbm_params.phi_c
 *  period_x/y  periodic lengths (0 = not periodic); periodic images are one node
 * Every edge used by one triangle only must be a wall edge.  Errors:
 * FELBM_ERR_INVALID_ARG (bad sizes/ids), FELBM_ERR_BAD_MESH (non-positive
 * area, open edge that is not a wall, wall edge that is not a boundary edge,
 * edge shared by more than two triangles).  *out is freed by felbm_mesh_destroy. */
int felbm_mesh_create(const double* xy, int32_t n_nodes, const int32_t* tri, int32_t n_tri,
                      const int32_t* wall_edges, const int32_t* wall_id, int32_t n_wall_edges,
                      double period_x, double period_y, felbm_mesh** out);
int felbm_mesh_info_get(const felbm_mesh* mesh, felbm_mesh_info* out);

/* One member mesh of a batch: the arguments of felbm_mesh_create. */
typedef struct felbm_mesh_desc {
    const double* xy;
    int32_t n_nodes;
    const int32_t* tri;
    int32_t n_tri;
    const int32_t* wall_edges;
    const int32_t* wall_id;
    int32_t n_wall_edges;
    double period_x, period_y;
} felbm_mesh_desc;

/* Merge independent meshes into one mesh (each keeps its own periodic
 * lengths; node ids of member k are offset by the node counts of members
 * 0..k-1; wall ids are used as given, so give each member its own ids to
 * give it its own contact angle).  Same validation and errors as
 * felbm_mesh_create.  Every kernel of felbm_step then advances all members in
 * the same launches; felbm_diagnostics_groups reports them one by one. */
int felbm_mesh_create_batch(int32_t n_meshes, const felbm_mesh_desc* meshes, felbm_mesh** out);

/* Batches.  A mesh may consist of several connected components -- e.g. many
 * independent droplet domains concatenated into one node/triangle list, each
 * with its own wall ids (and so its own contact angle).  felbm_step advances
 * all of them in the same kernel launches.  The components are the "groups",
 * numbered by their lowest caller node id (so concatenating meshes in order
 * numbers them in that order).  Node ranges of each group, caller order:
 * group_first_node[g] = lowest caller id of group g; sizes in group_nodes.
 * Either pointer may be NULL; arrays hold n_groups entries. */
int felbm_mesh_groups(const felbm_mesh* mesh, int32_t* group_first_node, int32_t* group_nodes);
void felbm_mesh_destroy(felbm_mesh* mesh);

/* Bytes of device workspace a state of this mesh and these params needs. */
int felbm_workspace_bytes(const felbm_mesh* mesh, const felbm_params* params, size_t* bytes);

/* Create a state on the device: upload the mesh tables into the workspace and
 * set g, h to the equilibria of eqn::g_eq and eqn::f_eq at the initial
 * fields: g = w p + rho cs2 (Gamma(u) - w), h = Gamma(u) C, with
 * rho = C rho_l + (1 - C) rho_v.
 *  C0  double [n_nodes] host, caller order (required)
 *  p0  double [n_nodes] host or NULL (p = 0)
 *  u0  double [2][n_nodes] host (u_x then u_y) or NULL (u = 0; the state
 *      at rest, g = w p, h = w C)
 * FP32_DEV states store C (FP64), p, u (rounded to FP32) and zero
 * deviations.  d_workspace: device pointer, 256-byte aligned, >=
 * felbm_workspace_bytes.  stream: cudaStream_t.  The mesh may be destroyed
 * after this call.  Synchronises the stream. */
int felbm_init(const felbm_mesh* mesh, const felbm_params* params, const double* C0, const double* p0,
               const double* u0, void* d_workspace, size_t workspace_bytes, void* stream, felbm_state** out);

/* Enqueue n_steps time steps (Sec. II.C): moments, chemical potential with the
 * wetting boundary (eqn:mp_mu, eqn:lapl_int_mp, eqn:bc2), element Laplacian of
 * mu (Sec. II.D), P0 forces at the barycentre (eq:G, eq:H, eq:intF),
 * collision (eqn::collide), weak-form streaming right-hand side
 * (eq:galerkin_lbm, force term +(dt M10 + dt^2 K) Phi, weak bounce-back at
 * walls) and the consistent-mass solve, all as one CUDA graph per step on the
 * state's stream.  Does not synchronise. */
int felbm_step(felbm_state* state, int32_t n_steps);

/* Reduce the diagnostics of Sec. III on the device (deterministic FP64
 * reductions) and copy them to *out.  req may be NULL (no band, substrate 0).
 * Synchronises the stream.  Returns FELBM_ERR_NONFINITE (and fills *out) if
 * the state holds a NaN or Inf. */
int felbm_diagnostics(felbm_state* state, const felbm_diag_request* req, felbm_diag* out);

/* Raw sums behind one felbm_diag and the step they belong to (doubles). */
#define FELBM_DIAG_SLOTS 16

/* felbm_diagnostics in two halves, so that reading one step's result back
 * does not hold up the host.  felbm_diagnostics_enqueue queues the same
 * device reductions on the state's stream, then an asynchronous copy of their
 * raw sums into `slots` (FELBM_DIAG_SLOTS doubles of host memory,
 * caller-owned; pinned for the copy to be asynchronous), writes the current
 * step count into the last slot, and returns without synchronising.  Once
 * the stream has passed that point (the caller synchronised the stream or an
 * event recorded after it, or called a synchronising function of the
 * library), felbm_diag_finish turns the sums into *out exactly as
 * felbm_diagnostics does (same req), returning FELBM_ERR_NONFINITE with *out
 * filled if the state held a NaN or Inf.  Neither allocates. */
int felbm_diagnostics_enqueue(felbm_state* state, const felbm_diag_request* req, double* slots);
int felbm_diag_finish(felbm_state* state, const felbm_diag_request* req, const double* slots, felbm_diag* out);

/* Batch schedule (FELBM_FP32_DEV states): members (groups) of at most
 * cta_max_nodes nodes each run in ONE thread block that performs the whole
 * time step with block-level barriers only (no kernel boundaries), on a side
 * branch of the step's CUDA graph; the larger members run the tiled kernels
 * meanwhile.  0 = tiled kernels for every member (default).  The step graph
 * is rebuilt at the next felbm_step.  Results do not depend on the schedule. */
int felbm_batch_schedule(felbm_state* state, int32_t cta_max_nodes);

/* Opt-in convergence check of the mass solve (Sec. II.C).  The solve runs a
 * fixed number of steps (no residual is formed in the step itself); with the
 * check on, every time step also computes, before the last step of its
 * solve, the residual r = b - M x of the current iterate over all 18
 * right-hand sides (b: the solve's right-hand side, carried through the
 * corrections of the mixed solve), and felbm_diagnostics, felbm_diag_finish
 * and felbm_diagnostics_groups report ||r|| / ||b|| of the last step's solve
 * in solver_residual and return FELBM_ERR_NOT_CONVERGED (with the diagnostics
 * filled, status = FELBM_ERR_NOT_CONVERGED) when it is above tol.  Costs one
 * extra pass over the mesh per step.  With a CTA batch schedule it covers the
 * members on the tiled kernels.  FELBM_ERR_UNSUPPORTED for the FP64 solver
 * mode.  enable = 0 switches it off (tol ignored).  The step graph is
 * rebuilt at the next felbm_step.  Synchronises. */
int felbm_solver_check(felbm_state* state, int32_t enable, double tol);

/* Threads per node of the FP32 solve sweeps (states with an FP32 solve):
 * 1, 2, 3 or 6, each owning 18 / parts of the node's right-hand sides.  Every
 * choice performs the same arithmetic per row, so the trajectory does not
 * depend on it; felbm_autotune picks one by timing.  Default 2.  The step
 * graph is rebuilt at the next felbm_step.  FELBM_ERR_INVALID_ARG for any
 * other value. */
int felbm_sweep_parts(felbm_state* state, int32_t parts);

/* Where the FP32 store sweeps of the solve read their operands (states with
 * an FP32 solve and an ELL pattern).  0: each thread gathers its row's
 * neighbours from global memory.  1: a persistent grid, one block per SM,
 * walks (node tile, part of the right-hand sides) items through up to four
 * stages of shared memory: 1D TMA bulk copies bring the tile's runs of the iterate,
 * right-hand side, ELL rows and inverse lumped mass, cp.async the tile's
 * halo, while the block computes an earlier item from another stage.
 * The tiled step splits the 18 right-hand sides in 3 or 6 parts (the
 * felbm_sweep_parts value if it is one of those and fits, else 6).  Same
 * arithmetic in the same order: the trajectory does not depend on it.
 * FELBM_ERR_UNSUPPORTED if a tile's halo exceeds the staged rows (504
 * nodes) or the rows are too long for two stages.  On the meshes measured
 * here the gathered form is faster (the autotuner keeps it).  A tiled sweep whose
 * copy has not landed after 0.2 s stops (and later blocks skip their work)
 * and sets an error bit that the next felbm_diagnostics or felbm_get_state
 * reports as FELBM_ERR_CUDA.
 * The step graph is rebuilt at the next felbm_step.  Default 0;
 * felbm_autotune picks one by timing. */
int felbm_sweep_tiled(felbm_state* state, int32_t on);

typedef struct felbm_tune_result {
    int32_t sweep_parts;     /* chosen threads per node of the FP32 solve sweeps */
    float parts_ms[4];       /* step time with 1, 2, 3, 6 threads per node (0 = not timed) */
    int32_t sweep_tiled;     /* 1: the tiled store sweeps were chosen (felbm_sweep_tiled) */
    float tiled_ms[4];       /* step time of the tiled sweeps with 1, 2, 3, 6 parts (0 = not timed) */
    int32_t cta_max_nodes;   /* chosen batch threshold (0 = tiled only) */
    int32_t n_candidates;
    int32_t candidates[16];  /* thresholds timed */
    float step_ms[16];       /* mean device time of one step for each */
} felbm_tune_result;

/* Autotuner: times `trials` steps (after one warm-up step) per candidate and
 * keeps the fastest -- first the threads per node of the FP32 solve sweeps
 * (1, 2, 3 or 6; states with an FP32 solve and an ELL pattern; see
 * felbm_sweep_parts), each gathered and tiled (felbm_sweep_tiled), then, for
 * FP32_DEV batches, each distinct split of the members (tiled only, CTA per
 * member up to 2^11 .. 2^17 nodes).  The state and the step count are saved
 * before and restored after, so the simulation is unchanged.  Synchronises. */
int felbm_autotune(felbm_state* state, int32_t trials, felbm_tune_result* out);

/* Diagnostics per group (see felbm_mesh_groups): out[g] for g < n_groups, each
 * reduced over its own nodes, triangles and wall edges in one CTA per group
 * (deterministic).  reqs: NULL or n_groups requests (band, substrate wall id
 * of each group).  mass0 / mass_drift_rel are relative to the group's mass
 * at felbm_init.  Synchronises.  Returns FELBM_ERR_NONFINITE if any group
 * holds a NaN or Inf (all of out is filled). */
int felbm_diagnostics_groups(felbm_state* state, const felbm_diag_request* reqs, int32_t n_groups,
                             felbm_diag* out);

/* Copy the distributions out / in: g, h double [9][n_nodes] host, caller order.
 * Pinned host memory makes the copies asynchronous DMA.  get_state synchronises
 * the stream.  set_state copies on a stream of its own into one of two input
 * buffers used in turn, so the copy overlaps the work already queued on the
 * state's stream (the previous step); it returns once the host arrays have
 * been read, and the conversion into the state stays queued on the state's
 * stream behind that work, ahead of any later work the caller enqueues there. */
int felbm_get_state(felbm_state* state, double* g, double* h);
int felbm_set_state(felbm_state* state, const double* g, const double* h);

/* Nodal fields of the last step's start (moments of the pre-collision state
 * and the chemical potential): each double [n_nodes] host, caller order, any
 * may be NULL.  Recomputes them from the current state first.  Synchronises. */
int felbm_get_fields(felbm_state* state, double* C, double* p, double* ux, double* uy, double* mu);

/* Solve M11 X = B for k right-hand sides with the state's mass matrix and
 * the same solver felbm_step uses (Sec. II.C: consistent mass matrix,
 * lumped-mass preconditioner).  B, X: double [k][n_nodes] host,
 * caller order; 1 <= k <= 18.  Uses the state's scratch buffers; do not
 * overlap with felbm_step on another stream.  Synchronises. */
int felbm_mass_solve(felbm_state* state, const double* B, double* X, int32_t k);

/* Capacity of the device scratch array behind felbm_mass_solve_static. */
#define FELBM_STATIC_SCRATCH_BYTES (64u << 20)

/* felbm_mass_solve without any device allocation, for callers that cannot
 * allocate: code running where cudaMalloc is not allowed or not wanted (a
 * stream-ordered section that must not synchronise, a plugin whose host
 * application owns all device memory) and that cannot lend the state's
 * workspace either, because felbm_step may be using it.  It enqueues CUDA
 * work, so it must not be called from inside a stream callback
 * (cudaLaunchHostFunc), where CUDA calls are not allowed.
 * The paper has no counterpart: this is an interface convenience only.
 *
 * Solves M11 X = B exactly as felbm_mass_solve does (same solver, same
 * arithmetic) but takes DEVICE pointers and keeps its iterates in one
 * library-owned static device array of FELBM_STATIC_SCRATCH_BYTES (64 MiB)
 * per GPU, held by every GPU that loads the library until the process
 * exits.  Nothing is allocated and nothing is freed.
 *  d_B, d_X  device pointers, double [k][n_nodes], caller order; 1 <= k <= 18.
 *            X may not alias B.
 *  Size limit: the 18-row scratch needs 648 bytes per node (padded to 64
 *  nodes), i.e. meshes up to ~103,000 nodes; larger meshes get
 *  FELBM_ERR_WORKSPACE before anything is enqueued.
 * Enqueued on the state's stream; returns without synchronising.  The first
 * call on a device looks up the array's device address (once per device, with
 * that device made current); make that first call before any stream capture.
 * The address is kept for the life of the process: the library must not be
 * used across a cudaDeviceReset of that device.
 * Every call shares the one array of its device and leaves its contents
 * behind: calls that overlap on the GPU race, so serialise them (one stream,
 * or events).  They may overlap with felbm_step, which does not touch it. */
int felbm_mass_solve_static(felbm_state* state, const double* d_B, double* d_X, int32_t k);

/* ---------------------------------------------------------------- adjoint
 * Reverse-mode derivatives of felbm_step for FELBM_FP64 states (the paper has
 * no adjoint).  With lambda = dL/dpsi^{n+1}
 * seeded, felbm_adjoint_step maps it to dL/dpsi^n using the CURRENT state as
 * psi^n (restore it with felbm_checkpoint_load / felbm_set_state first) and
 * adds (d psi^{n+1}/d phi_c)^T lambda to the wetting-potential gradient.  The
 * reverse of each part of the step: the mass solve (M11 is symmetric: the
 * same solver), the element residuals and the node gathers (transposed as
 * gathers, no atomics), the P0 forces and the collision (Jacobians by
 * forward-mode dual numbers), the chemical potential with its wetting flux,
 * and the moments.  Enqueued on the state's stream; does not synchronise. */
int felbm_adjoint_seed(felbm_state* state, const double* dL_dg, const double* dL_dh);  /* host [9][N] each */
int felbm_adjoint_step(felbm_state* state);
/* Copy lambda (= dL/dpsi of the state the last adjoint step was taken at;
 * either pointer pair may be NULL) and the accumulated dL/dphi_c per wall id
 * ([n_wall_ids] or NULL) to the host.  Synchronises. */
int felbm_adjoint_get(felbm_state* state, double* dL_dg, double* dL_dh, double* dL_dphi_c);

/* Replace the wetting potentials phi_c[0..n_wall_ids) of a state (e.g. between
 * runs of a gradient check); takes effect at the next step.  Synchronises. */
int felbm_set_wetting(felbm_state* state, const double* phi_c, int32_t n_wall_ids);

/* Device-to-device snapshots of the state (the checkpoints of the adjoint's
 * recomputation): d_buf is a caller-owned device buffer of
 * felbm_checkpoint_bytes.  Enqueued on the state's stream. */
int felbm_checkpoint_bytes(const felbm_state* state, size_t* bytes);
int felbm_checkpoint_save(felbm_state* state, void* d_buf);
int felbm_checkpoint_load(felbm_state* state, const void* d_buf);

/* Device time of the phases of one time step, milliseconds, from CUDA events
 * recorded inside the step's graph (instrumentation, not part of the method). */
typedef struct felbm_step_timing {
    float collide_ms;   /* moments and collision */
    float mu_ms;        /* chemical potential with the wetting flux */
    float gradmu_ms;    /* P0 gradient of mu */
    float element_ms;   /* element Laplacian of mu, forces, element residual */
    float rhs_ms;       /* streaming right-hand-side gather */
    float solve_ms;     /* all sweeps of the mass solve */
    float total_ms;
    int32_t solve_launches;  /* kernel launches inside solve_ms */
    int32_t launches;        /* kernel launches of one step */
} felbm_step_timing;

/* Switch the per-phase events on or off; the step graph is rebuilt at the
 * next felbm_step.  Off by default. */
int felbm_timing_enable(felbm_state* state, int32_t enable);

/* Phase times of the most recent felbm_step launch of the graph (the last of
 * its n_steps).  Synchronises the stream.  FELBM_ERR_INVALID_ARG if timing
 * is off or no step ran since it was switched on. */
int felbm_timing_get(felbm_state* state, felbm_step_timing* out);

/* Instrument: the FP64 FMA rate of the current device in TFLOP/s (2 flops
 * per FMA), from the best of three timed launches of independent FMA chains
 * on every SM, after a warm-up launch.  The roof of the kernels that the
 * FP64 pipe bounds (the FP64 step's element and right-hand-side kernels).
 * stream: cudaStream_t or NULL.  Synchronises the stream; allocates
 * nothing. */
int felbm_fp64_fma_rate(void* stream, double* tflops);

/* Release the host-side state object (the caller frees the workspace). */
void felbm_state_destroy(felbm_state* state);

#ifdef __cplusplus
}
#endif
#endif /* FELBM_H */
