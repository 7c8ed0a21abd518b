/*
 * felbm3d.h -- C ABI of the 3D FE-LBM step: two D3Q19 distribution sets on
 * unstructured linear tetrahedra (the paper's own setting, arXiv:1708.04678,
 * Sec. II: D3Q19 lattice, P1 tetrahedra, the wetting condition eqn:bc2 on
 * wall faces).  The scheme is that of felbm.h with d = 3:
 *  - collision eqn::collide, streaming eqn::stream in the Galerkin weak form
 *    eq:galerkin_lbm with P0 forces eq:G / eq:H at the element barycentre;
 *  - patch Laplacian of C (eqn:lapl_int_mp) divided by V = 3/4 |patch|
 *    (FELBM_LAP_CONSISTENT, equal to the lumped P1 Laplacian) or |patch|
 *    (FELBM_LAP_PAPER); wall faces carry the wetting flux of eqn:bc2;
 *  - element Laplacian of mu through the four faces (Sec. II.D), wall faces 0;
 *  - weak bounce-back of incoming populations on wall faces;
 *  - consistent-mass solve with the lumped-mass preconditioner, whose
 *    spectrum lies in [1/5, 1] on any P1 tetrahedral mesh.
 *
 * Conventions are those of felbm.h (return codes, felbm_last_error, caller
 * node numbering, caller-owned workspace, one stream per state, no device
 * allocation by the library).  Parameters use felbm_params; solver_iters 0
 * means 36 FP64 sweeps (solver_mode FP64, error bound 2 x 0.382^36) or 16 FP32
 * sweeps per correction (MIXED, 3 corrections for FP64 storage, 1 for
 * FP32_DEV storage).
 *
 * Distribution layout on the host: double [19][n_nodes], direction-major,
 * D3Q19 order e_0 = (0,0,0); e_1..e_6 = (1,0,0),(-1,0,0),(0,1,0),(0,-1,0),
 * (0,0,1),(0,0,-1); e_7..e_18 = (1,1,0),(-1,-1,0),(1,-1,0),(-1,1,0),
 * (1,0,1),(-1,0,-1),(1,0,-1),(-1,0,1),(0,1,1),(0,-1,-1),(0,1,-1),(0,-1,1);
 * weights 1/3, 1/18 (axis), 1/36 (diagonal); c_s^2 = 1/3.
 */
#ifndef FELBM3D_H
#define FELBM3D_H

#include "felbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct felbm3d_mesh felbm3d_mesh;
typedef struct felbm3d_state felbm3d_state;

typedef struct felbm3d_mesh_info {
    int32_t n_nodes, n_tet, n_wall_faces;
    int32_t nnz;              /* entries of the node-node sparsity pattern */
    int32_t max_degree;       /* largest row of that pattern */
    int32_t bandwidth;        /* after reverse Cuthill-McKee */
    int32_t max_incidence;    /* most tetrahedra at one node */
    double min_volume, total_volume;
} felbm3d_mesh_info;

typedef struct felbm3d_diag_request {
    double centre[3];         /* droplet centre for the interface band */
    double radius;            /* band = nodes with |r - radius| <= band */
    double band;              /* half width (the paper uses xi, Table I) */
    int32_t substrate_wall_id;/* wall id of the contact-angle measurement; <0: none */
} felbm3d_diag_request;

typedef struct felbm3d_diag {
    int64_t step;
    double mass, mass0, mass_drift_rel;  /* sum_i m_i C_i, m_i = |patch_i| / 4 */
    double kinetic_energy;    /* 1/2 sum_i rho_i |u_i|^2 / N */
    double max_u;             /* max_i |u_i| */
    double interface_rho_uu;  /* nodal-volume-weighted mean of rho |u|^2 over the band (Table I) */
    double p_in, p_out, delta_p; /* volume-weighted mean p over C >= 0.95 / C <= 0.05 */
    double wetted_area;       /* area of the substrate where the linear C >= 1/2 */
    double height;            /* highest C = 1/2 crossing on a tetrahedron edge above the mean substrate height */
    double base_diameter;     /* 2 sqrt(wetted_area / pi) */
    double theta_deg;         /* atan2(b, 2 (r - h)), r = (4 h^2 + b^2) / (8 h) (Sec. III.B) */
    int32_t status;           /* FELBM_OK or FELBM_ERR_NONFINITE */
} felbm3d_diag;

/* Preprocess a tetrahedral mesh (host only; no device work).
 *  xyz         double [n_nodes][3] node coordinates
 *  tet         int32  [n_tet][4] vertices; positive volume after the minimum image
 *  wall_faces  int32  [n_wall_faces][3] node triples of the boundary faces
 *  wall_id     int32  [n_wall_faces] wall id of each face (< FELBM_MAX_WALL_IDS)
 *  period      double [3] periodic lengths (0 = not periodic along that axis)
 * Every face that belongs to one tetrahedron only must be a wall face and
 * every wall face such a face.  Errors: FELBM_ERR_INVALID_ARG (null or
 * negative sizes, ids out of range, a node repeated in a tetrahedron),
 * FELBM_ERR_BAD_MESH (non-positive volume, a face of three or more
 * tetrahedra, boundary and wall faces differ). */
int felbm3d_mesh_create(const double* xyz, int32_t n_nodes, const int32_t* tet, int32_t n_tet,
                        const int32_t* wall_faces, const int32_t* wall_id, int32_t n_wall_faces,
                        const double* period, felbm3d_mesh** out);
int felbm3d_mesh_info_get(const felbm3d_mesh* mesh, felbm3d_mesh_info* out);
void felbm3d_mesh_destroy(felbm3d_mesh* mesh);

/* Bytes of device workspace felbm3d_init needs for this mesh and precision. */
int felbm3d_workspace_bytes(const felbm3d_mesh* mesh, const felbm_params* params, size_t* bytes);

/* Upload the mesh tables into d_workspace and set the state to rest:
 * g = w p0 with p0 = 0, h = w C0 (C0: double [n_nodes], caller order).
 * Enqueues on stream and synchronises it.  The mesh may be destroyed after. */
int felbm3d_init(const felbm3d_mesh* mesh, const felbm_params* params, const double* C0, void* d_workspace,
                 size_t workspace_bytes, void* stream, felbm3d_state** out);

/* Enqueue n_steps time steps (one CUDA graph launch each); asynchronous. */
int felbm3d_step(felbm3d_state* st, int32_t n_steps);

/* Global diagnostics of the current state (synchronises the stream). */
int felbm3d_diagnostics(felbm3d_state* st, const felbm3d_diag_request* req, felbm3d_diag* out);

/* felbm3d_diagnostics in two halves, as felbm_diagnostics_enqueue /
 * felbm_diag_finish in 2D: the reductions and an asynchronous copy of their
 * raw sums into `slots` (FELBM_DIAG_SLOTS doubles of caller-owned host
 * memory, pinned for an asynchronous copy; the last slot receives the step
 * count) are queued on the state's stream without a synchronisation; once
 * the stream has passed that point, felbm3d_diag_finish (same req) forms
 * *out exactly as felbm3d_diagnostics does. */
int felbm3d_diagnostics_enqueue(felbm3d_state* st, const felbm3d_diag_request* req, double* slots);
int felbm3d_diag_finish(felbm3d_state* st, const felbm3d_diag_request* req, const double* slots,
                        felbm3d_diag* out);

/* Copy the distributions to / from host arrays double [19][n_nodes] each
 * (caller order).  FP32_DEV storage converts: get returns psi^eq + dpsi, set
 * recomputes the fields and the FP32 deviations.  get_state synchronises the
 * stream.  set_state copies on a stream of its own into one of two input
 * buffers used in turn, so the copy overlaps the work already queued on the
 * state's stream; it returns once the host arrays have been read, and the
 * conversion stays queued on the state's stream behind that work. */
int felbm3d_get_state(felbm3d_state* st, double* g, double* h);
int felbm3d_set_state(felbm3d_state* st, const double* g, const double* h);

/* Macroscopic fields of the current state (caller order, double [n_nodes]
 * each; u as three arrays; mu is the chemical potential of the last step's
 * force evaluation, 0 before the first step).  Any pointer may be NULL. */
int felbm3d_get_fields(felbm3d_state* st, double* C, double* p, double* ux, double* uy, double* uz, double* mu);

/* Per-phase device times of the next felbm3d_step (graph event nodes):
 * enable = 1 records, felbm3d_timing_get reads the last recorded step:
 * ms[0] collision + chemical potential, ms[1] grad mu, ms[2] element forces
 * and residual, ms[3] right-hand side gather, ms[4] mass solve; total in ms[5]. */
int felbm3d_timing_enable(felbm3d_state* st, int32_t enable);
int felbm3d_timing_get(felbm3d_state* st, double* ms6);

/* Number of kernels one felbm3d_step launches. */
int felbm3d_step_launches(const felbm3d_state* st, int32_t* n);

void felbm3d_state_destroy(felbm3d_state* st);

#ifdef __cplusplus
}
#endif

#endif /* FELBM3D_H */
