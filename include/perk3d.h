/*
 * libperk 3D — P-ERK multirate time stepping of an octree DGSEM on one GB300.
 *
 * The three-dimensional counterpart of perk.h for the paper's Sec. 7.1.3 (the
 * Taylor-Green vortex on an adaptively refined octree, Eq. IC_TaylorGreen): the
 * same P-ERK step (Sec. 2, Eq. PartitionedRKSystem; Sec. 3.1,
 * Eq. PERK_ButcherTableauClassic; Sec. 3.3 for third order) over the level
 * partition of a 2:1-balanced periodic octree (Sec. 6.2), with the DGSEM of
 * Sec. 6.1 on hexahedra: flux-differencing volume integral with Ranocha's
 * entropy-conservative two-point flux, HLL / HLLC / HLLE / EC surface fluxes,
 * and L2 mortars at hanging faces (one large face against four small ones).
 * Compressible Euler or Navier-Stokes (BR1) equations.
 *
 * Conventions (in addition to those of perk.h, whose status codes and surface
 * flux identifiers are shared)
 *   - Solution and stage arrays are FP64 device memory owned by the caller,
 *     laid out U[n_elem][5][n][n][n] in C order, n = N+1 (N = 2 or 3):
 *     conserved variable (rho, rho v1, rho v2, rho v3, E), then the node index
 *     k along z, j along y, i along x.  Element e is the e-th cell passed to
 *     perk3d_mesh_upload.  U must be 16-byte aligned.
 *   - All device work is enqueued on the context's stream; host arrays are
 *     copied during the call; no exception crosses the ABI, and a failed call
 *     leaves a message readable with perk3d_last_error().
 */
#ifndef PERK3D_H
#define PERK3D_H

#include <stddef.h>
#include <stdint.h>

#include "perk.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct perk3d_ctx perk3d_ctx;

typedef struct {
  int N;             /* polynomial degree: 2 (the paper's Taylor-Green runs, 27 nodes) or 3 (64 nodes) */
  double gamma;      /* ratio of specific heats, > 1 */
  int surface_flux;  /* perk_surface_flux: HLL, HLLC, EC or HLLE (the paper's choice in Sec. 7.1.3) */
  int use_graph;     /* nonzero: perk3d_step replays a captured CUDA graph of the whole step */
  int equations;     /* perk_equations: Euler, or Navier-Stokes with BR1 viscous terms (gradients of
                        (v1, v2, v3, T = p/rho) by central lifting, stress mu (grad v + grad v^T -
                        (2/3) div v I), heat flux kappa grad T with kappa = mu gamma / ((gamma-1) Pr),
                        central viscous face flux; mortar averages as for the inviscid traces) */
  double mu;         /* dynamic viscosity (Navier-Stokes), > 0 */
  double prandtl;    /* Prandtl number (Navier-Stokes), > 0 */
} perk3d_problem;

/* Creates a context on the current CUDA device (INVALID_ARG for N outside {2, 3}, gamma <= 1,
 * an unknown flux or equation set, or a non-positive mu or Pr for Navier-Stokes; CUDA when no
 * device is usable). */
perk_status perk3d_create(const perk3d_problem* prob, perk3d_ctx** out);
/* Frees the context and every device buffer it owns.  NULL is ignored. */
void perk3d_destroy(perk3d_ctx* ctx);
/* Message of the last failed call on ctx ("" if none); ctx == NULL: the last failed
 * context-free call of this thread. */
const char* perk3d_last_error(const perk3d_ctx* ctx);
/* Sets the stream (a cudaStream_t cast to void*; NULL = legacy default stream). */
perk_status perk3d_set_stream(perk3d_ctx* ctx, void* stream);

/* Mesh upload (Sec. 6.2, TreeMesh in 3D).  cells[4*e + {0,1,2,3}] = (level, ix, iy, iz) of
 * leaf e: level 0 is the periodic cube [x0, x0+length]^3 and the cell covers
 * [ix, ix+1) x [iy, iy+1) x [iz, iz+1) in units of length / 2^level (level <= 19).  The
 * leaves must tile the cube exactly and be 2:1 balanced across faces (else INVALID_ARG).
 * Builds interfaces and mortars on the host, uploads them and runs the level partition
 * when a tableau is set.  Invalidates any captured step graph. */
perk_status perk3d_mesh_upload(perk3d_ctx* ctx, int64_t n_cells, const int32_t* cells, double x0, double length);

/* Host utility (no device work): the connectivity perk3d_mesh_upload builds for the same
 * cells.  Interfaces: ifs[4*q + {0,1,2,3}] = (left, right, dir, 0): the +dir face of left
 * meets the -dir face of right (dir 0 = x, 1 = y, 2 = z).  Mortars: morts[6*q + {0..5}] =
 * (large, s0, s1, s2, s3, dir | large_side << 2): the small cells ordered s_{q1 + 2 q2} by
 * their quadrant (q1, q2) of the large face along its tangential axes t1 < t2 (0 = lower
 * half); large_side 0 means the large cell lies on the -dir side.  Counts go to *n_if and
 * *n_mort; the arrays are filled only when their capacities (in records) suffice. */
perk_status perk3d_mesh_faces(int64_t n_cells, const int32_t* cells, int64_t* n_if, int32_t* ifs, int64_t if_cap,
                              int64_t* n_mort, int32_t* morts, int64_t mort_cap);

/* Sizes, levels and per-stage active counts (the struct of perk.h; index_bytes also counts
 * the mortars' small-cell table). */
perk_status perk3d_mesh_query(const perk3d_ctx* ctx, perk_mesh_info* info);

/* P-ERK coefficient table with the conventions of perk_set_tableau (order 2 or 3, S <= 64
 * stages, R <= 8 members with ascending E[r], E[R-1] = S; c[S]; a[r*S + i] = a_{i+1,i}^{(r)},
 * zero where member r does not evaluate stage i).  The tables of perk_perk2_disk_tableau and
 * perk_perk3_disk_tableau apply unchanged.  Re-runs the partition when a mesh is present. */
perk_status perk3d_set_tableau(perk3d_ctx* ctx, int order, int S, int R, const int32_t* E, const double* c,
                               const double* a);

/* Right-hand sides with the stage state given (d_Y, d_K: n_elem * 5 n^3 doubles each):
 * K = F(Y) on every element, or K = I^{act(stage)} F(Y) on the members active at stage
 * (0-based; entries of inactive elements are left untouched, not zeroed). */
perk_status perk3d_rhs_full(perk3d_ctx* ctx, const double* d_Y, double* d_K);
perk_status perk3d_rhs_active(perk3d_ctx* ctx, int stage, const double* d_Y, double* d_K);

/* One P-ERK step of size dt in place (Eq. PartitionedRKSystem): per stage one face launch
 * and one volume launch over the active prefixes, stage states formed inside the kernels,
 * then the guarded update.  A step whose new state would have rho <= 0, p <= 0 or a
 * non-finite value is not committed (U keeps U_n) and perk3d_check reports NONFINITE. */
perk_status perk3d_step(perk3d_ctx* ctx, double* d_U, double dt);
/* Synchronises the stream; NONFINITE if a step since the last check was rejected (the flag
 * is then cleared), else OK. */
perk_status perk3d_check(perk3d_ctx* ctx);
/* dt = cfl * min_e h_e / ((N+1) max_nodes(|v1| + |v2| + |v3| + 3c)) on the device
 * (Eq. TimestepConstraint with the three axes' convective speeds).  Blocks. */
perk_status perk3d_compute_dt(perk3d_ctx* ctx, const double* d_U, double cfl, double* dt);

/* perk3d_step without a graph, with CUDA events around every launch; blocks.  Kinds:
 * 0 = faces (interfaces and mortars, one launch per stage), 1 = volume, 2 = final update,
 * 3 = viscous terms (Navier-Stokes: the four BR1 launches of a stage, timed as one group).
 * Accumulates into acc (the struct of perk.h). */
perk_status perk3d_step_profiled(perk3d_ctx* ctx, double* d_U, double dt, perk_kernel_times* acc);
/* Steps, element-stage evaluations and node-stage (DoF-stage) updates since creation. */
perk_status perk3d_get_counters(const perk3d_ctx* ctx, perk_counters* out);

/* Adaptive refinement (Sec. 7.1.3: the enstrophy indicator of Eq. Enstrophy; the AMR cycle of
 * Sec. 6.2 before the partition is re-assigned).  Thresholds apply to the indicator below. */
typedef struct {
  int32_t level_min, level_max;   /* allowed levels of the adapted mesh */
  double refine_above;            /* refine cells whose indicator exceeds this */
  double coarsen_below;           /* cells below this may coarsen (all eight siblings together) */
} perk3d_amr_params;

/* Indicator per element (device output d_eta[n_elem]): the largest nodal value of the enstrophy
 * rho |curl v|^2 / 2, the velocity derivatives taken from the element's nodal polynomial,
 * (2/h) D along each axis.  Asynchronous. */
perk_status perk3d_amr_indicator(perk3d_ctx* ctx, const double* d_U, double* d_eta);

/* Plans one AMR cycle on the host: desired levels either from the indicator of d_U and prm
 * (level + 1 above refine_above up to level_max, level - 1 below coarsen_below down to
 * level_min), or given (desired: host array n_elem, each within one level of the cell's), then
 * raised to their least fixed point under the sibling rule (a cell coarsens only with its seven
 * siblings, all wanting to) and the 2:1 rule across faces.  *n_new receives the number of
 * cells of the new mesh.  Blocks when the indicator is computed. */
perk_status perk3d_adapt_plan(perk3d_ctx* ctx, const perk3d_amr_params* prm, const int32_t* desired, const double* d_U,
                              int64_t* n_new);

/* Applies the plan: d_Unew (n_new elements, caller-owned, distinct from d_Uold) receives the
 * transferred solution (kept cells copied, refined cells' children interpolated from the
 * parent polynomial, coarsened groups L2-projected onto the parent), and the new leaves (in
 * Morton order) become the context's mesh with its connectivity and partition rebuilt.  A plan
 * that changes no cell copies the state and keeps the mesh. */
perk_status perk3d_adapt_commit(perk3d_ctx* ctx, const double* d_Uold, double* d_Unew);

/* Host utility (no device work, no context): the plan perk3d_adapt_plan makes from given desired
 * levels, for the leaf list cells[4 * n_cells] (a 2:1-balanced tiling of the cube, as for
 * perk3d_mesh_upload).  levels[n_cells] receives the desired levels raised to the sibling and 2:1
 * rules; *n_new the number of new leaves; when cap >= *n_new, new_cells[4 * n_new] receives them in
 * Morton order and map[9 * n_new] their transfer records: map[9 q] = kind | cx << 2 | cy << 3 |
 * cz << 4 (kind 0: copy of old cell map[9 q + 1]; 1: child (cx, cy, cz) of old cell map[9 q + 1];
 * 2: parent of the old cells map[9 q + 1 + (cx + 2 cy + 4 cz)]).  INVALID_ARG for a malformed mesh
 * or a desired level more than one away from its cell's. */
perk_status perk3d_amr_plan_cells(int64_t n_cells, const int32_t* cells, const int32_t* desired, int32_t* levels,
                                  int64_t* n_new, int32_t* new_cells, int32_t* map, int64_t cap);

/* The current leaves (host, 4 * n_elem int32: level, ix, iy, iz), cap in cells. */
perk_status perk3d_get_cells(const perk3d_ctx* ctx, int32_t* cells, int64_t cap);

#ifdef __cplusplus
}
#endif

#endif /* PERK3D_H */
