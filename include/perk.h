/*
 * libperk — P-ERK multirate time stepping of a quadtree DGSEM on one GB300.
 *
 * C ABI of the library.  The method is the Paired-Explicit Runge-Kutta (P-ERK)
 * scheme applied to the partitioned ODE of a DGSEM semidiscretisation whose
 * partitions are the refinement levels of an adaptively refined quadtree
 * (Doehring et al., arXiv 2403.05144: Sec. 2, Eq. PartitionedODESys and
 * Eq. PartitionedRKSystem; Sec. 3.1, Eq. PERK_ButcherTableauClassic; Sec. 6.2).
 *
 * Conventions shared by every call
 *   - Solution and stage arrays are FP64, device memory owned by the caller,
 *     laid out U[n_elem][4][n][n] in C order with n = N+1 = 4: conserved
 *     variable (rho, rho v1, rho v2, E), then the node index j along y, then
 *     the node index i along x.  Element e is the e-th cell passed to
 *     perk_mesh_upload.  Pointers are not retained after a call returns.
 *   - All device work is enqueued on the context's stream (perk_set_stream);
 *     calls return once the work is enqueued unless stated otherwise.
 *   - Host arrays are copied during the call.
 *   - Every call returns a perk_status; no exception crosses the ABI.  On an
 *     error the context keeps a message readable with perk_last_error().
 */
#ifndef PERK_H
#define PERK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PERK_OK = 0,
  PERK_E_INVALID_ARG = 1, /* bad pointer, size, level, or an unbalanced / non-periodic mesh */
  PERK_E_CUDA = 2,        /* a CUDA runtime call failed; the message names it */
  PERK_E_NONFINITE = 3,   /* a step produced NaN/Inf or non-positive density or pressure;
                             the step was not committed and U is unchanged */
  PERK_E_TIMEOUT = 4,     /* a bounded device wait expired */
  PERK_E_NOT_READY = 5,   /* mesh or tableau missing */
  PERK_E_OOM = 6          /* device allocation failed */
} perk_status;

/* Surface fluxes: HLL with Davis' wave speeds, HLLC (Toro), the entropy-conservative two-point
 * flux, and HLLE (HLL with Einfeldt's Roe-averaged bounds, the flux of the paper's
 * shock-capturing runs, Sec. 7.2). */
typedef enum { PERK_SURFACE_HLL = 0, PERK_SURFACE_HLLC = 1, PERK_SURFACE_EC = 2, PERK_SURFACE_HLLE = 3 } perk_surface_flux;

/* Subcell shock capturing of the volume term (Sec. 7.2; Hennemann, Rueda-Ramirez, Hindenlang
 * and Gassner 2021).  Per element, from the nodal indicator variable epsilon (rho p, or rho as
 * in the paper's KH run): its orthonormal-Legendre modes m_ab, the shares of the highest mode
 * shells, energy = max(E_{max(a,b)=N} / E_all, E_{max(a,b)=N-1} / E_{max(a,b)<=N-1}), and the
 * blending factor alpha = 1 / (1 + exp(-(s/T)(energy - T))), T = 0.5 10^(-1.8 (N+1)^(1/4)),
 * s = ln((1 - 1e-4)/1e-4), set to 0 below 1e-3 and capped at alpha_max.  The volume term becomes
 * (1 - alpha) (flux differencing) + alpha (first-order finite volumes on the LGL subcells, the
 * surface flux between neighbouring nodes); the surface term is unchanged. */
typedef enum { PERK_SHOCK_OFF = 0, PERK_SHOCK_DENSITY_PRESSURE = 1, PERK_SHOCK_DENSITY = 2 } perk_shock;

/* Equations: compressible Euler, or Navier-Stokes with BR1 viscous terms
 * (Sec. 7.1; gradients of (v1, v2, T = p/rho), central lifting and viscous
 * flux, constant viscosity mu, heat conductivity mu gamma / ((gamma-1) Pr)). */
typedef enum { PERK_EULER = 0, PERK_NAVIER_STOKES = 1 } perk_equations;

typedef struct perk_ctx perk_ctx;

/* Problem description; N = 3 (4 x 4 Gauss-Lobatto nodes per quadrilateral). */
typedef struct {
  int N;                 /* polynomial degree; must be 3 */
  double gamma;          /* ratio of specific heats, > 1 */
  int surface_flux;      /* perk_surface_flux */
  int use_graph;         /* nonzero: perk_step replays a captured CUDA graph of the whole step */
  int equations;         /* perk_equations */
  double mu;             /* dynamic viscosity (Navier-Stokes), > 0 */
  double prandtl;        /* Prandtl number (Navier-Stokes), > 0 */
  int shock_capturing;   /* perk_shock; PERK_SHOCK_OFF (0) for the plain volume term */
  double alpha_max;      /* cap of the blending factor, in (0, 1] when shock capturing is on */
} perk_problem;

/* Creates a context on the current CUDA device.  *out receives the handle. */
perk_status perk_create(const perk_problem* prob, perk_ctx** out);
/* Frees the context and every device buffer it owns.  NULL is ignored. */
void perk_destroy(perk_ctx* ctx);
/* Message of the last failed call on ctx ("" if none).  Valid until the next call.
 * With ctx == NULL: the message of the last failed context-free call on this thread. */
const char* perk_last_error(const perk_ctx* ctx);
/* Sets the stream (a cudaStream_t cast to void*; NULL = legacy default stream). */
perk_status perk_set_stream(perk_ctx* ctx, void* stream);

/* Mesh upload (Sec. 6.2, TreeMesh).  cells[3*e + {0,1,2}] = (level, ix, iy) of
 * leaf e: level 0 is the periodic square [x0, x0+length]^2 and the cell covers
 * [ix, ix+1) x [iy, iy+1) in units of length / 2^level (level <= 20).  The leaves must tile
 * the square exactly and be 2:1 balanced across faces (else INVALID_ARG).
 * Builds interfaces (equal-size faces) and mortars (2:1 hanging faces) on the
 * host, uploads them, and runs the level partition (perk_partition) if a
 * tableau is set.  Invalidates any captured step graph. */
perk_status perk_mesh_upload(perk_ctx* ctx, int64_t n_cells, const int32_t* cells, double x0, double length);

/* Host utility (no device work): the face connectivity perk_mesh_upload would
 * build for the same cells.  Interfaces: ifs[4*q + {0,1,2,3}] = (left, right,
 * dir, 0): the +dir face of `left` meets the -dir face of `right` (dir 0 = x,
 * 1 = y).  Mortars: morts[4*q + {0,1,2,3}] = (large, small_lo, small_hi,
 * dir | large_side << 1): the large cell's face against the two small cells
 * (ordered by the tangential coordinate); large_side 0 means the large cell is
 * on the -dir side.  *n_if and *n_mort receive the counts; the arrays are
 * filled only if their capacities (in records) suffice. */
perk_status perk_mesh_faces(int64_t n_cells, const int32_t* cells, int64_t* n_if, int32_t* ifs, int64_t if_cap,
                            int64_t* n_mort, int32_t* morts, int64_t mort_cap);

/* Ensemble of independent simulations in one context (batching): member m's
 * leaves are cells[3 * (offset_m + k) + ...], k < n_cells[m], with the same
 * conventions as perk_mesh_upload, every member on its own periodic square
 * [x0, x0 + length]^2.  Elements are numbered member after member; faces never
 * cross members.  Each member has its own level partition (its finest present
 * level gets the finest P-ERK member), but all members share one coefficient
 * table, so one launch per kernel and stage covers the active work of every
 * member.  perk_step gives every member the same dt; perk_step_dts one dt per
 * member.  AMR (perk_adapt_*) adapts every member's mesh. */
perk_status perk_ensemble_upload(perk_ctx* ctx, int n_members, const int64_t* n_cells, const int32_t* cells, double x0,
                                 double length);
/* Member of every element (host, n_elem int32), cap in elements. */
perk_status perk_get_members(const perk_ctx* ctx, int32_t* member, int64_t cap);

typedef struct {
  int64_t n_elem;
  int64_t n_interfaces;
  int64_t n_mortars;
  int32_t level_min, level_max;
  int32_t S;                  /* stages of the current tableau (0 if none) */
  int64_t dof_stage_updates;  /* sum over stages of active nodes, per step */
  int64_t active_elements[64];/* active elements per stage (first S entries) */
  int64_t active_interfaces[64];
  int64_t active_mortars[64];
  int64_t index_bytes;        /* device bytes of the partition data (method ids and sorted lists) */
} perk_mesh_info;
perk_status perk_mesh_query(const perk_ctx* ctx, perk_mesh_info* info);

/* P-ERK coefficient table (Sec. 3.1, Eq. PERK_ButcherTableauClassic; Sec. 4.3).
 * order: 2 (b = e_S) or 3 (b = 1/6 on K_1 and K_{S-1}, 2/3 on K_S; Eq. PERK_ThirdOrderShuOsher).
 * S stages (2 <= S <= 64), R members (1 <= R <= 8) with ascending E[r] <= S.
 * c[i], i = 0..S-1: shared abscissae.  a[r*S + i] = a_{i+1,i}^{(r)} (the
 * coefficient of K_{i} in stage i+1, 1-based), zero where member r has no such
 * entry; a_{i,1}^{(r)} = c_i - a_{i,i-1}^{(r)} by internal consistency.
 * Member r evaluates K_1 and K_{S-E[r]+2} .. K_S.  Runs perk_partition if a
 * mesh is present.  Invalidates any captured step graph. */
perk_status perk_set_tableau(perk_ctx* ctx, int order, int S, int R, const int32_t* E, const double* c,
                             const double* a);

/* Stage patterns (Sec. 3.2.4).  eval[r*S + i] (0 or 1): member r evaluates stage i (0-based);
 * src[r*S + i]: the stage it couples to at stage i besides K_1, with the coefficient a[r*S + i]
 * (Y_i = U + dt ((c_i - a) K_1 + a K_src)).  Second order, b = e_S.  Each member evaluates the
 * first and the last stage and E[r] stages in all; a member's stages are also evaluated by every
 * finer member (so each stage's active elements stay a prefix of the sorted lists); a nonzero
 * coupling needs src < i and an evaluated source stage; the largest member evaluates every stage.
 * INVALID_ARG otherwise.  When some member couples to a stage other than K_{i-1}, the step keeps
 * all S stages (S x n_elem x 512 B of device memory), and derivatives are refused. */
perk_status perk_set_tableau_pattern(perk_ctx* ctx, int order, int S, int R, const int32_t* E,
                                     const uint8_t* eval, const int32_t* src, const double* c, const double* a);

/* Host utility: the disk-polynomial family of perk_perk2_disk_tableau with a stage pattern:
 * 0 classic (1, S-E+2 .. S), 1 alternating (1 and S - floor((E-1-k)(S-1)/(E-1) + 1/2),
 * k = 1 .. E-1; S = 6, E = 4 gives 1, 3, 4, 6 as in Eq. PERK_ButcherTableauAlternating), 2 early
 * shared evaluations (1 .. E-1 and S, Eq. PERK_ButcherTableauEarlyShared).  Each evaluated stage
 * after the first one past K_1 couples to the member's previous evaluated stage; the couplings
 * follow from the polynomial's coefficients along that chain (Eq. PERKCoeffsConstruction).
 * Fills c[S], eval[R*S], src[R*S], a[R*S] for perk_set_tableau_pattern. */
perk_status perk_perk2_pattern_tableau(int S, int R, const int32_t* E, int pattern, double* c, uint8_t* eval,
                                       int32_t* src, double* a);

/* Weights of the final update of a second-order tableau (Sec. 3.1):
 * U_{n+1} = U_n + dt (b1 K_1 + bS K_S), b1 + bS = 1, bS > 0, with bS c_S = 1/2
 * for the abscissae already set (INVALID_ARG otherwise; NOT_READY without a
 * second-order tableau).  perk_set_tableau resets the weights to b = e_S
 * (second order) or (1/6, ..., 1/6, 2/3) on K_1, K_{S-1}, K_S (third order).
 * The step, its admissibility check and the step adjoint use them. */
perk_status perk_set_weights(perk_ctx* ctx, double b1, double bS);

/* Host utility (Sec. 4.3.1, Eq. PERKCoeffsConstruction): fills c[S] and
 * a[R*S] of a second-order family whose member r has the stability polynomial
 * P(z) = 1/E + ((E-1)/E)(1 + z/(E-1))^E, E = E[r] (the second-order optimum
 * for the disk |z + E - 1| <= E - 1). */
perk_status perk_perk2_disk_tableau(int S, int R, const int32_t* E, double* c, double* a);

/* The same family for the weights b_1 = 1 - bS, b_S = bS (0 < bS <= 1) of the
 * variants in Sec. 3.1: abscissae c_i = (i-1)/(2 bS (S-1)), so c_S = 1/(2 bS)
 * (bS = 1/2: Heun's weights, c_S = 1; bS = 3/4: Ralston's, c_S = 2/3); the
 * construction divides the polynomial's coefficients by bS.  bS = 1 gives
 * perk_perk2_disk_tableau.  Use with perk_set_weights. */
perk_status perk_perk2_disk_tableau_weights(int S, int R, const int32_t* E, double bS, double* c, double* a);

/* Host utility (Sec. 4.3.1, Eq. PERKCoeffsConstruction) for any second-order
 * stability polynomial, e.g. one optimised for a spectrum (Sec. 4.2): a[S]
 * receives the a_{i+1,i} (layout of one row of perk_set_tableau's a) of the
 * member with E evaluations in an S-stage family with weights b_1 = 1 - bS,
 * b_S = bS whose stability polynomial has the monomial coefficients
 * alpha[0..E]; alpha[0..2] must be 1, 1, 1/2.  The abscissae are those of
 * perk_perk2_disk_tableau_weights.  INVALID_ARG when a product in the
 * construction vanishes. */
perk_status perk_perk2_member(int S, int E, double bS, const double* alpha, double* a);

/* Third-order members (Sec. 3.3, Eq. PERK_ThirdOrderShuOsher; Sec. 4.3.2).
 * perk_perk3_disk_alpha: monomial coefficients alpha[0..E] of a degree-E,
 * third-order polynomial stable on the largest disk |z + r| <= r among
 * sum_k d_k (1 + z/r)^k, d >= 0, sum d = 1 (*radius receives r): feasibility
 * of the three order conditions for d is a linear program, solved exactly by
 * enumerating its basic solutions, and r is found by bisection.
 * perk_perk3_member: the free entries a_{i,i-1} (written to a_out[S] in the
 * layout of perk_set_tableau) of a member with E evaluations whose stability
 * polynomial has the coefficients alpha_3..alpha_E, with 0 < a_i < c_i; the
 * paper's nonlinear system, solved by damped Newton iterations from fixed
 * starting points (several solutions may exist; the first admissible one is
 * returned).  c_i = (i-1)/(S-3) for i <= S-2, c_{S-1} = 1, c_S = 1/2.
 * perk_perk3_disk_tableau: c[S] and a[R*S] of a whole family from both. */
perk_status perk_perk3_disk_alpha(int E, double* alpha, double* radius);
perk_status perk_perk3_member(int S, int E, const double* alpha, double* a_out);
perk_status perk_perk3_disk_tableau(int S, int R, const int32_t* E, double* c, double* a);

/* Level partition on the device (Sec. 6.2): member of every element from its
 * level (finest present level -> member R-1, next -> R-2, ..., the rest -> 0),
 * of every interface from its elements, of every mortar from its fine side;
 * then the element, interface and mortar lists sorted finest-member-first so
 * that the work active at every stage is a prefix of each list.  Blocks until
 * the per-stage counts are back on the host.  Normally called implicitly. */
perk_status perk_partition(perk_ctx* ctx);

/* Host utility: the N+1 Gauss-Lobatto nodes x[] (ascending, on [-1, 1]) and
 * weights w[] at which the library collocates the solution (only N = 3 is
 * built for stepping; any 1 <= N <= 16 is returned here).  Node (i, j) of an
 * element [x_lo, x_lo + h] x [y_lo, y_lo + h] sits at
 * (x_lo + h (1 + x[i]) / 2, y_lo + h (1 + x[j]) / 2). */
perk_status perk_reference_nodes(int N, double* x, double* w);

/* Full right-hand side K = F(Y) on every element (no partitioning). */
perk_status perk_rhs_full(perk_ctx* ctx, const double* d_Y, double* d_K);

/* Partitioned right-hand side of stage `stage` (0-based): K = I^{act} F(Y)
 * (Sec. 2.2 mask matrices).  Writes K only for elements of members active at
 * that stage; other elements of d_K are left untouched.  d_Y is the full
 * stage vector (active and inactive elements). */
perk_status perk_rhs_active(perk_ctx* ctx, int stage, const double* d_Y, double* d_K);

/* One P-ERK step of size dt, in place on d_U (Eq. PartitionedRKSystem).
 * Stage i forms Y_i element-wise from U_n, K_1 and K_{i-1} with the element's
 * member coefficients and evaluates F only on the active prefix.  The update
 * is committed only if every new node state is finite with positive density
 * and pressure; otherwise U is left unchanged and the context's sticky error
 * flag is raised (read it with perk_check).  Asynchronous. */
perk_status perk_step(perk_ctx* ctx, double* d_U, double dt);

/* perk_step with one step size per ensemble member (host array dts[n_members]). */
perk_status perk_step_dts(perk_ctx* ctx, double* d_U, const double* dts);

/* Synchronises the stream and returns PERK_E_NONFINITE if any step since the
 * last check was rejected (then clears the flag), PERK_E_TIMEOUT if a fused
 * stage gave up waiting for its face fluxes (the step was not committed
 * either), else PERK_OK. */
perk_status perk_check(perk_ctx* ctx);

/* One launch per stage (Eq. PartitionedRKSystem, each stage's partitioned RHS): for the
 * Euler equations with the plain volume term, the numerical fluxes of a stage's active
 * interfaces and mortars and the volume terms of its active elements run as one kernel whose
 * work items (faces first) are dealt in order to its blocks; each element's volume work waits,
 * with a bounded wait, for its four face fluxes before the surface lifting.  On by default
 * (enabled = 1); enabled = 0 selects two launches per stage (face fluxes, then volume terms).
 * enabled = 2 selects one launch per step for steps of at most 32 stages without a stage
 * pattern: the items of all stages are dealt in stage order from one counter, and an item waits
 * (bounded) for the stage vectors of the elements it reads through per-element progress stamps;
 * a wait that gives up abandons the step, which is then not committed (perk_check reports
 * PERK_E_TIMEOUT).  Results are bitwise the same in every mode.  For the Navier-Stokes
 * equations mode 1 puts the inviscid face and volume terms of a stage in one launch (BR1's
 * launches follow it) and mode 2 acts as mode 1; shock capturing always uses two launches.
 * Returns PERK_E_INVALID_ARG for other values. */
perk_status perk_set_stage_fusion(perk_ctx* ctx, int enabled);

/* Step size dt = cfl * min_e h_e / ((N+1) max_nodes(|v1| + |v2| + 2c)) computed
 * on the device (Eq. CFL_DG, Eq. TimestepConstraint).  Blocks; *dt receives it.
 * NONFINITE (and *dt untouched) when some node has no admissible wave speed:
 * rho <= 0, p <= 0 or a NaN/Inf entry. */
perk_status perk_compute_dt(perk_ctx* ctx, const double* d_U, double cfl, double* dt);

/* The step size of every ensemble member (host array dts[n_members]); for a
 * single mesh dts[0] equals perk_compute_dt's value.  Blocks.  NONFINITE as
 * for perk_compute_dt if any member has a node without an admissible state. */
perk_status perk_compute_dt_members(perk_ctx* ctx, const double* d_U, double cfl, double* dts);

/* Counters accumulated since creation (reporting, Sec. 6.4.1). */
typedef struct {
  int64_t steps;
  int64_t element_stage_evaluations; /* sum over steps and stages of active elements */
  int64_t dof_stage_updates;         /* the same in nodes */
  int64_t rejected_steps_checked;    /* steps found rejected by perk_check */
  int64_t device_allocations;        /* cudaMalloc calls the context made since its creation */
} perk_counters;
perk_status perk_get_counters(const perk_ctx* ctx, perk_counters* out);

/* Caller-owned workspace (the statement of the problem in Sec. 2 leaves memory to the caller;
 * the library's own device memory can be replaced by one block the caller allocates, e.g. a
 * torch tensor, bound once).  The block holds every device buffer of the mesh (levels, members,
 * interface and mortar records), of the level partition (method ids, sorted lists, per-stage
 * counts), of the step (K_1 and the two alternating stage buffers, the face fluxes, the
 * Navier-Stokes gradient and viscous-flux buffers, all S stages for a stage pattern), of the step
 * size and of an AMR cycle (indicator values, transfer records), laid out for meshes of up to
 * a given number of cells (at most 2 interfaces and 2 mortars per cell).
 * perk_workspace_bytes: *bytes receives the size of that layout for meshes of up to n_cells cells
 * (0: the current mesh's count) with the context's present equations and tableau; query it after
 * perk_set_tableau (a stage pattern adds S x n_cells x 512 B).
 * perk_bind_workspace: d_ws is device memory of `bytes` bytes, 256-byte aligned, owned by the
 * caller, which must keep it alive and unused by others until the context is destroyed or
 * another block is bound.  The call synchronises the context's stream, moves the buffers'
 * contents into the block, frees the library's own copies and drops the captured step graph.
 * After it, mesh upload, partition, step, step size, AMR and tuning make no device allocation
 * (perk_counters.device_allocations stays put); a mesh with more cells than the block serves is
 * refused with OOM (before any work of the call).  d_ws == NULL with bytes == 0 unbinds: the
 * buffers move back to the library's own allocations.  INVALID_ARG for a block smaller than the
 * current mesh needs or misaligned.  The derivative entry points (JVP, VJP, step adjoint) keep
 * allocating their own work arrays. */
perk_status perk_workspace_bytes(const perk_ctx* ctx, int64_t n_cells, size_t* bytes);
perk_status perk_bind_workspace(perk_ctx* ctx, void* d_ws, size_t bytes);

/* Derivatives of the partitioned right-hand side (the Jacobian apply that the
 * spectrum estimation of Sec. 4.1 iterates with, and the discrete adjoint).
 * stage = -1: the full F; stage = i >= 0: I^{act(i)} F as in perk_rhs_active.
 * perk_rhs_jvp: d_Kd = J(Y) V on the active elements (others untouched).
 * perk_rhs_vjp: d_g = J(Y)^T lam over every element; lam is read on the
 * active elements only (its other entries are treated as zero).  Both
 * differentiate the library's own discrete operator exactly (its branch
 * decisions are taken on the values of Y).  Device arrays, U layout.
 * Built for the Euler equations (INVALID_ARG for Navier-Stokes contexts). */
perk_status perk_rhs_jvp(perk_ctx* ctx, int stage, const double* d_Y, const double* d_V, double* d_Kd);
perk_status perk_rhs_vjp(perk_ctx* ctx, int stage, const double* d_Y, const double* d_lam, double* d_g);

/* Adjoint of one P-ERK step (Eq. PartitionedRKSystem, reverse sweep): given
 * U_n (device) and lam_np1 = dL/dU_{n+1}, writes lam_n = (dU_{n+1}/dU_n)^T
 * lam_np1 (device, distinct from lam_np1).  Recomputes and stores the step's
 * S stages (S x n_elem x 64 doubles of work space), then walks the stages
 * backwards: adjoint of each partitioned RHS by perk_rhs_vjp's kernels and of
 * the element-wise stage combinations.  The mesh must not change between the
 * forward step and this call.  Asynchronous. */
perk_status perk_step_vjp(perk_ctx* ctx, const double* d_Un, double dt, const double* d_lam_np1, double* d_lam_n);

/* The same adjoint split in two, for callers that keep the stages of the steps
 * they are going to reverse (the recomputation of a checkpoint window).
 * perk_step_store: one step d_U <- U_{n+1} exactly as perk_step computes it
 * (same kernels, same admissibility check and flag), additionally writing the
 * S stage derivatives to d_K (caller-owned device memory, S x n_elem x 64
 * doubles, stage i at d_K + i * n_elem * 64, U layout each).
 * perk_step_vjp_stored: the reverse sweep of perk_step_vjp from those stored
 * stages: d_Un is the state the stages were computed from (not the updated
 * one), d_K is read only.  The mesh and dt must be those of the store call.
 * Euler single-member contexts; INVALID_ARG otherwise.  Asynchronous. */
perk_status perk_step_store(perk_ctx* ctx, double* d_U, double dt, double* d_K);
perk_status perk_step_vjp_stored(perk_ctx* ctx, const double* d_Un, double dt, const double* d_K,
                                 const double* d_lam_np1, double* d_lam_n);

/* Chooses the elements per block of the volume kernel (2, 4 or 8; 2 until
 * this is called) for this context: the volume term of every element of the
 * current mesh at the stage state d_U (device, U layout) is timed with each
 * choice (CUDA events, one untimed and five timed launches each) and the
 * fastest is kept for every later launch, including a re-captured step graph.
 * *elems_per_block (may be NULL) receives the choice.  Results do not depend
 * on the choice.  Blocks. */
perk_status perk_autotune_volume(perk_ctx* ctx, const double* d_U, int32_t* elems_per_block);

/* Chooses the launch structure of the step for this context and mesh: how the stages of
 * Eq. PartitionedRKSystem are launched, not what they compute (the modes of
 * perk_set_stage_fusion: 1 one launch per stage, 2 one launch per step, 0 two launches per
 * stage; only 0 where the equations or shock capturing allow no fusion): one untimed and five
 * timed steps from the state d_U (device, U layout; left unchanged) with the step sizes dts
 * (host, one per ensemble member) in each mode (CUDA events), and the fastest is kept for every
 * later step.  *mode (may be NULL) receives it.  Results do not depend on the mode.
 * PERK_E_NOT_READY if a rejected step is pending (perk_check first).  Blocks. */
perk_status perk_autotune_step(perk_ctx* ctx, const double* d_U, const double* dts, int32_t* mode);
/* Sets the elements per block of the volume kernel (2, 4 or 8; INVALID_ARG
 * otherwise) without timing. */
perk_status perk_set_volume_blocks(perk_ctx* ctx, int32_t elems_per_block);

/* Adaptive mesh refinement (Sec. 7: the AMR callback every N_AMR steps, after
 * which the partition is re-assigned, Sec. 6.2).  Indicators (dimensionless):
 *   PERK_INDICATOR_DENSITY: the density gradient
 *     eta_e = h_e max_nodes |grad rho| / mean_e(rho);
 *   PERK_INDICATOR_LOHNER_VX: Loehner's second-difference estimator of the
 *     velocity v_x (the shear-layer indicator of Sec. 7.1.1; Loehner 1987 in
 *     the nodal form of Fryxell et al. 2000): the largest, over every three
 *     consecutive nodes u_-, u_0, u_+ of a grid line of the element in both
 *     directions, of |u_+ - 2 u_0 + u_-| / (|u_+ - u_0| + |u_0 - u_-|
 *     + eps (|u_+| + 2 |u_0| + |u_-|)), eps = PERK_LOHNER_EPS (0 where the
 *     denominator vanishes); in [0, 1].
 * Desired level of a cell: level + 1 if eta > refine_above (below level_max),
 * level - 1 if eta < coarsen_below (above level_min), else level; raised to
 * the least fixed point of two rules: a cell coarsens only together with its
 * three siblings (all leaves, all wanting to coarsen), and face neighbours of
 * the new mesh differ by at most one level. */
typedef enum { PERK_INDICATOR_DENSITY = 0, PERK_INDICATOR_LOHNER_VX = 1 } perk_indicator;
#define PERK_LOHNER_EPS 0.2
typedef struct {
  int32_t level_min, level_max;
  double refine_above, coarsen_below;
  int32_t indicator; /* perk_indicator */
} perk_amr_params;

/* eta of every cell of d_U into d_eta[n_elem] (device) by the given indicator
 * (INVALID_ARG for an unknown one). */
perk_status perk_amr_indicator(perk_ctx* ctx, int32_t indicator, const double* d_U, double* d_eta);

/* Plans one adaptation.  With desired == NULL the indicator of d_U and `prm`
 * decide; otherwise desired[n_elem] (host) gives each cell's wanted level
 * (level - 1 .. level + 1) and prm/d_U are ignored.  Either way the two rules
 * above are then enforced.  *n_new receives the number of cells of the new
 * mesh (its leaves are kept in Morton order).  Blocks. */
perk_status perk_adapt_plan(perk_ctx* ctx, const perk_amr_params* prm, const int32_t* desired, const double* d_U,
                            int64_t* n_new);

/* Executes the plan: d_Unew[n_new] (device, distinct from d_Uold) receives the
 * solution on the new leaves: copied, interpolated exactly from the parent
 * (refined cells) or the L2 projection of the four children (coarsened
 * cells); then the mesh is replaced and re-partitioned on the device.  Blocks. */
perk_status perk_adapt_commit(perk_ctx* ctx, const double* d_Uold, double* d_Unew);

/* perk_adapt_commit, then the step size of d_Unew on the new mesh for `cfl` (as
 * perk_compute_dt, Eq. CFL_DG, Eq. TimestepConstraint): on the device path it is computed with
 * the partition's counts and read back with them, so the call waits once.  PERK_E_NONFINITE as
 * perk_compute_dt.  Blocks. */
perk_status perk_adapt_commit_dt(perk_ctx* ctx, const double* d_Uold, double* d_Unew, double cfl, double* dt);

/* Host utility (no device work, no context): the balanced levels perk_adapt_plan derives from
 * desired levels for a single mesh: desired[n_cells] (each within one level of its cell's)
 * raised to the least fixed point of the sibling rule (a cell coarsens only with its three
 * siblings, all wanting to) and the 2:1 rule across faces, written to levels[n_cells].  cells as
 * for perk_mesh_upload; INVALID_ARG for a malformed mesh or a jump of more than one level. */
perk_status perk_amr_balance(int64_t n_cells, const int32_t* cells, const int32_t* desired, int32_t* levels);

/* The current leaves (host, 3 * n_elem int32: level, ix, iy), cap in cells. */
perk_status perk_get_cells(const perk_ctx* ctx, int32_t* cells, int64_t cap);

/* Per-kernel timing of one step (tracing).  Runs the step like perk_step but
 * without a graph, with CUDA events recorded on the context's stream around
 * every launch, and blocks until the step is done.  Kernel kinds:
 * 0 = face fluxes, 1 = volume integral (with stage fusion: the whole stage, face
 * fluxes included, and kind 0 stays empty), 2 = final update, 3 = viscous terms
 * (Navier-Stokes: the four BR1 kernels of a stage, timed and counted as one
 * group).  ms[k] and launches[k] are accumulated (not reset) so a caller can
 * sum over steps. */
typedef struct {
  double ms[4];
  int64_t launches[4];
  int64_t element_stages; /* active elements summed over the profiled stages */
} perk_kernel_times;
perk_status perk_step_profiled(perk_ctx* ctx, double* d_U, double dt, perk_kernel_times* acc);

/* Diagnostics: the volume kernel's own logarithm and reciprocal (table-driven
 * logarithm after Tang 1990; Newton-Raphson reciprocal) evaluated on d_x[n]
 * (device, positive normal values): d_out[2q] = ln x_q, d_out[2q+1] = 1/x_q
 * (device, 2n doubles).  For testing their error against reference values. */
perk_status perk_selftest_math(perk_ctx* ctx, int64_t n, const double* d_x, double* d_out);

/* Throughput of the FP64 units of the current device, measured by short
 * microbenchmarks (~0.3 s): dependent-free FMA chains (returns FLOP/s, an FMA
 * counted as 2), and the division and natural-logarithm rates of CUDA's FP64
 * implementations (operations/s).  Blocks. */
perk_status perk_measure_fp64(double* fma_flops, double* div_per_s, double* log_per_s);

/* Allocation-free step size (no counterpart in the paper).  Computes the same
 * dt as perk_compute_dt, without a context and without allocating any device
 * memory, for callers that must not allocate: e.g. a solver invoked as a
 * custom call inside another framework that owns the device memory and its
 * allocator, where a cudaMalloc would bypass that pool and synchronise the
 * device.  Inputs: d_U as everywhere (device), d_level[n_elem] the refinement
 * level of each cell (device, int32), the domain length, gamma and cfl.
 * Output: *dt (host).  Runs on `stream` (a cudaStream_t, NULL = legacy
 * default stream) and blocks until the result is on the host.
 * Scratch: a file-scope device array of 64 KiB + 8 B that every GPU which
 * loads the library holds until the process exits; n_elem may not exceed
 * PERK_NOALLOC_MAX_ELEM (else INVALID_ARG).  The first call on a device looks
 * the array's device address up (cudaGetSymbolAddress) and keeps it for later
 * calls on that device; make that first call before any stream capture.  The
 * kept address does not survive cudaDeviceReset: after a reset of a device, do
 * not call this entry point on it again in the same process.  Every call
 * shares the one array, so calls that overlap on the GPU (other streams, other
 * host threads) race; serialise them.  NONFINITE as for perk_compute_dt. */
#define PERK_NOALLOC_MAX_ELEM 131072
perk_status perk_compute_dt_noalloc(const double* d_U, const int32_t* d_level, int64_t n_elem, double length,
                                    double gamma, double cfl, void* stream, double* dt);

#ifdef __cplusplus
}
#endif
#endif /* PERK_H */
