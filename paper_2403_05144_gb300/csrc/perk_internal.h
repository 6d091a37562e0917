// Internal declarations shared by the host runtime (perk_host.cpp) and the
// kernels (perk_kernels.cu).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "perk.h"

namespace perk {

constexpr int NN = 4;             // LGL nodes per direction (N = 3)
constexpr int NODES = NN * NN;    // nodes per element
constexpr int NV = 4;             // conserved variables
constexpr int ELEM = NV * NODES;  // doubles per element
constexpr int MAX_S = 64;
constexpr int MAX_R = 8;
constexpr int DT_THREADS = 256;   // threads per block of the CFL step-size reduction
constexpr int DT_MAX_BLOCKS = 1024;   // its grid cap (grid-stride), the size of its per-block scratch

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount), looked up
// once per device and cached; grid caps of the grid-stride kernels are multiples of it.
int device_sm_count();
// Blocks of the fused stage kernel the current device holds at once (0 if unknown), cached per
// device; looked up when a context is created.
int stage_resident_blocks();

// Reference-element operators, computed on the host once per context.
struct Ops {
  double dsplit[NN][NN];  // 2 D_ij off the diagonal, 0 on it (LGL: 2 D_00 + 1/w_0 = 0 = 2 D_NN - 1/w_N)
  double dmat[NN][NN];    // the derivative matrix D_ij = l_j'(x_i) itself
  double inv_w0;          // 1 / w_0 = 1 / w_N
  double p_lo[NN][NN];    // large-face trace -> lower half-face nodes (interpolation)
  double p_hi[NN][NN];    // large-face trace -> upper half-face nodes
  double r_lo[NN][NN];    // lower half-face flux -> large face (exact L2 projection)
  double r_hi[NN][NN];    // upper half-face flux -> large face
  double gamma;
  double inv_gm1;         // 1 / (gamma - 1)
  double gm1;             // gamma - 1
  int surface_flux;       // perk_surface_flux
  // subcell shock capturing (perk_shock): indicator variable, cap, inverse of the orthonormal
  // Legendre Vandermonde matrix at the nodes, 1/w_i, threshold T and sharpness s / T
  int shock;
  double alpha_max;
  double vinv[NN][NN];
  double inv_w[NN];
  double sc_T, sc_s_over_T;
};

// Y = U + dt * (alpha * K1 + beta * Kprev) for an element of a given member at a given stage;
// Kprev = K_{i-1}, or with all stages stored (StageArgs::Kall, stage patterns) K_src.
struct StageCoef {
  double alpha;
  double beta;
  int32_t src;   // 0-based stage of Kprev when StageArgs::Kall is set
  int32_t pad;
};

// Where the stage state comes from.
enum YSource { Y_GIVEN = 0, Y_COMBINE = 1 };

struct StageArgs {
  const double* Y;        // Y_GIVEN: the stage vector
  const double* U;        // Y_COMBINE: U_n
  const double* K1;       //            K_1
  const double* Kp;       //            K_{i-1}
  const StageCoef* coef;  //            [R] coefficients of this stage
  const double* dt;       //            device array: dt of each ensemble member
  const int32_t* member;  //            ensemble member of each element (nullptr: member 0)
  const double* Kall;     //            all stages, stage s at Kall + s * nd (nullptr: use Kp)
  int64_t nd;
  // one launch per step only: the elements' progress stamps (stage s of the step complete at
  // prog_base + s + 1), the stage these arguments serve, and the flag raised if a wait gives up
  const unsigned long long* prog;
  unsigned long long prog_base;
  int stage;
  int* err;
};

#ifdef __CUDACC__
// the stage a member couples to besides K_1
__device__ __forceinline__ const double* coupled_stage(const StageArgs& sa, const StageCoef& c) {
  return sa.Kall ? sa.Kall + (int64_t)c.src * sa.nd : sa.Kp;
}
#endif

// Final-update description (P-ERK2: b = e_S; P-ERK3: b on K_1, K_{S-1}, K_S).
struct UpdateArgs {
  double b1, bp, bs;      // weights of K_1, K_{S-1}, K_S
  const double* U;
  const double* K1;
  const double* Kp;
  int* flag;              // raised (set to 1) when any new state is not admissible
  const int32_t* member;  // ensemble member of each element (nullptr: member 0)
  unsigned long long* stage_ctl;  // fused stage kernels' counters, advanced by the final update (or nullptr)
};

// ---- reference-element routines for any degree N (perk_host.cpp; host only) ----
double legendre(int n, double x, double* dp);                              // P_n(x), P_n'(x)
void lgl(int N, std::vector<double>& x, std::vector<double>& w);          // Gauss-Lobatto nodes, weights
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);
void lagrange_values(const std::vector<double>& x, double t, double* out);  // l_j(t), j < x.size()
std::vector<double> log_table();   // [inv_c[128], ln_c[128]] of the table-driven logarithm

// ---- kernel launchers (perk_kernels.cu); all return cudaGetLastError() ----

// mort_flag_bits: low bits of a mortar record's .w that carry its geometry (2 in 2D: dir,
// large side; 3 in 3D: dir in two bits, large side); the P-ERK member is stored above them.
cudaError_t launch_partition(cudaStream_t st, int64_t n_elem, int64_t n_if, int64_t n_mort, const int32_t* level,
                             const int4* if_raw, const int4* mort_raw, int R, int S, const int32_t* stage_minmem,
                             const int32_t* member, int n_members, int32_t* member_lmax /* [n_members] */,
                             int32_t* method, int32_t* elem_sorted, int4* if_sorted, int4* mort_sorted,
                             int64_t* counts /* [3][MAX_S] */, int32_t* level_minmax /* [2] */,
                             int mort_flag_bits = 2, const int64_t* d_nfaces = nullptr);
// (d_nfaces: if set, the interface and mortar counts are read from d_nfaces[0], d_nfaces[1] on the
// device instead of n_if, n_mort, which are then only upper bounds)

// per-member CFL reduction: out[m] = min over member m's elements of h_e / lambda_e (out pre-set to +inf)
cudaError_t launch_dt_members(cudaStream_t st, int64_t n_elem, const double* U, const int32_t* level,
                              const int32_t* member, int n_members, double length, double gamma, double* out);

cudaError_t launch_faces(cudaStream_t st, YSource ysrc, const Ops& ops, int64_t n_if, const int4* ifs, int64_t n_mort,
                         const int4* morts, const int32_t* method, const StageArgs& sa, double* surf);

// elems_per_block: 2, 4 or 8 (cudaErrorInvalidValue otherwise)
constexpr int VOL_EPB_DEFAULT = 2;
cudaError_t launch_volume(cudaStream_t st, YSource ysrc, const Ops& ops, int64_t n, const int32_t* elems,
                          const int32_t* level, const int32_t* method, double inv_len2, const StageArgs& sa,
                          const double* surf, double* K, const UpdateArgs* check, const double* log_table,
                          int elems_per_block = VOL_EPB_DEFAULT);

// One stage in one launch (faces and volume; Euler without shock capturing): ctl[MAX_S + 1] (zero
// before the first step; the step's final update, with UpdateArgs::stage_ctl = ctl, makes it ready
// for the next step), stamps[4 * n_elem] (zero, or stamps of earlier launches with the same ctl),
// err: bit 1 raised if a volume item gives up waiting.
// One launch per step (k_step): the work items of all stages, dealt in stage order (faces, then
// volume items, within each stage) from one counter; stage i's items are first[i] .. first[i+1].
constexpr int STEP_MAX_S = 32;
struct StepPlan {
  int S;
  int64_t first[STEP_MAX_S + 1];
  int64_t n_if[STEP_MAX_S], n_mort[STEP_MAX_S], n_el[STEP_MAX_S];   // active counts of each stage
  double* K[STEP_MAX_S];          // stage i's output
  const double* Kp[STEP_MAX_S];   // K_{i-1} as stage i reads it
};
// items of one stage (faces first), as k_step deals them
int64_t step_stage_items(int64_t n_if, int64_t n_mort, int64_t n_el);
// sa: U, K_1, the coefficients of stage 0 (stage i at sa.coef + i * MAX_R), dt, member;
// check: the last stage's admissibility arguments; ctl[0] is the item counter (zero at launch;
// the commit resets it), ctl[MAX_S] the step count; prog: n progress stamps
cudaError_t launch_step(cudaStream_t st, const Ops& ops, const StepPlan& plan, const int4* ifs, const int4* morts,
                        const int32_t* elems, const int32_t* level, const int32_t* method, double two_over_len,
                        const StageArgs& sa, double* surf, const UpdateArgs& check, const double* log_table,
                        unsigned long long* ctl, unsigned long long* stamps, unsigned long long* prog, int* err);
cudaError_t launch_stage(cudaStream_t st, int stage, const Ops& ops, int64_t n_if, const int4* ifs, int64_t n_mort,
                         const int4* morts, int64_t n_el, const int32_t* elems, const int32_t* level,
                         const int32_t* method, double two_over_len, const StageArgs& sa, double* surf, double* K,
                         const UpdateArgs* check, const double* log_table, unsigned long long* ctl,
                         unsigned long long* stamps, int* err);

// log_table: [inv_c[128], ln_c[128]] of the volume kernel's logarithm (see perk_kernels.cu)
constexpr int LOG_TABLE_SIZE = 128;
cudaError_t launch_selftest_math(cudaStream_t st, int64_t n, const double* x, double* out, const double* log_table);

cudaError_t launch_commit(cudaStream_t st, int64_t n_elem, const UpdateArgs& ua, const double* Ks, const double* dt,
                          double* U);

cudaError_t launch_set_scalar(cudaStream_t st, double* p, double v);

cudaError_t launch_indicator(cudaStream_t st, int64_t n, const double* U, const Ops& ops, double w0, double w1,
                             int kind, double* eta);

// ---- AMR cycle on the device (perk_amr.cu); cells are int4 (level, ix, iy, member) in
// member-major Morton order ----
struct AmrPlanArgs {
  int level_min, level_max;
  double refine_above, coarsen_below;
};
// desired levels from eta (when eta is set; else d holds them already), balanced in place; then
// off[n + 1] = exclusive offsets of the new leaves, info[0] = new cell count, info[1] = changed,
// info[4] = 1 if the balance did not settle within its pass bound
cudaError_t launch_amr_plan(cudaStream_t st, int64_t n, const int4* cells, const double* eta, const AmrPlanArgs& a,
                            int64_t n_if, const int4* ifs, int64_t n_mort, const int4* morts, int32_t* d,
                            int32_t* off, int64_t* info);
// new leaves (out), their Morton keys and transfer records (5 int32 each)
cudaError_t launch_amr_leaves(cudaStream_t st, int64_t n, const int4* cells, const int32_t* d, const int32_t* off,
                              int4* out, unsigned long long* key, int32_t* map);
// interfaces and mortars of a leaf list with its keys (scratch cnt_*, off_*: n each); counts to
// info[2], info[3]; ifs and morts need room for 2 n records each
cudaError_t launch_connect(cudaStream_t st, int64_t n, const int4* cells, const unsigned long long* key,
                           int32_t* cnt_if, int32_t* cnt_mort, int32_t* off_if, int32_t* off_mort, int4* ifs,
                           int4* morts, int64_t* info);
// level and member of every cell
cudaError_t launch_amr_install(cudaStream_t st, int64_t n, const int4* cells, int32_t* level, int32_t* member);
cudaError_t launch_transfer(cudaStream_t st, int64_t n, const int32_t* map, const double* Uold, const Ops& ops,
                            double* Unew);

// derivatives (perk_adjoint.cu)
cudaError_t launch_jvp(cudaStream_t st, const Ops& ops, int64_t n_if, const int4* ifs, int64_t n_mort,
                       const int4* morts, int64_t n_el, const int32_t* elems, const int32_t* level,
                       double two_over_len, const double* Y, const double* V, const double* logt, double* surf,
                       double* surf_d, double* K, double* Kd);
// VJP of one partitioned RHS evaluation: the face adjoints into gsurf (which must be zero) and the
// volume adjoint of the active prefix into g, in one launch of dealt items (n_act = 0: faces only;
// n_if = n_mort = 0: volume only; *ticket is the launch's item counter and must be zero); then the
// gather g = (active ? g : 0) + face adjoints.
cudaError_t launch_vjp_stage(cudaStream_t st, YSource ysrc, const Ops& ops, int64_t n_act, const int32_t* elems,
                             int64_t n_if, const int4* ifs, int64_t n_mort, const int4* morts, const int32_t* level,
                             const int32_t* method, int min_member, double two_over_len, const StageArgs& sa,
                             const double* lam, const double* logt, double* g, double* gsurf,
                             unsigned long long* ticket);
cudaError_t launch_vjp_gather(cudaStream_t st, int64_t n, const int32_t* method, int min_member, const double* gsurf,
                              double* g);
// over the elements elems[0 .. n) (the stage's halo); clears the face adjoints it gathers
cudaError_t launch_adj_accum(cudaStream_t st, int64_t n, const int32_t* elems, const int32_t* method, int min_member,
                             const StageCoef* coef, double dt, const double* g, double* gsurf, double* lamU,
                             double* lamK1, double* lamKp, int assign_p);
cudaError_t launch_adj_seed(cudaStream_t st, int64_t n, double dt, double b1, double bp, double bs, const double* lam,
                            double* lamU, double* lamK1, double* lamKp, double* lamKs);

// BR1 viscous terms of one stage (perk_br1.cu): gradients on every element and face, viscous
// flux and divergence on the active ones; K += viscous part; check: admissibility on the last stage
cudaError_t launch_br1(cudaStream_t st, YSource ysrc, const Ops& ops, double mu, double kappa, int64_t n_if_all,
                       int64_t n_mort_all, int64_t n_if_act, int64_t n_mort_act, const int4* ifs, const int4* morts,
                       int64_t n_all, int64_t n_act, const int32_t* elems, const int32_t* level, const int32_t* method,
                       double two_over_len, const StageArgs& sa, double* wsurf, double* q, double* vsurf, double* K,
                       const UpdateArgs* check);

// Records the message of a failed context-free call (read by perk_last_error(NULL)).
perk_status set_context_free_error(perk_status s, const char* msg);

cudaError_t launch_dt(cudaStream_t st, int64_t n_elem, const double* U, const int32_t* level, double length,
                      double gamma, double* block_min, int n_blocks, double* out);

}  // namespace perk
