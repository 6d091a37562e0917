// Host runtime of libperk: the C ABI declared in include/perk.h.
//
// Owns the reference-element operators, the quadtree connectivity built from a
// leaf-cell list, the device copies of the mesh and of the level partition,
// the P-ERK coefficient table and the stage buffers, and drives one P-ERK
// step as 2S + 1 kernel launches (optionally replayed from a CUDA graph).

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "perk.h"
#include "perk_internal.h"

using namespace perk;

// ---------------------------------------------------------------------------
// Reference-element operators (N = 3 is the built case of the 2D path; the
// routines are generic in N and shared with the 3D runtime).
namespace perk {

double legendre(int n, double x, double* dp) {
  // P_n(x) and P_n'(x) by the three-term recurrence
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) {
    if (dp) *dp = 0.0;
    return 1.0;
  }
  for (int k = 2; k <= n; ++k) {
    const double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
    const double d2 = d0 + (2 * k - 1) * p1;
    p0 = p1;
    p1 = p2;
    d0 = d1;
    d1 = d2;
  }
  if (dp) *dp = d1;
  return p1;
}

// Gauss-Lobatto nodes: end points and the roots of P_N', found by Newton from
// Chebyshev-Gauss-Lobatto guesses using (1 - x^2) P_N' = N (P_{N-1} - x P_N).
void lgl(int N, std::vector<double>& x, std::vector<double>& w) {
  x.assign(N + 1, 0.0);
  w.assign(N + 1, 0.0);
  for (int i = 0; i <= N; ++i) {
    double xi = -std::cos(M_PI * i / N);
    if (i > 0 && i < N) {
      for (int it = 0; it < 100; ++it) {
        // q(x) = P_{N+1} - P_{N-1} vanishes exactly at the interior LGL nodes
        double dq1, dq0;
        const double q = legendre(N + 1, xi, &dq1) - legendre(N - 1, xi, &dq0);
        const double dx = q / (dq1 - dq0);
        xi -= dx;
        if (std::fabs(dx) < 1e-17) break;
      }
    }
    x[i] = xi;
    const double pn = legendre(N, xi, nullptr);
    w[i] = 2.0 / (N * (N + 1) * pn * pn);
  }
}

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double xi = -std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      const double p = legendre(n, xi, &dp);
      const double dx = p / dp;
      xi -= dx;
      if (std::fabs(dx) < 1e-17) break;
    }
    legendre(n, xi, &dp);
    x[i] = xi;
    w[i] = 2.0 / ((1.0 - xi * xi) * dp * dp);
  }
}

// Barycentric weights and Lagrange basis values l_j(t).
void lagrange_values(const std::vector<double>& x, double t, double* out) {
  const int n = (int)x.size();
  for (int j = 0; j < n; ++j) {
    double v = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) v *= (t - x[k]) / (x[j] - x[k]);
    out[j] = v;
  }
}

// Table of the volume kernel's logarithm: inv_c[j] = fl(1/c_j), c_j = 1 + (j + 1/2)/128,
// and ln_c[j] = -ln(inv_c[j]) evaluated in extended precision, then rounded.
std::vector<double> log_table() {
  std::vector<double> t(2 * LOG_TABLE_SIZE);
  for (int j = 0; j < LOG_TABLE_SIZE; ++j) {
    const long double c = 1.0L + (j + 0.5L) / LOG_TABLE_SIZE;
    const double inv = (double)(1.0L / c);
    t[j] = inv;
    t[LOG_TABLE_SIZE + j] = (double)(-logl((long double)inv));
  }
  return t;
}

}  // namespace perk

namespace {

bool invert4(const double A[NN][NN], double inv[NN][NN]) {
  double M[NN][2 * NN];
  for (int i = 0; i < NN; ++i)
    for (int j = 0; j < 2 * NN; ++j) M[i][j] = j < NN ? A[i][j] : (j - NN == i ? 1.0 : 0.0);
  for (int c = 0; c < NN; ++c) {
    int piv = c;
    for (int r = c + 1; r < NN; ++r)
      if (std::fabs(M[r][c]) > std::fabs(M[piv][c])) piv = r;
    if (M[piv][c] == 0.0) return false;
    for (int j = 0; j < 2 * NN; ++j) std::swap(M[c][j], M[piv][j]);
    const double d = M[c][c];
    for (int j = 0; j < 2 * NN; ++j) M[c][j] /= d;
    for (int r = 0; r < NN; ++r)
      if (r != c) {
        const double f = M[r][c];
        for (int j = 0; j < 2 * NN; ++j) M[r][j] -= f * M[c][j];
      }
  }
  for (int i = 0; i < NN; ++i)
    for (int j = 0; j < NN; ++j) inv[i][j] = M[i][j + NN];
  return true;
}

Ops build_ops(double gamma, int surface_flux, int shock = PERK_SHOCK_OFF, double alpha_max = 0.5) {
  Ops o{};
  std::vector<double> x, w;
  lgl(NN - 1, x, w);
  // shock capturing: V_ik = L_k(x_i) sqrt(k + 1/2) (orthonormal Legendre), its inverse, 1/w_i
  o.shock = shock;
  o.alpha_max = alpha_max;
  {
    double V[NN][NN];
    for (int i = 0; i < NN; ++i) {
      double p0 = 1.0, p1 = x[i];
      for (int k = 0; k < NN; ++k) {
        double pk;
        if (k == 0) {
          pk = 1.0;
        } else if (k == 1) {
          pk = x[i];
        } else {
          pk = ((2.0 * k - 1.0) * x[i] * p1 - (k - 1.0) * p0) / k;   // Bonnet's recursion
          p0 = p1;
          p1 = pk;
        }
        V[i][k] = pk * std::sqrt(k + 0.5);
      }
    }
    invert4(V, o.vinv);
    for (int i = 0; i < NN; ++i) o.inv_w[i] = 1.0 / w[i];
    o.sc_T = 0.5 * std::pow(10.0, -1.8 * std::pow((double)NN, 0.25));
    o.sc_s_over_T = std::log((1.0 - 1e-4) / 1e-4) / o.sc_T;
  }
  // derivative matrix from barycentric weights: D_ij = (lam_j / lam_i) / (x_i - x_j), rows sum to 0
  double lam[NN];
  for (int j = 0; j < NN; ++j) {
    double p = 1.0;
    for (int k = 0; k < NN; ++k)
      if (k != j) p *= x[j] - x[k];
    lam[j] = 1.0 / p;
  }
  for (int i = 0; i < NN; ++i)
    for (int j = 0; j < NN; ++j) o.dsplit[i][j] = (i == j) ? 0.0 : 2.0 * (lam[j] / lam[i]) / (x[i] - x[j]);
  for (int i = 0; i < NN; ++i) {
    double row = 0.0;
    for (int j = 0; j < NN; ++j)
      if (j != i) {
        o.dmat[i][j] = 0.5 * o.dsplit[i][j];
        row += o.dmat[i][j];
      }
    o.dmat[i][i] = -row;   // a derivative matrix annihilates constants
  }
  o.inv_w0 = 1.0 / w[0];
  // mortar operators: forward interpolation P_h[k][l] = l_l(position of node k of half h)
  for (int k = 0; k < NN; ++k) {
    lagrange_values(x, 0.5 * (x[k] - 1.0), o.p_lo[k]);
    lagrange_values(x, 0.5 * (x[k] + 1.0), o.p_hi[k]);
  }
  // exact mass matrix M_lm = int l_l l_m (Gauss-Legendre, NN points: exact to degree 2NN-1)
  std::vector<double> xg, wg;
  gauss_legendre(NN, xg, wg);
  double M[NN][NN] = {}, Mi[NN][NN];
  for (int g = 0; g < NN; ++g) {
    double L[NN];
    lagrange_values(x, xg[g], L);
    for (int l = 0; l < NN; ++l)
      for (int m = 0; m < NN; ++m) M[l][m] += wg[g] * L[l] * L[m];
  }
  invert4(M, Mi);
  // reverse (L2 projection) R_h = 1/2 M^{-1} P_h^T M
  for (int h = 0; h < 2; ++h) {
    const double(*P)[NN] = h ? o.p_hi : o.p_lo;
    double PtM[NN][NN] = {};
    for (int a = 0; a < NN; ++a)
      for (int b = 0; b < NN; ++b)
        for (int c = 0; c < NN; ++c) PtM[a][b] += P[c][a] * M[c][b];
    double(*R)[NN] = h ? o.r_hi : o.r_lo;
    for (int a = 0; a < NN; ++a)
      for (int b = 0; b < NN; ++b) {
        double s = 0.0;
        for (int c = 0; c < NN; ++c) s += Mi[a][c] * PtM[c][b];
        R[a][b] = 0.5 * s;
      }
  }
  o.gamma = gamma;
  o.gm1 = gamma - 1.0;
  o.inv_gm1 = 1.0 / (gamma - 1.0);
  o.surface_flux = surface_flux;
  return o;
}


// A device buffer of the context: allocated by the library (cudaMalloc, counted in *allocs), or
// carved from a caller-bound workspace (ext: never freed here, and never grown: a request beyond
// the carved capacity fails with cudaErrorMemoryAllocation).
template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t cap = 0;
  bool ext = false;
  int64_t* allocs = nullptr;
  cudaError_t ensure(size_t n) {
    if (n <= cap && p) return cudaSuccess;
    if (ext) return cudaErrorMemoryAllocation;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) {
      cap = std::max<size_t>(n, 1);
      if (allocs) *allocs += 1;
    }
    return e;
  }
  void release() {
    if (p && !ext) cudaFree(p);
    p = nullptr;
    cap = 0;
    ext = false;
  }
};

}  // namespace

struct perk_ctx {
  perk_problem prob{};
  Ops ops{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  // pinned host block for the small readbacks (counts, plan sizes, dt, flag): copies into it are
  // asynchronous, so a call that reads several values back waits once
  struct Pinned {
    int64_t counts[6 * MAX_S];
    int64_t info[8];
    int64_t nf[2];
    int32_t minmax[2];
    double dt;
    int flag;
  };
  Pinned* h_pin = nullptr;
  // perk_adapt_commit_dt: the new state whose step size the partition's readback brings along
  const double* pending_dt_U = nullptr;
  bool dt_folded = false;
  std::string err;

  // mesh (host)
  bool has_mesh = false;
  int64_t n_elem = 0, n_if = 0, n_mort = 0;
  double x0 = 0.0, length = 1.0;
  std::vector<int32_t> h_level;
  std::vector<int32_t> h_cells;   // [n_elem][3] (level, ix, iy)
  int n_members = 1;              // ensemble members (independent meshes in one context)
  std::vector<int32_t> h_member;  // [n_elem] member of each element
  std::vector<double> cur_dts;    // dt of each member as last set on the device
  std::vector<int4> h_if, h_mort;

  // device copy of the leaves (level, ix, iy, member) and whether they are in member-major
  // Morton order (then AMR plans and the new mesh's connectivity are computed on the device);
  // host_stale: the host copies (h_cells, h_level, h_member, h_if, h_mort) lag a device-built mesh
  DevBuf<int4> d_cells, d_newcells;
  DevBuf<unsigned long long> d_key;
  DevBuf<int32_t> d_des, d_off, d_cnt_if, d_cnt_mort, d_off_if, d_off_mort;
  DevBuf<int64_t> d_info;
  bool mesh_morton = false;
  bool host_stale = false;

  // pending AMR plan (perk_adapt_plan -> perk_adapt_commit)
  bool has_plan = false;
  bool plan_device = false;          // planned on the device (plan_n_new cells)
  int64_t plan_n_new = 0;
  bool plan_identity = false;        // the plan changes no cell
  std::vector<int32_t> plan_cells;   // new leaves [n][3]
  std::vector<int32_t> plan_member;  // their ensemble members
  std::vector<int32_t> plan_map;     // [n][5] transfer records
  DevBuf<int32_t> d_map;
  DevBuf<double> d_eta;

  // adjoint work space
  DevBuf<double> d_surf_d, d_Kall, d_g, d_lamK1, d_lamKa, d_lamKb;
  DevBuf<unsigned long long> d_rctl;   // item counters of the fused reverse stages
  // elements per block of the volume kernel (perk_autotune_volume)
  int vol_epb = VOL_EPB_DEFAULT;
  // second stream of the reverse sweep: face adjoints run beside the volume adjoint
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // Navier-Stokes (BR1) work space
  DevBuf<double> d_wsurf, d_q, d_vsurf;
  bool viscous() const { return prob.equations == PERK_NAVIER_STOKES; }
  bool differentiable() const {
    return prob.shock_capturing == PERK_SHOCK_OFF && prob.surface_flux != PERK_SURFACE_HLLE && !pattern_mode;
  }
  double kappa() const { return prob.mu * prob.gamma / ((prob.gamma - 1.0) * prob.prandtl); }
  int32_t lmin = 0, lmax = 0;

  // tableau; weights of the final update U + dt (w_b1 K_1 + w_bp K_{S-1} + w_bs K_S)
  bool has_tab = false;
  int order = 2, S = 0, R = 0;
  // stage pattern: src[r*S + i] = the stage (0-based) member r couples to at stage i besides K_1;
  // stage_minmem[i] = the coarsest member active at stage i (members are nested);
  // pattern_mode: some member does not couple to K_{i-1}, so the step keeps every stage
  std::vector<int32_t> src;
  int32_t stage_minmem[MAX_S] = {};
  bool pattern_mode = false;
  DevBuf<double> d_Kpat;
  double w_b1 = 0.0, w_bp = 0.0, w_bs = 1.0;
  int32_t E[MAX_R] = {};
  std::vector<double> c, a;  // c[S], a[R*S]

  // partition results (host copies)
  bool partitioned = false;
  int part_S = 0;
  int64_t act_el[MAX_S] = {}, act_if[MAX_S] = {}, act_mort[MAX_S] = {};
  // per stage, the prefixes of the one-level halo of the active members (BR1 gradients)
  int64_t halo_el[MAX_S] = {}, halo_if[MAX_S] = {}, halo_mort[MAX_S] = {};

  // device buffers
  DevBuf<int32_t> d_level, d_method, d_elem_sorted, d_E, d_minmax, d_member, d_member_lmax;
  DevBuf<int4> d_if_raw, d_mort_raw, d_if_sorted, d_mort_sorted;
  DevBuf<int64_t> d_counts;
  DevBuf<double> d_surf, d_K1, d_Ka, d_Kb, d_dt, d_block_min, d_dt_out;
  DevBuf<StageCoef> d_coef;
  DevBuf<int> d_flag;
  DevBuf<double> d_logtab;   // table of the volume kernel's logarithm

  // one launch per stage (k_stage: faces and volume together; perk_set_stage_fusion) where the
  // equations allow it; its work counters and per-face stamps.  On by default: on GB300 it is the
  // faster form (KH 3,904 cells 0.603 against 0.618 ms/step, 114,688 cells 5.53 against 5.58)
  bool fuse_stage = true;
  // one launch per step (k_step: all stages' items dealt in order, element progress stamps), where
  // one launch per stage would be used and the step has at most STEP_MAX_S stages
  bool fuse_step = false;
  DevBuf<unsigned long long> d_ctl, d_stamp, d_prog;   // d_prog: element progress of the one-launch step
  // (Navier-Stokes: the inviscid face and volume terms in one launch, BR1's launches after it)
  bool stage_fused() const { return fuse_stage && prob.shock_capturing == PERK_SHOCK_OFF; }
  bool step_fused() const { return fuse_step && stage_fused() && !viscous() && !pattern_mode && S <= STEP_MAX_S; }

  // graphs of the stage-storing step and of the reverse step, keyed by their arguments (valid
  // flags cleared with the step graph's)
  cudaGraphExec_t graph_store = nullptr, graph_rev = nullptr;
  bool store_valid = false, rev_valid = false;
  const void* store_key[2] = {nullptr, nullptr};
  const void* rev_key[4] = {nullptr, nullptr, nullptr, nullptr};
  double rev_dt = 0.0;
  bool rev_recompute = false;

  // graph of one step (graph_valid: matches the current mesh, tableau and buffers)
  cudaGraphExec_t graph = nullptr;
  bool graph_valid = false;
  double* graph_U = nullptr;

  // caller-bound workspace (perk_bind_workspace): base, size and the cells its layout serves
  char* ws_base = nullptr;
  size_t ws_bytes = 0;
  int64_t ws_cells = 0;

  perk_counters counters{};
};

namespace {

thread_local std::string g_err;  // message of the last failed context-free call on this thread

perk_status fail(perk_ctx* ctx, perk_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx)
    ctx->err = buf;
  else
    g_err = buf;
  return s;
}

#define PERK_CUDA(ctx, call)                                                                        \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? PERK_E_OOM : PERK_E_CUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                               \
  } while (0)

// marks the step graph stale; the executable graph is kept for an in-place update
void drop_graph(perk_ctx* ctx) {
  ctx->graph_valid = false;
  ctx->store_valid = false;
  ctx->rev_valid = false;
}

void destroy_graph(perk_ctx* ctx) {
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  if (ctx->graph_store) cudaGraphExecDestroy(ctx->graph_store);
  if (ctx->graph_rev) cudaGraphExecDestroy(ctx->graph_rev);
  ctx->graph = ctx->graph_store = ctx->graph_rev = nullptr;
  drop_graph(ctx);
  ctx->graph_U = nullptr;
}

// ---- device buffers and the caller-bound workspace ----

// Every device buffer of the context.
template <class F>
void for_each_buffer(perk_ctx* c, F&& f) {
  f(c->d_level); f(c->d_member); f(c->d_member_lmax); f(c->d_method); f(c->d_elem_sorted); f(c->d_E);
  f(c->d_minmax); f(c->d_if_raw); f(c->d_mort_raw); f(c->d_if_sorted); f(c->d_mort_sorted); f(c->d_counts);
  f(c->d_surf); f(c->d_K1); f(c->d_Ka); f(c->d_Kb); f(c->d_dt); f(c->d_block_min); f(c->d_dt_out); f(c->d_coef);
  f(c->d_flag); f(c->d_logtab); f(c->d_map); f(c->d_eta); f(c->d_surf_d); f(c->d_Kall); f(c->d_Kpat); f(c->d_g);
  f(c->d_lamK1); f(c->d_lamKa); f(c->d_lamKb); f(c->d_rctl); f(c->d_wsurf); f(c->d_q); f(c->d_vsurf);
  f(c->d_cells); f(c->d_newcells); f(c->d_key); f(c->d_des); f(c->d_off); f(c->d_cnt_if); f(c->d_cnt_mort);
  f(c->d_off_if); f(c->d_off_mort); f(c->d_info); f(c->d_ctl); f(c->d_stamp); f(c->d_prog);
}

// The buffers a caller-bound workspace holds, in layout order, with their sizes (elements of
// their type) for meshes of up to `cells` cells: everything the mesh, the partition, the
// step's stages, the step size and an AMR cycle use.  A mesh has at most 2 interfaces and 2
// mortars per cell (four faces per cell; an interface takes two of them, a mortar three).
// The derivative entry points keep allocating their own work arrays.
template <class F>
void for_each_workspace_buffer(perk_ctx* c, int64_t cells, F&& f) {
  const size_t n = (size_t)std::max<int64_t>(cells, 1);
  f(c->d_surf, n * ELEM); f(c->d_K1, n * ELEM); f(c->d_Ka, n * ELEM); f(c->d_Kb, n * ELEM);
  if (c->pattern_mode) f(c->d_Kpat, n * ELEM * (size_t)c->S);
  if (c->viscous()) {
    f(c->d_wsurf, n * 64); f(c->d_q, n * 128); f(c->d_vsurf, n * 64);
  }
  f(c->d_eta, n); f(c->d_dt, n); f(c->d_block_min, std::max<size_t>(n, DT_MAX_BLOCKS)); f(c->d_dt_out, (size_t)1);
  f(c->d_coef, (size_t)MAX_S * MAX_R); f(c->d_counts, (size_t)6 * MAX_S); f(c->d_logtab, (size_t)2 * LOG_TABLE_SIZE);
  f(c->d_if_raw, 2 * n); f(c->d_if_sorted, 2 * n); f(c->d_mort_raw, 2 * n); f(c->d_mort_sorted, 2 * n);
  f(c->d_level, n); f(c->d_method, n); f(c->d_elem_sorted, n); f(c->d_member, n); f(c->d_member_lmax, n);
  f(c->d_map, 5 * n); f(c->d_E, (size_t)MAX_S); f(c->d_minmax, (size_t)2); f(c->d_flag, (size_t)1);
  f(c->d_cells, n); f(c->d_newcells, n); f(c->d_key, n); f(c->d_des, n); f(c->d_off, n + 1);
  f(c->d_cnt_if, n); f(c->d_cnt_mort, n); f(c->d_off_if, n); f(c->d_off_mort, n); f(c->d_info, (size_t)8);
  f(c->d_ctl, (size_t)MAX_S + 1); f(c->d_stamp, 4 * n); f(c->d_prog, n);
}

// a mesh-sized buffer for n entries: a quarter of headroom when the library allocates it (the
// mesh grows over a run), the exact size from a bound workspace (carved for its cell count)
template <class T>
cudaError_t grow(DevBuf<T>& b, size_t n) {
  if (n <= b.cap && b.p) return cudaSuccess;
  return b.ext ? b.ensure(n) : b.ensure(n + n / 4);
}

constexpr size_t WS_ALIGN = 256;
inline size_t ws_align(size_t off) { return (off + WS_ALIGN - 1) / WS_ALIGN * WS_ALIGN; }

// bytes of the workspace layout for meshes of up to `cells` cells
size_t workspace_layout_bytes(perk_ctx* c, int64_t cells) {
  size_t off = 0;
  for_each_workspace_buffer(c, cells, [&](auto& b, size_t count) {
    off = ws_align(off) + count * sizeof(*b.p);
  });
  return off;
}

struct CellKey {
  int64_t v;
  bool operator==(const CellKey& o) const { return v == o.v; }
};
struct CellHash {
  size_t operator()(const CellKey& k) const { return std::hash<int64_t>()(k.v); }
};
// member (16 bits) | level (5 bits) | ix (21 bits) | iy (21 bits)
inline CellKey key_of(int m, int l, int64_t ix, int64_t iy) {
  return CellKey{((int64_t)m << 47) | ((int64_t)l << 42) | (ix << 21) | iy};
}
constexpr int MAX_LEVEL = 20;
constexpr int MAX_MEMBERS = 65535;

// Morton key of a leaf's lower-left corner at resolution lmax (bits interleaved x, y)
uint64_t morton_key(int l, int64_t ix, int64_t iy, int lmax) {
  const uint64_t X = (uint64_t)ix << (lmax - l), Y = (uint64_t)iy << (lmax - l);
  uint64_t z = 0;
  for (int b = 0; b < 31; ++b) z |= ((X >> b) & 1ull) << (2 * b) | ((Y >> b) & 1ull) << (2 * b + 1);
  return z;
}

// Open-addressing hash table from cell keys to int32 values (linear probing,
// capacity a power of two at least twice the number of entries).
class FlatMap {
 public:
  explicit FlatMap(size_t n) {
    size_t cap = 16;
    while (cap < 2 * n + 2) cap <<= 1;
    keys_.assign(cap, kEmpty);
    vals_.resize(cap);
    mask_ = cap - 1;
  }
  // inserts (key, v) unless present; returns false if the key was present
  bool insert(int64_t key, int32_t v) {
    size_t h = slot(key);
    while (keys_[h] != kEmpty) {
      if (keys_[h] == key) return false;
      h = (h + 1) & mask_;
    }
    keys_[h] = key;
    vals_[h] = v;
    return true;
  }
  int32_t find(int64_t key) const {
    size_t h = slot(key);
    while (keys_[h] != kEmpty) {
      if (keys_[h] == key) return vals_[h];
      h = (h + 1) & mask_;
    }
    return -1;
  }
  int32_t* find_ptr(int64_t key) {
    size_t h = slot(key);
    while (keys_[h] != kEmpty) {
      if (keys_[h] == key) return &vals_[h];
      h = (h + 1) & mask_;
    }
    return nullptr;
  }

 private:
  static constexpr int64_t kEmpty = -1;
  size_t slot(int64_t key) const {
    uint64_t z = (uint64_t)key + 0x9E3779B97F4A7C15ull;   // splitmix64 finaliser
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return (size_t)(z ^ (z >> 31)) & mask_;
  }
  std::vector<int64_t> keys_;
  std::vector<int32_t> vals_;
  size_t mask_ = 0;
};

// Interfaces and mortars of a periodic, 2:1-balanced leaf list by a walk over
// each leaf's four face neighbourhoods in the implicit quadtree.
perk_status build_connectivity(perk_ctx* ctx, int64_t n, const int32_t* cells, const int32_t* member,
                               std::vector<int4>& ifs, std::vector<int4>& morts) {
  FlatMap leaf((size_t)n);
  int n_members = 1;
  int lmax = 0;
  for (int64_t e = 0; e < n; ++e) {
    const int l = cells[3 * e], ix = cells[3 * e + 1], iy = cells[3 * e + 2];
    const int m = member ? member[e] : 0;
    if (l < 0 || l > MAX_LEVEL) return fail(ctx, PERK_E_INVALID_ARG, "cell %lld: level %d out of range", (long long)e, l);
    if (m < 0 || m >= MAX_MEMBERS) return fail(ctx, PERK_E_INVALID_ARG, "cell %lld: member out of range", (long long)e);
    n_members = std::max(n_members, m + 1);
    lmax = std::max(lmax, l);
    const int64_t side = (int64_t)1 << l;
    if (ix < 0 || iy < 0 || ix >= side || iy >= side)
      return fail(ctx, PERK_E_INVALID_ARG, "cell %lld: index outside level %d", (long long)e, l);
    if (!leaf.insert(key_of(m, l, ix, iy).v, (int32_t)e))
      return fail(ctx, PERK_E_INVALID_ARG, "cell %lld duplicated", (long long)e);
  }
  // exact tiling of every member's square: the cells' Morton intervals (at the finest
  // level) must follow each other without gap or overlap from 0 to 4^lmax
  {
    std::vector<std::pair<std::pair<int32_t, uint64_t>, uint64_t>> iv((size_t)n);
    for (int64_t e = 0; e < n; ++e) {
      const int l = cells[3 * e];
      const uint64_t z = morton_key(l, cells[3 * e + 1], cells[3 * e + 2], lmax);
      iv[e] = {{member ? member[e] : 0, z}, z + (1ull << (2 * (lmax - l)))};
    }
    if (!std::is_sorted(iv.begin(), iv.end())) std::sort(iv.begin(), iv.end());
    int32_t cur_m = -1;
    uint64_t next = 0;
    for (const auto& q : iv) {
      if (q.first.first != cur_m) {
        if (cur_m >= 0 && next != (1ull << (2 * lmax)))
          return fail(ctx, PERK_E_INVALID_ARG, "cells of member %d do not tile the domain", cur_m);
        if (q.first.first != cur_m + 1 || q.first.second != 0)
          return fail(ctx, PERK_E_INVALID_ARG, "cells of member %d do not tile the domain", q.first.first);
        cur_m = q.first.first;
        next = 0;
      }
      if (q.first.second != next) return fail(ctx, PERK_E_INVALID_ARG, "cells of member %d overlap or leave a gap", cur_m);
      next = q.second;
    }
    if (next != (1ull << (2 * lmax)) || cur_m + 1 != n_members)
      return fail(ctx, PERK_E_INVALID_ARG, "cells do not tile the domain");
  }
  for (int64_t e = 0; e < n; ++e) {
    const int l = cells[3 * e];
    const int64_t ix = cells[3 * e + 1], iy = cells[3 * e + 2];
    const int mb = member ? member[e] : 0;
    auto find = [&](int ll, int64_t x, int64_t y) -> int32_t {
      if (ll < 0 || ll > MAX_LEVEL) return -1;
      return leaf.find(key_of(mb, ll, x, y).v);
    };
    const int64_t side = (int64_t)1 << l;
    for (int dir = 0; dir < 2; ++dir) {
      // +dir neighbour region (same level)
      const int64_t px = dir == 0 ? (ix + 1) % side : ix;
      const int64_t py = dir == 1 ? (iy + 1) % side : iy;
      const int32_t same = find(l, px, py);
      if (same >= 0) {
        ifs.push_back(make_int4((int)e, same, dir, 0));
      } else if (l > 0 && find(l - 1, px >> 1, py >> 1) >= 0) {
        // this leaf is the small side of a mortar whose large side is the +dir neighbour: built there
      } else {
        // the +dir region must be refined once: its two children along the face
        const int64_t cx0 = 2 * px, cy0 = 2 * py;
        const int32_t s0 = find(l + 1, cx0, cy0);
        const int32_t s1 = find(l + 1, dir == 0 ? cx0 : cx0 + 1, dir == 0 ? cy0 + 1 : cy0);
        if (s0 < 0 || s1 < 0) return fail(ctx, PERK_E_INVALID_ARG, "mesh not 2:1 balanced at cell %lld", (long long)e);
        morts.push_back(make_int4((int)e, s0, s1, dir | (0 << 1)));
      }
      // -dir neighbour region: only detect mortars with this leaf as the large (right) side
      const int64_t mx = dir == 0 ? (ix + side - 1) % side : ix;
      const int64_t my = dir == 1 ? (iy + side - 1) % side : iy;
      if (find(l, mx, my) >= 0) continue;                         // interface, built from the other side
      if (l > 0 && find(l - 1, mx >> 1, my >> 1) >= 0) continue;  // small side of a mortar
      const int64_t cx0 = dir == 0 ? 2 * mx + 1 : 2 * mx, cy0 = dir == 0 ? 2 * my : 2 * my + 1;
      const int32_t s0 = find(l + 1, cx0, cy0);
      const int32_t s1 = find(l + 1, dir == 0 ? cx0 : cx0 + 1, dir == 0 ? cy0 + 1 : cy0);
      if (s0 < 0 || s1 < 0) return fail(ctx, PERK_E_INVALID_ARG, "mesh not 2:1 balanced at cell %lld", (long long)e);
      morts.push_back(make_int4((int)e, s0, s1, dir | (1 << 1)));
    }
  }
  return PERK_OK;
}

// Level partition on the device and its per-stage counts on the host.  device_faces: the
// interface and mortar counts of the mesh are on the device (d_info[2], d_info[3], written by the
// device connectivity build) and come back with the partition's counts.
perk_status run_partition(perk_ctx* ctx, bool device_faces = false) {
  if (!ctx->has_mesh) return fail(ctx, PERK_E_NOT_READY, "no mesh");
  int R = 1, S = 1;
  int32_t minmem[MAX_S] = {0};
  if (ctx->has_tab) {
    R = ctx->R;
    S = ctx->S;
    std::copy(ctx->stage_minmem, ctx->stage_minmem + MAX_S, minmem);
  }
  PERK_CUDA(ctx, ctx->d_E.ensure(MAX_S));
  PERK_CUDA(ctx, cudaMemcpyAsync(ctx->d_E.p, minmem, sizeof(int32_t) * MAX_S, cudaMemcpyHostToDevice, ctx->stream));
  PERK_CUDA(ctx, launch_partition(ctx->stream, ctx->n_elem, ctx->n_if, ctx->n_mort, ctx->d_level.p, ctx->d_if_raw.p,
                                  ctx->d_mort_raw.p, R, S, ctx->d_E.p, ctx->n_members > 1 ? ctx->d_member.p : nullptr,
                                  ctx->n_members, ctx->d_member_lmax.p, ctx->d_method.p, ctx->d_elem_sorted.p,
                                  ctx->d_if_sorted.p, ctx->d_mort_sorted.p, ctx->d_counts.p, ctx->d_minmax.p, 2,
                                  device_faces ? ctx->d_info.p + 2 : nullptr));
  perk_ctx::Pinned* pin = ctx->h_pin;
  const int64_t* counts = pin->counts;
  const int32_t* mm = pin->minmax;
  const int64_t* nf = pin->nf;
  pin->nf[0] = ctx->n_if;
  pin->nf[1] = ctx->n_mort;
  PERK_CUDA(ctx, cudaMemcpyAsync(pin->counts, ctx->d_counts.p, sizeof pin->counts, cudaMemcpyDeviceToHost,
                                 ctx->stream));
  PERK_CUDA(ctx, cudaMemcpyAsync(pin->minmax, ctx->d_minmax.p, sizeof pin->minmax, cudaMemcpyDeviceToHost,
                                 ctx->stream));
  if (device_faces)
    PERK_CUDA(ctx, cudaMemcpyAsync(pin->nf, ctx->d_info.p + 2, sizeof pin->nf, cudaMemcpyDeviceToHost, ctx->stream));
  if (ctx->pending_dt_U) {
    // the step size of the new state, read back with the counts (one wait for both)
    const int nb = (int)std::min<int64_t>(DT_MAX_BLOCKS, (ctx->n_elem * NODES + DT_THREADS - 1) / DT_THREADS);
    if (ctx->d_block_min.cap < (size_t)nb) return fail(ctx, PERK_E_INVALID_ARG, "internal: step-size scratch too small");
    PERK_CUDA(ctx, launch_dt(ctx->stream, ctx->n_elem, ctx->pending_dt_U, ctx->d_level.p, ctx->length, ctx->ops.gamma,
                             ctx->d_block_min.p, nb, ctx->d_dt_out.p));
    PERK_CUDA(ctx, cudaMemcpyAsync(&pin->dt, ctx->d_dt_out.p, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    ctx->dt_folded = true;
  }
  PERK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->n_if = nf[0];
  ctx->n_mort = nf[1];
  for (int i = 0; i < MAX_S; ++i) {
    ctx->act_el[i] = i < S ? counts[i] : 0;
    ctx->act_if[i] = i < S ? counts[MAX_S + i] : 0;
    ctx->act_mort[i] = i < S ? counts[2 * MAX_S + i] : 0;
    ctx->halo_el[i] = i < S ? counts[3 * MAX_S + i] : 0;
    ctx->halo_if[i] = i < S ? counts[4 * MAX_S + i] : 0;
    ctx->halo_mort[i] = i < S ? counts[5 * MAX_S + i] : 0;
  }
  ctx->lmin = mm[0];
  ctx->lmax = mm[1];
  ctx->part_S = S;
  ctx->partitioned = true;
  drop_graph(ctx);
  return PERK_OK;
}

// device dt of every member: dts[m] (per member) or the same dt for all; uploads only on change
perk_status set_dts(perk_ctx* ctx, const double* dts, double dt) {
  bool changed = false;
  for (int m = 0; m < ctx->n_members; ++m) {
    const double v = dts ? dts[m] : dt;
    if (!std::isfinite(v) || !(v > 0.0)) return fail(ctx, PERK_E_INVALID_ARG, "bad dt of member %d", m);
    if (!(ctx->cur_dts[m] == v)) {
      ctx->cur_dts[m] = v;
      changed = true;
    }
  }
  if (!changed) return PERK_OK;
  if (ctx->n_members == 1) {
    PERK_CUDA(ctx, launch_set_scalar(ctx->stream, ctx->d_dt.p, ctx->cur_dts[0]));
  } else {
    // pageable source: the call returns once the values are staged, so the vector may change afterwards
    PERK_CUDA(ctx, cudaMemcpyAsync(ctx->d_dt.p, ctx->cur_dts.data(), ctx->n_members * sizeof(double),
                                   cudaMemcpyHostToDevice, ctx->stream));
  }
  return PERK_OK;
}

// CUDA events around individual launches (perk_step_profiled)
struct LaunchTimer {
  std::vector<cudaEvent_t> start, stop;
  std::vector<int> kind;
  cudaError_t begin(cudaStream_t st) {
    cudaEvent_t a;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    start.push_back(a);
    return cudaEventRecord(a, st);
  }
  cudaError_t end(cudaStream_t st, int k) {
    cudaEvent_t b;
    cudaError_t e = cudaEventCreate(&b);
    if (e != cudaSuccess) return e;
    stop.push_back(b);
    kind.push_back(k);
    return cudaEventRecord(b, st);
  }
  ~LaunchTimer() {
    for (auto e : start) cudaEventDestroy(e);
    for (auto e : stop) cudaEventDestroy(e);
  }
};

#define TIMED(ctx, timer, st, kind, call)            \
  do {                                               \
    if (timer) PERK_CUDA(ctx, (timer)->begin(st));   \
    PERK_CUDA(ctx, call);                            \
    if (timer) PERK_CUDA(ctx, (timer)->end(st, kind)); \
  } while (0)

perk_status set_mesh(perk_ctx* ctx, int64_t n_cells, const int32_t* cells, const int32_t* member, double x0,
                     double length) {
  if (ctx->ws_base && n_cells > ctx->ws_cells)
    return fail(ctx, PERK_E_OOM,
                "the bound workspace serves meshes of up to %lld cells, this one has %lld: bind a larger one "
                "(perk_workspace_bytes)", (long long)ctx->ws_cells, (long long)n_cells);
  std::vector<int4> ifs, morts;
  ifs.reserve((size_t)n_cells * 2);
  perk_status s = build_connectivity(ctx, n_cells, cells, member, ifs, morts);
  if (s != PERK_OK) return s;
  drop_graph(ctx);
  int n_members = 1;
  ctx->h_member.assign(n_cells, 0);
  if (member)
    for (int64_t e = 0; e < n_cells; ++e) {
      ctx->h_member[e] = member[e];
      n_members = std::max(n_members, member[e] + 1);
    }
  if (n_members != ctx->n_members || (int)ctx->cur_dts.size() != n_members) {
    ctx->n_members = n_members;
    ctx->cur_dts.assign(n_members, NAN);
  }
  PERK_CUDA(ctx, ctx->d_dt.ensure((size_t)n_members));
  PERK_CUDA(ctx, ctx->d_member_lmax.ensure((size_t)n_members));
  PERK_CUDA(ctx, ctx->d_member.ensure((size_t)n_cells));
  PERK_CUDA(ctx, cudaMemcpyAsync(ctx->d_member.p, ctx->h_member.data(), n_cells * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, ctx->stream));
  ctx->n_elem = n_cells;
  ctx->n_if = (int64_t)ifs.size();
  ctx->n_mort = (int64_t)morts.size();
  ctx->x0 = x0;
  ctx->length = length;
  ctx->h_cells.assign(cells, cells + 3 * n_cells);
  ctx->h_level.resize(n_cells);
  for (int64_t e = 0; e < n_cells; ++e) ctx->h_level[e] = cells[3 * e];
  ctx->h_if = std::move(ifs);
  ctx->h_mort = std::move(morts);
  const size_t ne = (size_t)n_cells;
  PERK_CUDA(ctx, ctx->d_level.ensure(ne));
  PERK_CUDA(ctx, ctx->d_method.ensure(ne));
  PERK_CUDA(ctx, ctx->d_elem_sorted.ensure(ne));
  PERK_CUDA(ctx, ctx->d_if_raw.ensure(ctx->h_if.size()));
  PERK_CUDA(ctx, ctx->d_if_sorted.ensure(ctx->h_if.size()));
  PERK_CUDA(ctx, ctx->d_mort_raw.ensure(ctx->h_mort.size()));
  PERK_CUDA(ctx, ctx->d_mort_sorted.ensure(ctx->h_mort.size()));
  PERK_CUDA(ctx, ctx->d_surf.ensure(ne * ELEM));
  PERK_CUDA(ctx, ctx->d_K1.ensure(ne * ELEM));
  PERK_CUDA(ctx, ctx->d_Ka.ensure(ne * ELEM));
  PERK_CUDA(ctx, ctx->d_Kb.ensure(ne * ELEM));
  PERK_CUDA(ctx, ctx->d_eta.ensure(ne));
  if (ctx->viscous()) {
    PERK_CUDA(ctx, ctx->d_wsurf.ensure(ne * 64));
    PERK_CUDA(ctx, ctx->d_q.ensure(ne * 128));   // BR1 viscous fluxes [e][2 directions][4][16]
    PERK_CUDA(ctx, ctx->d_vsurf.ensure(ne * 64));
  }
  // per-block minima of the step-size reduction: its grid is capped at DT_MAX_BLOCKS blocks
  PERK_CUDA(ctx, ctx->d_block_min.ensure((size_t)DT_MAX_BLOCKS));
  // face stamps of the fused stage kernel: zero is older than any launch
  PERK_CUDA(ctx, ctx->d_stamp.ensure(4 * ne));
  PERK_CUDA(ctx, cudaMemsetAsync(ctx->d_stamp.p, 0, 4 * ne * sizeof(unsigned long long), ctx->stream));
  PERK_CUDA(ctx, ctx->d_prog.ensure(ne));
  PERK_CUDA(ctx, cudaMemsetAsync(ctx->d_prog.p, 0, ne * sizeof(unsigned long long), ctx->stream));
  PERK_CUDA(ctx, cudaMemcpyAsync(ctx->d_level.p, ctx->h_level.data(), ne * sizeof(int32_t), cudaMemcpyHostToDevice,
                                 ctx->stream));
  if (!ctx->h_if.empty())
    PERK_CUDA(ctx, cudaMemcpyAsync(ctx->d_if_raw.p, ctx->h_if.data(), ctx->h_if.size() * sizeof(int4),
                                   cudaMemcpyHostToDevice, ctx->stream));
  if (!ctx->h_mort.empty())
    PERK_CUDA(ctx, cudaMemcpyAsync(ctx->d_mort_raw.p, ctx->h_mort.data(), ctx->h_mort.size() * sizeof(int4),
                                   cudaMemcpyHostToDevice, ctx->stream));
  {
    // device copy of the leaves; member-major Morton order enables the device AMR path
    std::vector<int4> c4(ne);
    bool sorted = true;
    uint64_t prev = 0;
    for (size_t e = 0; e < ne; ++e) {
      const int m = member ? member[e] : 0;
      c4[e] = make_int4(cells[3 * e], cells[3 * e + 1], cells[3 * e + 2], m);
      const uint64_t key = ((uint64_t)m << 40) | morton_key(cells[3 * e], cells[3 * e + 1], cells[3 * e + 2], MAX_LEVEL);
      if (e > 0 && key <= prev) sorted = false;
      prev = key;
    }
    PERK_CUDA(ctx, ctx->d_cells.ensure(ne));
    PERK_CUDA(ctx, cudaMemcpyAsync(ctx->d_cells.p, c4.data(), ne * sizeof(int4), cudaMemcpyHostToDevice, ctx->stream));
    ctx->mesh_morton = sorted;
    ctx->host_stale = false;
  }
  ctx->has_mesh = true;
  return run_partition(ctx);
}

// Host copies of a mesh the device built (AMR on the device): leaves, levels, members, face records.
perk_status sync_host_mesh(perk_ctx* ctx) {
  if (!ctx->host_stale) return PERK_OK;
  const int64_t n = ctx->n_elem;
  std::vector<int4> c4((size_t)n);
  ctx->h_if.resize((size_t)ctx->n_if);
  ctx->h_mort.resize((size_t)ctx->n_mort);
  PERK_CUDA(ctx, cudaMemcpyAsync(c4.data(), ctx->d_cells.p, n * sizeof(int4), cudaMemcpyDeviceToHost, ctx->stream));
  if (ctx->n_if)
    PERK_CUDA(ctx, cudaMemcpyAsync(ctx->h_if.data(), ctx->d_if_raw.p, ctx->n_if * sizeof(int4), cudaMemcpyDeviceToHost,
                                   ctx->stream));
  if (ctx->n_mort)
    PERK_CUDA(ctx, cudaMemcpyAsync(ctx->h_mort.data(), ctx->d_mort_raw.p, ctx->n_mort * sizeof(int4),
                                   cudaMemcpyDeviceToHost, ctx->stream));
  PERK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->h_cells.resize(3 * (size_t)n);
  ctx->h_level.resize((size_t)n);
  ctx->h_member.resize((size_t)n);
  for (int64_t e = 0; e < n; ++e) {
    ctx->h_cells[3 * e] = c4[e].x;
    ctx->h_cells[3 * e + 1] = c4[e].y;
    ctx->h_cells[3 * e + 2] = c4[e].z;
    ctx->h_level[e] = c4[e].x;
    ctx->h_member[e] = c4[e].w;
  }
  ctx->host_stale = false;
  return PERK_OK;
}


// Desired levels raised to the least fixed point of the sibling rule (a cell
// coarsens only with all three siblings, all leaves that want to coarsen) and
// the 2:1 rule across faces of the current mesh.
void balance_levels(const perk_ctx* ctx, std::vector<int32_t>& d) {
  const int64_t n = ctx->n_elem;
  const int32_t* c = ctx->h_cells.data();
  // sibling groups: members of the same parent, as a list per parent (group id by hash)
  const int32_t* mb = ctx->h_member.data();
  FlatMap gid((size_t)n);
  std::vector<int32_t> group_of(n, -1), gcount, gfirst;
  std::vector<int32_t> gmembers;            // 4 slots per group
  for (int64_t e = 0; e < n; ++e) {
    if (c[3 * e] == 0) continue;
    const int64_t k = key_of(mb[e], c[3 * e], c[3 * e + 1] >> 1, c[3 * e + 2] >> 1).v;
    int32_t g = gid.find(k);
    if (g < 0) {
      g = (int32_t)gcount.size();
      gid.insert(k, g);
      gcount.push_back(0);
      gmembers.insert(gmembers.end(), 4, -1);
    }
    if (gcount[g] < 4) gmembers[4 * g + gcount[g]] = (int32_t)e;
    gcount[g] += 1;
    group_of[e] = g;
  }
  std::vector<std::pair<int32_t, int32_t>> pairs;
  for (const int4& f : ctx->h_if) pairs.emplace_back(f.x, f.y);
  for (const int4& m : ctx->h_mort) {
    pairs.emplace_back(m.x, m.y);
    pairs.emplace_back(m.x, m.z);
  }
  bool changed = true;
  while (changed) {
    changed = false;
    for (int64_t e = 0; e < n; ++e) {
      if (d[e] >= c[3 * e]) continue;
      const int32_t g = group_of[e];
      bool ok = g >= 0 && gcount[g] == 4;
      if (ok)
        for (int q = 0; q < 4; ++q) ok = ok && d[gmembers[4 * g + q]] < c[3 * gmembers[4 * g + q]];
      if (!ok) {
        if (g < 0) {
          d[e] = c[3 * e];
          changed = true;
          continue;
        }
        for (int q = 0; q < 4 && q < gcount[g]; ++q) {
          const int32_t m = gmembers[4 * g + q];
          if (d[m] < c[3 * m]) {
            d[m] = c[3 * m];
            changed = true;
          }
        }
      }
    }
    for (const auto& pr : pairs) {
      const int32_t a = pr.first, b = pr.second;
      if (d[a] > d[b] + 1) {
        d[b] = d[a] - 1;
        changed = true;
      } else if (d[b] > d[a] + 1) {
        d[a] = d[b] - 1;
        changed = true;
      }
    }
  }
}

// the stage launches of one step on stream st (also used under graph capture)
perk_status enqueue_step(perk_ctx* ctx, cudaStream_t st, double* d_U, LaunchTimer* timer = nullptr) {
  const int S = ctx->S;
  const size_t nd = (size_t)ctx->n_elem * ELEM;
  // classic pattern: K_1 has its own buffer and K_2, K_3, ... alternate between two others;
  // a stage pattern keeps every stage (stage i at Kall + i * nd), since a member may couple to
  // any earlier stage it evaluated
  double* Kall = nullptr;
  if (ctx->pattern_mode) {
    // allocated by prepare_step before any capture
    if (!ctx->d_Kpat.p || ctx->d_Kpat.cap < nd * S) return fail(ctx, PERK_E_NOT_READY, "stage storage not prepared");
    Kall = ctx->d_Kpat.p;
  }
  double* Kbuf[3] = {ctx->d_K1.p, ctx->d_Ka.p, ctx->d_Kb.p};
  auto stage_out = [&](int i, int cur) { return Kall ? Kall + (size_t)i * nd : Kbuf[cur]; };
  int prev = 0, cur = 0;
  double* K_before_last = Kall ? Kall + (size_t)(S > 1 ? S - 2 : 0) * nd : nullptr;   // K_{S-1}
  UpdateArgs ua{};
  ua.b1 = ctx->w_b1;
  ua.bp = ctx->w_bp;
  ua.bs = ctx->w_bs;
  ua.U = d_U;
  ua.K1 = Kall ? Kall : ctx->d_K1.p;
  ua.flag = ctx->d_flag.p;
  ua.member = ctx->n_members > 1 ? ctx->d_member.p : nullptr;
  if (ctx->step_fused() && !timer) {
    // one launch for all stages: the same buffers as the stage-by-stage loop below
    StepPlan plan{};
    plan.S = S;
    plan.first[0] = 0;
    for (int i = 0; i < S; ++i) {
      cur = (i == 0) ? 0 : (i % 2 == 1 ? 1 : 2);
      plan.n_if[i] = ctx->act_if[i];
      plan.n_mort[i] = ctx->act_mort[i];
      plan.n_el[i] = ctx->act_el[i];
      plan.first[i + 1] = plan.first[i] + step_stage_items(ctx->act_if[i], ctx->act_mort[i], ctx->act_el[i]);
      plan.K[i] = Kbuf[cur];
      plan.Kp[i] = Kbuf[prev];
      if (i == S - 1) K_before_last = Kbuf[prev];
      prev = cur;
    }
    StageArgs sa{};
    sa.U = d_U;
    sa.K1 = ctx->d_K1.p;
    sa.nd = (int64_t)nd;
    sa.coef = ctx->d_coef.p;
    sa.dt = ctx->d_dt.p;
    sa.member = ua.member;
    UpdateArgs chk = ua;
    chk.Kp = K_before_last;
    PERK_CUDA(ctx, launch_step(st, ctx->ops, plan, ctx->d_if_sorted.p, ctx->d_mort_sorted.p, ctx->d_elem_sorted.p,
                               ctx->d_level.p, ctx->d_method.p, 2.0 / ctx->length, sa, ctx->d_surf.p, chk,
                               ctx->d_logtab.p, ctx->d_ctl.p, ctx->d_stamp.p, ctx->d_prog.p, ctx->d_flag.p));
    ua.Kp = K_before_last;
    ua.stage_ctl = ctx->d_ctl.p;
    PERK_CUDA(ctx, launch_commit(st, ctx->n_elem, ua, Kbuf[cur], ctx->d_dt.p, d_U));
    return PERK_OK;
  }
  for (int i = 0; i < S; ++i) {
    cur = (i == 0) ? 0 : (i % 2 == 1 ? 1 : 2);
    StageArgs sa{};
    sa.U = d_U;
    sa.K1 = Kall ? Kall : ctx->d_K1.p;
    sa.Kp = Kall ? nullptr : Kbuf[prev];
    sa.Kall = Kall;
    sa.nd = (int64_t)nd;
    sa.coef = ctx->d_coef.p + (size_t)i * MAX_R;
    sa.dt = ctx->d_dt.p;
    sa.member = ctx->n_members > 1 ? ctx->d_member.p : nullptr;
    const bool last = (i == S - 1);
    if (last && !Kall) K_before_last = Kbuf[prev];
    UpdateArgs chk = ua;
    chk.Kp = K_before_last;
    const bool visc = ctx->viscous();
    if (ctx->stage_fused()) {
      TIMED(ctx, timer, st, 1,
            launch_stage(st, i, ctx->ops, ctx->act_if[i], ctx->d_if_sorted.p, ctx->act_mort[i], ctx->d_mort_sorted.p,
                         ctx->act_el[i], ctx->d_elem_sorted.p, ctx->d_level.p, ctx->d_method.p, 2.0 / ctx->length,
                         sa, ctx->d_surf.p, stage_out(i, cur), (last && !visc) ? &chk : nullptr, ctx->d_logtab.p,
                         ctx->d_ctl.p, ctx->d_stamp.p, ctx->d_flag.p));
      if (visc)
        TIMED(ctx, timer, st, 3,
              launch_br1(st, Y_COMBINE, ctx->ops, ctx->prob.mu, ctx->kappa(), ctx->halo_if[i], ctx->halo_mort[i],
                         ctx->act_if[i], ctx->act_mort[i], ctx->d_if_sorted.p, ctx->d_mort_sorted.p, ctx->halo_el[i],
                         ctx->act_el[i], ctx->d_elem_sorted.p, ctx->d_level.p, ctx->d_method.p, 2.0 / ctx->length,
                         sa, ctx->d_wsurf.p, ctx->d_q.p, ctx->d_vsurf.p, stage_out(i, cur), last ? &chk : nullptr));
      prev = cur;
      continue;
    }
    TIMED(ctx, timer, st, 0,
          launch_faces(st, Y_COMBINE, ctx->ops, ctx->act_if[i], ctx->d_if_sorted.p, ctx->act_mort[i],
                       ctx->d_mort_sorted.p, ctx->d_method.p, sa, ctx->d_surf.p));
    TIMED(ctx, timer, st, 1,
          launch_volume(st, Y_COMBINE, ctx->ops, ctx->act_el[i], ctx->d_elem_sorted.p, ctx->d_level.p,
                        ctx->d_method.p, 2.0 / ctx->length, sa, ctx->d_surf.p, stage_out(i, cur),
                        (last && !visc) ? &chk : nullptr, ctx->d_logtab.p, ctx->vol_epb));
    if (visc)
      TIMED(ctx, timer, st, 3,
            launch_br1(st, Y_COMBINE, ctx->ops, ctx->prob.mu, ctx->kappa(), ctx->halo_if[i], ctx->halo_mort[i],
                       ctx->act_if[i], ctx->act_mort[i], ctx->d_if_sorted.p, ctx->d_mort_sorted.p, ctx->halo_el[i],
                       ctx->act_el[i],
                       ctx->d_elem_sorted.p, ctx->d_level.p, ctx->d_method.p, 2.0 / ctx->length, sa,
                       ctx->d_wsurf.p, ctx->d_q.p, ctx->d_vsurf.p, stage_out(i, cur), last ? &chk : nullptr));
    prev = cur;
  }
  ua.Kp = K_before_last;
  ua.stage_ctl = ctx->stage_fused() ? ctx->d_ctl.p : nullptr;
  TIMED(ctx, timer, st, 2, launch_commit(st, ctx->n_elem, ua, stage_out(S - 1, cur), ctx->d_dt.p, d_U));
  return PERK_OK;
}

perk_status upload_coef(perk_ctx* ctx) {
  std::vector<StageCoef> coef((size_t)MAX_S * MAX_R, StageCoef{0.0, 0.0, 0, 0});
  for (int i = 1; i < ctx->S; ++i)
    for (int r = 0; r < ctx->R; ++r) {
      const double beta = ctx->a[(size_t)r * ctx->S + i];
      coef[(size_t)i * MAX_R + r] = StageCoef{ctx->c[i] - beta, beta, ctx->src[(size_t)r * ctx->S + i], 0};
    }
  PERK_CUDA(ctx, ctx->d_coef.ensure((size_t)MAX_S * MAX_R));
  PERK_CUDA(ctx, cudaMemcpyAsync(ctx->d_coef.p, coef.data(), coef.size() * sizeof(StageCoef), cudaMemcpyHostToDevice,
                                 ctx->stream));
  PERK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return PERK_OK;
}

}  // namespace

perk_status perk::set_context_free_error(perk_status s, const char* msg) { return fail(nullptr, s, "%s", msg); }

// ---------------------------------------------------------------------------
extern "C" {

perk_status perk_create(const perk_problem* prob, perk_ctx** out) {
  if (!prob || !out) return PERK_E_INVALID_ARG;
  *out = nullptr;
  if (prob->N != 3 || !(prob->gamma > 1.0) || prob->surface_flux < 0 || prob->surface_flux > 3)
    return PERK_E_INVALID_ARG;
  if (prob->shock_capturing < PERK_SHOCK_OFF || prob->shock_capturing > PERK_SHOCK_DENSITY) return PERK_E_INVALID_ARG;
  if (prob->shock_capturing != PERK_SHOCK_OFF && !(prob->alpha_max > 0.0 && prob->alpha_max <= 1.0))
    return PERK_E_INVALID_ARG;
  if (prob->equations != PERK_EULER && prob->equations != PERK_NAVIER_STOKES) return PERK_E_INVALID_ARG;
  if (prob->equations == PERK_NAVIER_STOKES && (!(prob->mu > 0.0) || !(prob->prandtl > 0.0))) return PERK_E_INVALID_ARG;
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) return PERK_E_CUDA;
  perk_ctx* ctx = new perk_ctx();
  ctx->prob = *prob;
  ctx->ops = build_ops(prob->gamma, prob->surface_flux, prob->shock_capturing, prob->alpha_max);
  for_each_buffer(ctx, [ctx](auto& b) { b.allocs = &ctx->counters.device_allocations; });
  device_sm_count();   // cached before any graph capture
  stage_resident_blocks();
  if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&ctx->h_pin), sizeof(perk_ctx::Pinned)) != cudaSuccess ||
      ctx->d_dt.ensure(1) != cudaSuccess || ctx->d_flag.ensure(1) != cudaSuccess ||
      ctx->d_logtab.ensure(2 * LOG_TABLE_SIZE) != cudaSuccess ||
      ctx->d_counts.ensure(6 * MAX_S) != cudaSuccess || ctx->d_minmax.ensure(2) != cudaSuccess ||
      ctx->d_dt_out.ensure(1) != cudaSuccess || ctx->d_ctl.ensure(MAX_S + 1) != cudaSuccess) {
    perk_destroy(ctx);
    return PERK_E_CUDA;
  }
  cudaMemset(ctx->d_flag.p, 0, sizeof(int));
  cudaMemset(ctx->d_ctl.p, 0, (MAX_S + 1) * sizeof(unsigned long long));
  {
    const std::vector<double> t = log_table();
    cudaMemcpy(ctx->d_logtab.p, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    perk_destroy(ctx);
    return PERK_E_CUDA;
  }
  *out = ctx;
  return PERK_OK;
}

void perk_destroy(perk_ctx* ctx) {
  if (!ctx) return;
  destroy_graph(ctx);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->h_pin) cudaFreeHost(ctx->h_pin);
  if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  for_each_buffer(ctx, [](auto& b) { b.release(); });
  delete ctx;
}

const char* perk_last_error(const perk_ctx* ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

perk_status perk_set_stream(perk_ctx* ctx, void* stream) {
  if (!ctx) return PERK_E_INVALID_ARG;
  ctx->stream = (cudaStream_t)stream;
  return PERK_OK;
}

perk_status perk_mesh_upload(perk_ctx* ctx, int64_t n_cells, const int32_t* cells, double x0, double length) {
  if (!ctx) return PERK_E_INVALID_ARG;
  if (n_cells <= 0 || !cells || !(length > 0.0) || n_cells > (int64_t)1 << 30)
    return fail(ctx, PERK_E_INVALID_ARG, "invalid mesh arguments");
  ctx->has_plan = false;
  return set_mesh(ctx, n_cells, cells, nullptr, x0, length);
}

perk_status perk_ensemble_upload(perk_ctx* ctx, int n_members, const int64_t* n_cells, const int32_t* cells, double x0,
                                 double length) {
  if (!ctx) return PERK_E_INVALID_ARG;
  if (n_members < 1 || n_members > MAX_MEMBERS || !n_cells || !cells || !(length > 0.0))
    return fail(ctx, PERK_E_INVALID_ARG, "invalid ensemble arguments");
  std::vector<int32_t> member;
  for (int m = 0; m < n_members; ++m) {
    if (n_cells[m] <= 0) return fail(ctx, PERK_E_INVALID_ARG, "member %d has no cells", m);
    member.insert(member.end(), (size_t)n_cells[m], m);
  }
  if ((int64_t)member.size() > (int64_t)1 << 30) return fail(ctx, PERK_E_INVALID_ARG, "ensemble too large");
  ctx->has_plan = false;
  return set_mesh(ctx, (int64_t)member.size(), cells, member.data(), x0, length);
}

perk_status perk_get_members(const perk_ctx* ctx, int32_t* member, int64_t cap) {
  if (!ctx || !member) return PERK_E_INVALID_ARG;
  if (!ctx->has_mesh) return PERK_E_NOT_READY;
  if (cap < ctx->n_elem) return PERK_E_INVALID_ARG;
  {
    perk_status s = sync_host_mesh(const_cast<perk_ctx*>(ctx));
    if (s != PERK_OK) return s;
  }
  std::copy(ctx->h_member.begin(), ctx->h_member.end(), member);
  return PERK_OK;
}

perk_status perk_mesh_faces(int64_t n_cells, const int32_t* cells, int64_t* n_if, int32_t* ifs, int64_t if_cap,
                            int64_t* n_mort, int32_t* morts, int64_t mort_cap) {
  if (n_cells <= 0 || !cells || !n_if || !n_mort) return PERK_E_INVALID_ARG;
  std::vector<int4> vi, vm;
  perk_status s = build_connectivity(nullptr, n_cells, cells, nullptr, vi, vm);
  if (s != PERK_OK) return s;
  *n_if = (int64_t)vi.size();
  *n_mort = (int64_t)vm.size();
  if (ifs && if_cap >= *n_if)
    for (size_t q = 0; q < vi.size(); ++q) {
      ifs[4 * q] = vi[q].x;
      ifs[4 * q + 1] = vi[q].y;
      ifs[4 * q + 2] = vi[q].z;
      ifs[4 * q + 3] = vi[q].w;
    }
  if (morts && mort_cap >= *n_mort)
    for (size_t q = 0; q < vm.size(); ++q) {
      morts[4 * q] = vm[q].x;
      morts[4 * q + 1] = vm[q].y;
      morts[4 * q + 2] = vm[q].z;
      morts[4 * q + 3] = vm[q].w;
    }
  return PERK_OK;
}

perk_status perk_mesh_query(const perk_ctx* ctx, perk_mesh_info* info) {
  if (!ctx || !info) return PERK_E_INVALID_ARG;
  std::memset(info, 0, sizeof *info);
  if (!ctx->has_mesh) return PERK_E_NOT_READY;
  info->n_elem = ctx->n_elem;
  info->n_interfaces = ctx->n_if;
  info->n_mortars = ctx->n_mort;
  info->level_min = ctx->lmin;
  info->level_max = ctx->lmax;
  info->S = ctx->has_tab ? ctx->S : 0;
  int64_t dof = 0;
  for (int i = 0; i < ctx->part_S && i < 64; ++i) {
    info->active_elements[i] = ctx->act_el[i];
    info->active_interfaces[i] = ctx->act_if[i];
    info->active_mortars[i] = ctx->act_mort[i];
    dof += ctx->act_el[i] * NODES;
  }
  info->dof_stage_updates = ctx->has_tab ? dof : 0;
  info->index_bytes = (int64_t)(ctx->n_elem * 2 * sizeof(int32_t) + ctx->n_if * sizeof(int4) +
                                ctx->n_mort * sizeof(int4));
  return PERK_OK;
}

namespace {
// Eq. PERKCoeffsConstruction: the a_{i,i-1} of a second-order member with e stage evaluations
// from the monomial coefficients alpha[0..e] of its stability polynomial, for the weights
// b_1 = 1 - bs, b_S = bs and abscissae c_i = (i-1)/(2 bs (S-1)); the coefficient of z^{3+j} is
// bs c_{S-1-j} prod_{q=0}^{j} a_{S-q} (1-based stage indices), j = 0..e-3.
// False if a product vanishes or a coefficient is not finite.
bool perk2_member_from_alpha(int S, int e, double bs, const double* alpha, double* ar) {
  for (int i = 0; i < S; ++i) ar[i] = 0.0;
  double prod = 1.0;
  for (int j = 0; j <= e - 3; ++j) {
    const int stage = S - j;                    // 1-based stage whose a_{stage,stage-1} is found
    const double cprev = (double)(stage - 2) / (2.0 * bs * (S - 1));   // c_{stage-1}
    const double den = bs * cprev * prod;
    if (!(den != 0.0)) return false;
    const double v = alpha[3 + j] / den;
    if (!std::isfinite(v)) return false;
    ar[stage - 1] = v;                           // a[r*S + i] = a_{i+1,i}, i = stage - 1
    prod *= v;
  }
  return true;
}
}  // namespace

perk_status perk_perk2_disk_tableau(int S, int R, const int32_t* E, double* c, double* a) {
  return perk_perk2_disk_tableau_weights(S, R, E, 1.0, c, a);
}

perk_status perk_perk2_disk_tableau_weights(int S, int R, const int32_t* E, double bs, double* c, double* a) {
  if (S < 2 || S > MAX_S || R < 1 || R > MAX_R || !E || !c || !a || !(bs > 0.0) || !(bs <= 1.0))
    return PERK_E_INVALID_ARG;
  for (int r = 0; r < R; ++r)
    if (E[r] < 2 || E[r] > S || (r > 0 && E[r] < E[r - 1])) return PERK_E_INVALID_ARG;
  for (int i = 0; i < S; ++i) c[i] = (double)i / (2.0 * bs * (S - 1));
  for (int r = 0; r < R; ++r) {
    const int e = E[r];
    // coefficients of P(z) = 1/e + ((e-1)/e) (1 + z/(e-1))^e: alpha_k = ((e-1)/e) C(e,k) / (e-1)^k
    std::vector<double> alpha(e + 1);
    double binom = 1.0;
    for (int k = 0; k <= e; ++k) {
      alpha[k] = ((e - 1.0) / e) * binom / std::pow(e - 1.0, k);
      binom = binom * (e - k) / (k + 1);
    }
    if (!perk2_member_from_alpha(S, e, bs, alpha.data(), a + (size_t)r * S)) return PERK_E_INVALID_ARG;
  }
  return PERK_OK;
}

perk_status perk_perk2_member(int S, int E, double bs, const double* alpha, double* a) {
  if (S < 2 || S > MAX_S || E < 2 || E > S || !alpha || !a || !(bs > 0.0) || !(bs <= 1.0))
    return PERK_E_INVALID_ARG;
  if (std::fabs(alpha[0] - 1.0) > 1e-12 || std::fabs(alpha[1] - 1.0) > 1e-12 || std::fabs(alpha[2] - 0.5) > 1e-12)
    return fail(nullptr, PERK_E_INVALID_ARG, "alpha[0..2] must be 1, 1, 1/2 (second order)");
  if (!perk2_member_from_alpha(S, E, bs, alpha, a))
    return fail(nullptr, PERK_E_INVALID_ARG, "the polynomial has no member of this form (a zero product)");
  return PERK_OK;
}

perk_status perk_perk2_pattern_tableau(int S, int R, const int32_t* E, int pattern, double* c, uint8_t* eval,
                                       int32_t* src, double* a) {
  if (S < 2 || S > MAX_S || R < 1 || R > MAX_R || !E || !c || !eval || !src || !a || pattern < 0 || pattern > 2)
    return PERK_E_INVALID_ARG;
  for (int r = 0; r < R; ++r)
    if (E[r] < 2 || E[r] > S || (r > 0 && E[r] < E[r - 1])) return PERK_E_INVALID_ARG;
  for (int i = 0; i < S; ++i) c[i] = (double)i / (2.0 * (S - 1));
  for (int r = 0; r < R; ++r) {
    const int e = E[r];
    // the member's stages (1-based), ascending: classic 1, S-E+2 .. S; early 1 .. E-1, S;
    // alternating 1 and S - floor((E-1-k)(S-1)/(E-1) + 1/2), k = 1 .. E-1
    std::vector<int> st(e);
    st[0] = 1;
    for (int k = 1; k < e; ++k) {
      if (e == S || pattern == 0)
        st[k] = S - e + 1 + k;
      else if (pattern == 2)
        st[k] = k < e - 1 ? k + 1 : S;
      else
        st[k] = S - (int)std::floor((double)(e - 1 - k) * (S - 1) / (e - 1) + 0.5);
    }
    for (int k = 1; k < e; ++k)
      if (st[k] <= st[k - 1]) return PERK_E_INVALID_ARG;
    uint8_t* ev = eval + (size_t)r * S;
    int32_t* sr = src + (size_t)r * S;
    double* ar = a + (size_t)r * S;
    for (int i = 0; i < S; ++i) {
      ev[i] = 0;
      sr[i] = i > 0 ? i - 1 : 0;
      ar[i] = 0.0;
    }
    for (int k = 0; k < e; ++k) ev[st[k] - 1] = 1;
    // coefficients of the disk polynomial and the couplings s_k -> s_{k-1} from the last stage
    // backwards: the coefficient of z^{3+j} is c_{s_{E-2-j}} prod_{q=0}^{j} a_{s_{E-1-q}, s_{E-2-q}}
    std::vector<double> alpha(e + 1);
    double binom = 1.0;
    for (int k = 0; k <= e; ++k) {
      alpha[k] = ((e - 1.0) / e) * binom / std::pow(e - 1.0, k);
      binom = binom * (e - k) / (k + 1);
    }
    double prod = 1.0;
    for (int j = 0; j <= e - 3; ++j) {
      const int hi = st[e - 1 - j], lo = st[e - 2 - j];
      const double den = c[lo - 1] * prod;
      if (!(den != 0.0)) return PERK_E_INVALID_ARG;
      const double v = alpha[3 + j] / den;
      ar[hi - 1] = v;
      sr[hi - 1] = lo - 1;
      prod *= v;
    }
  }
  return PERK_OK;
}

// ---- third-order construction --------------------------------------------------------
namespace {

// 4x4 Gaussian elimination with partial pivoting; false if singular
bool solve4(double M[4][4], double g[4], double x[4]) {
  double A[4][5];
  for (int i = 0; i < 4; ++i) {
    for (int j = 0; j < 4; ++j) A[i][j] = M[i][j];
    A[i][4] = g[i];
  }
  for (int c = 0; c < 4; ++c) {
    int piv = c;
    for (int r = c + 1; r < 4; ++r)
      if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
    if (std::fabs(A[piv][c]) < 1e-300) return false;
    for (int j = 0; j < 5; ++j) std::swap(A[c][j], A[piv][j]);
    for (int r = 0; r < 4; ++r)
      if (r != c) {
        const double f = A[r][c] / A[c][c];
        for (int j = c; j < 5; ++j) A[r][j] -= f * A[c][j];
      }
  }
  for (int i = 0; i < 4; ++i) x[i] = A[i][4] / A[i][i];
  return true;
}

// a feasible d >= 0 of sum d = 1, sum k d = r, sum k(k-1) d = r^2, sum k(k-1)(k-2) d = r^3 (k = 0..E),
// by enumerating the basic solutions (at most four nonzeros); empty if none
std::vector<double> order3_weights(int E, double r) {
  const double g0[4] = {1.0, r, r * r, r * r * r};
  for (int a = 0; a <= E; ++a)
    for (int b = a + 1; b <= E; ++b)
      for (int c = b + 1; c <= E; ++c)
        for (int d = c + 1; d <= E; ++d) {
          const int cols[4] = {a, b, c, d};
          double M[4][4], g[4], x[4];
          for (int j = 0; j < 4; ++j) {
            const double k = cols[j];
            M[0][j] = 1.0;
            M[1][j] = k;
            M[2][j] = k * (k - 1.0);
            M[3][j] = k * (k - 1.0) * (k - 2.0);
          }
          for (int i = 0; i < 4; ++i) g[i] = g0[i];
          if (!solve4(M, g, x)) continue;
          bool ok = true;
          for (int j = 0; j < 4; ++j) ok = ok && x[j] >= -1e-13;
          if (!ok) continue;
          std::vector<double> w(E + 1, 0.0);
          for (int j = 0; j < 4; ++j) w[cols[j]] = std::max(0.0, x[j]);
          return w;
        }
  return {};
}

double binom(int n, int k) {
  double v = 1.0;
  for (int j = 1; j <= k; ++j) v = v * (n - k + j) / j;
  return v;
}

// coefficients p_0..p_S of 1 + z b^T (I - z A)^{-1} 1 of a P-ERK3 member (free entries x)
void perk3_poly(int S, int E, const double* c, const double* b, const std::vector<double>& x, std::vector<double>& p) {
  std::vector<double> A((size_t)S * S, 0.0);
  for (int i = 1; i < S; ++i) A[(size_t)i * S] = c[i];
  for (int q = 0; q < E - 2; ++q) {
    const int i = S - E + 2 + q;  // 0-based row
    A[(size_t)i * S + i - 1] = x[q];
    A[(size_t)i * S] = c[i] - x[q];
  }
  std::vector<double> v(S, 1.0), w(S);
  p.assign(S + 1, 0.0);
  p[0] = 1.0;
  for (int k = 1; k <= S; ++k) {
    double s = 0.0;
    for (int i = 0; i < S; ++i) s += b[i] * v[i];
    p[k] = s;
    for (int i = 0; i < S; ++i) {
      double t = 0.0;
      for (int j = 0; j < i; ++j) t += A[(size_t)i * S + j] * v[j];
      w[i] = t;
    }
    v.swap(w);
  }
}

// dense solve (n <= 64) with partial pivoting
bool solve_dense(std::vector<double> A, std::vector<double>& b, int n) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = r;
    if (std::fabs(A[(size_t)piv * n + c]) < 1e-300) return false;
    for (int j = 0; j < n; ++j) std::swap(A[(size_t)c * n + j], A[(size_t)piv * n + j]);
    std::swap(b[c], b[piv]);
    for (int r = c + 1; r < n; ++r) {
      const double f = A[(size_t)r * n + c] / A[(size_t)c * n + c];
      for (int j = c; j < n; ++j) A[(size_t)r * n + j] -= f * A[(size_t)c * n + j];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int j = r + 1; j < n; ++j) s -= A[(size_t)r * n + j] * b[j];
    b[r] = s / A[(size_t)r * n + r];
  }
  return true;
}

}  // namespace

perk_status perk_perk3_disk_alpha(int E, double* alpha, double* radius) {
  if (E < 3 || E > MAX_S || !alpha) return PERK_E_INVALID_ARG;
  double lo = 0.5, hi = (double)E;
  if (order3_weights(E, lo).empty()) return fail(nullptr, PERK_E_INVALID_ARG, "no third-order disk polynomial");
  for (int it = 0; it < 200 && hi - lo > 1e-13 * hi; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (!order3_weights(E, mid).empty())
      lo = mid;
    else
      hi = mid;
  }
  const std::vector<double> d = order3_weights(E, lo);
  for (int m = 0; m <= E; ++m) {
    double s = 0.0;
    for (int j = m; j <= E; ++j) s += d[j] * binom(j, m);
    alpha[m] = s / std::pow(lo, m);
  }
  if (radius) *radius = lo;
  return PERK_OK;
}

perk_status perk_perk3_member(int S, int E, const double* alpha, double* a_out) {
  if (S < 3 || S > MAX_S || E < 3 || E > S || !alpha || !a_out) return PERK_E_INVALID_ARG;
  std::vector<double> c(S), b(S, 0.0);
  for (int i = 1; i < S - 2; ++i) c[i] = (double)i / (S - 3.0);
  c[0] = 0.0;
  c[S - 2] = 1.0;
  c[S - 1] = 0.5;
  b[0] = 1.0 / 6.0;
  b[S - 2] += 1.0 / 6.0;
  b[S - 1] += 2.0 / 3.0;
  const int n = E - 2;
  auto residual = [&](const std::vector<double>& x, std::vector<double>& r) {
    std::vector<double> p;
    perk3_poly(S, E, c.data(), b.data(), x, p);
    r.resize(n);
    for (int k = 0; k < n; ++k) r[k] = (p[3 + k] - alpha[3 + k]) / alpha[3 + k];
  };
  auto norm = [](const std::vector<double>& r) {
    double m = 0.0;
    for (double v : r) m = std::max(m, std::fabs(v));
    return m;
  };
  const double starts[] = {0.5, 0.3, 0.7, 0.2, 0.8, 0.4, 0.6, 0.1, 0.9};
  for (double t0 : starts) {
    std::vector<double> x(n), r, rt, xt;
    for (int q = 0; q < n; ++q) x[q] = t0 * c[S - E + 2 + q];
    residual(x, r);
    for (int it = 0; it < 200 && norm(r) > 1e-14; ++it) {
      // Jacobian by central differences
      std::vector<double> J((size_t)n * n);
      for (int j = 0; j < n; ++j) {
        const double h = 1e-7 * std::max(1e-3, std::fabs(x[j]));
        std::vector<double> xp = x, xm = x, rp, rm;
        xp[j] += h;
        xm[j] -= h;
        residual(xp, rp);
        residual(xm, rm);
        for (int i = 0; i < n; ++i) J[(size_t)i * n + j] = (rp[i] - rm[i]) / (2.0 * h);
      }
      std::vector<double> dx(r);
      if (!solve_dense(J, dx, n)) break;
      // damped step keeping 0 < x < c
      double lam = 1.0;
      bool moved = false;
      for (int ls = 0; ls < 40; ++ls, lam *= 0.5) {
        xt = x;
        bool inside = true;
        for (int q = 0; q < n; ++q) {
          xt[q] -= lam * dx[q];
          const double cq = c[S - E + 2 + q];
          inside = inside && xt[q] > 0.0 && xt[q] < cq;
        }
        if (!inside) continue;
        residual(xt, rt);
        if (norm(rt) < norm(r)) {
          x = xt;
          r = rt;
          moved = true;
          break;
        }
      }
      if (!moved) break;
    }
    if (norm(r) < 1e-11) {
      for (int i = 0; i < S; ++i) a_out[i] = 0.0;
      for (int q = 0; q < n; ++q) a_out[S - E + 2 + q] = x[q];
      return PERK_OK;
    }
  }
  return fail(nullptr, PERK_E_INVALID_ARG, "no admissible third-order member found");
}

perk_status perk_perk3_disk_tableau(int S, int R, const int32_t* E, double* c, double* a) {
  if (S < 3 || S > MAX_S || R < 1 || R > MAX_R || !E || !c || !a) return PERK_E_INVALID_ARG;
  for (int r = 0; r < R; ++r)
    if (E[r] < 3 || E[r] > S || (r > 0 && E[r] < E[r - 1])) return PERK_E_INVALID_ARG;
  for (int i = 1; i < S - 2; ++i) c[i] = (double)i / (S - 3.0);
  c[0] = 0.0;
  c[S - 2] = 1.0;
  c[S - 1] = 0.5;
  std::vector<double> alpha(MAX_S + 1);
  for (int r = 0; r < R; ++r) {
    perk_status s = perk_perk3_disk_alpha(E[r], alpha.data(), nullptr);
    if (s != PERK_OK) return s;
    s = perk_perk3_member(S, E[r], alpha.data(), a + (size_t)r * S);
    if (s != PERK_OK) return s;
  }
  return PERK_OK;
}

perk_status perk_set_tableau(perk_ctx* ctx, int order, int S, int R, const int32_t* E, const double* c,
                             const double* a) {
  if (!ctx) return PERK_E_INVALID_ARG;
  if ((order != 2 && order != 3) || S < 1 || S > MAX_S || R < 1 || R > MAX_R || !E || !c || !a)
    return fail(ctx, PERK_E_INVALID_ARG, "invalid tableau dimensions");
  if (order == 3 && S < 3) return fail(ctx, PERK_E_INVALID_ARG, "third order needs S >= 3");
  for (int r = 0; r < R; ++r)
    if (E[r] < 1 || E[r] > S || (r > 0 && E[r] < E[r - 1]))
      return fail(ctx, PERK_E_INVALID_ARG, "member evaluations must ascend within [1, S]");
  if (E[R - 1] != S) return fail(ctx, PERK_E_INVALID_ARG, "the largest member must evaluate every stage");
  ctx->order = order;
  ctx->S = S;
  ctx->R = R;
  ctx->w_b1 = order == 3 ? 1.0 / 6.0 : 0.0;
  ctx->w_bp = order == 3 ? 1.0 / 6.0 : 0.0;
  ctx->w_bs = order == 3 ? 2.0 / 3.0 : 1.0;
  std::copy(E, E + R, ctx->E);
  ctx->c.assign(c, c + S);
  ctx->a.assign(a, a + (size_t)R * S);
  // a_{i,i-1}^{(r)} may be nonzero only where member r evaluates stage i-1 (stage 1, or S-E+2 .. S);
  // anything else would combine a stale stage
  for (int r = 0; r < R; ++r)
    for (int i0 = 1; i0 < S; ++i0) {
      const bool evaluated = (i0 == 1) || (i0 >= S - E[r] + 2);
      if (!evaluated && ctx->a[(size_t)r * S + i0] != 0.0)
        return fail(ctx, PERK_E_INVALID_ARG, "member %d: a_{%d,%d} != 0 but stage %d is not evaluated", r, i0 + 1,
                    i0, i0);
    }
  // classic pattern: stage i couples to K_{i-1}; member r is active at stage i >= 1 iff E[r] >= S - i + 1
  ctx->src.assign((size_t)R * S, 0);
  for (int r = 0; r < R; ++r)
    for (int i = 1; i < S; ++i) ctx->src[(size_t)r * S + i] = i - 1;
  for (int i = 0; i < MAX_S; ++i) {
    int mm = R;
    for (int r = R - 1; r >= 0; --r)
      if (i == 0 || E[r] >= S - i + 1) mm = r;
    ctx->stage_minmem[i] = i < S ? mm : R;
  }
  ctx->pattern_mode = false;
  ctx->has_tab = true;
  drop_graph(ctx);
  perk_status s = upload_coef(ctx);
  if (s != PERK_OK) return s;
  if (ctx->has_mesh) return run_partition(ctx);
  return PERK_OK;
}

perk_status perk_set_tableau_pattern(perk_ctx* ctx, int order, int S, int R, const int32_t* E,
                                     const uint8_t* eval, const int32_t* src, const double* c, const double* a) {
  if (!ctx) return PERK_E_INVALID_ARG;
  if (order != 2 || S < 2 || S > MAX_S || R < 1 || R > MAX_R || !E || !eval || !src || !c || !a)
    return fail(ctx, PERK_E_INVALID_ARG, "invalid pattern tableau (second order, 2 <= S <= %d)", MAX_S);
  for (int r = 0; r < R; ++r) {
    if (E[r] < 2 || E[r] > S || (r > 0 && E[r] < E[r - 1]))
      return fail(ctx, PERK_E_INVALID_ARG, "member evaluations must ascend within [2, S]");
    const uint8_t* ev = eval + (size_t)r * S;
    int count = 0;
    for (int i = 0; i < S; ++i) count += ev[i] ? 1 : 0;
    if (!ev[0] || !ev[S - 1] || count != E[r])
      return fail(ctx, PERK_E_INVALID_ARG, "member %d must evaluate stage 1, stage S and E = %d stages in all", r, E[r]);
    if (r > 0)
      for (int i = 0; i < S; ++i)
        if (eval[(size_t)(r - 1) * S + i] && !ev[i])
          return fail(ctx, PERK_E_INVALID_ARG, "member %d evaluates stage %d but the finer member %d does not", r - 1,
                      i + 1, r);
    for (int i = 1; i < S; ++i) {
      const int32_t sr = src[(size_t)r * S + i];
      const double ar = a[(size_t)r * S + i];
      if (sr < 0 || sr >= i) return fail(ctx, PERK_E_INVALID_ARG, "member %d, stage %d: source stage out of range", r, i + 1);
      if (ar != 0.0 && !ev[sr])
        return fail(ctx, PERK_E_INVALID_ARG, "member %d, stage %d couples to stage %d, which it does not evaluate", r,
                    i + 1, sr + 1);
    }
  }
  if (E[R - 1] != S) return fail(ctx, PERK_E_INVALID_ARG, "the largest member must evaluate every stage");
  ctx->order = order;
  ctx->S = S;
  ctx->R = R;
  ctx->w_b1 = 0.0;
  ctx->w_bp = 0.0;
  ctx->w_bs = 1.0;
  std::copy(E, E + R, ctx->E);
  ctx->c.assign(c, c + S);
  ctx->a.assign(a, a + (size_t)R * S);
  ctx->src.assign(src, src + (size_t)R * S);
  bool classic = true;
  for (int r = 0; r < R; ++r)
    for (int i = 1; i < S; ++i) classic = classic && (ctx->a[(size_t)r * S + i] == 0.0 || ctx->src[(size_t)r * S + i] == i - 1);
  for (int i = 0; i < MAX_S; ++i) {
    int mm = R;
    for (int r = R - 1; r >= 0; --r)
      if (i < S && eval[(size_t)r * S + i]) mm = r;
    ctx->stage_minmem[i] = mm;
  }
  ctx->pattern_mode = !classic;
  ctx->has_tab = true;
  drop_graph(ctx);
  perk_status s = upload_coef(ctx);
  if (s != PERK_OK) return s;
  if (ctx->has_mesh) return run_partition(ctx);
  return PERK_OK;
}

perk_status perk_set_weights(perk_ctx* ctx, double b1, double bs) {
  if (!ctx) return PERK_E_INVALID_ARG;
  if (!ctx->has_tab || ctx->order != 2 || ctx->S < 2) return fail(ctx, PERK_E_NOT_READY, "needs a second-order tableau");
  if (!(bs > 0.0) || !std::isfinite(b1) || std::fabs(b1 + bs - 1.0) > 1e-14)
    return fail(ctx, PERK_E_INVALID_ARG, "weights must satisfy b1 + bS = 1, bS > 0");
  if (std::fabs(bs * ctx->c[ctx->S - 1] - 0.5) > 1e-12)
    return fail(ctx, PERK_E_INVALID_ARG, "second order needs bS c_S = 1/2 (c_S = %.17g)", ctx->c[ctx->S - 1]);
  ctx->w_b1 = b1;
  ctx->w_bp = 0.0;
  ctx->w_bs = bs;
  drop_graph(ctx);
  return PERK_OK;
}

perk_status perk_reference_nodes(int N, double* x, double* w) {
  if (N < 1 || N > 16 || !x || !w) return PERK_E_INVALID_ARG;
  std::vector<double> xv, wv;
  lgl(N, xv, wv);
  std::copy(xv.begin(), xv.end(), x);
  std::copy(wv.begin(), wv.end(), w);
  return PERK_OK;
}

perk_status perk_partition(perk_ctx* ctx) {
  if (!ctx) return PERK_E_INVALID_ARG;
  return run_partition(ctx);
}

static perk_status rhs_given(perk_ctx* ctx, int stage, const double* d_Y, double* d_K) {
  if (!ctx->has_mesh || !ctx->partitioned) return fail(ctx, PERK_E_NOT_READY, "no mesh");
  if (!d_Y || !d_K) return fail(ctx, PERK_E_INVALID_ARG, "null array");
  StageArgs sa{};
  sa.Y = d_Y;
  const int64_t ne = stage < 0 ? ctx->n_elem : ctx->act_el[stage];
  const int64_t ni = stage < 0 ? ctx->n_if : ctx->act_if[stage];
  const int64_t nm = stage < 0 ? ctx->n_mort : ctx->act_mort[stage];
  PERK_CUDA(ctx, launch_faces(ctx->stream, Y_GIVEN, ctx->ops, ni, ctx->d_if_sorted.p, nm, ctx->d_mort_sorted.p,
                              ctx->d_method.p, sa, ctx->d_surf.p));
  PERK_CUDA(ctx, launch_volume(ctx->stream, Y_GIVEN, ctx->ops, ne, ctx->d_elem_sorted.p, ctx->d_level.p,
                               ctx->d_method.p, 2.0 / ctx->length, sa, ctx->d_surf.p, d_K, nullptr, ctx->d_logtab.p,
                               ctx->vol_epb));
  if (ctx->viscous())
    PERK_CUDA(ctx, launch_br1(ctx->stream, Y_GIVEN, ctx->ops, ctx->prob.mu, ctx->kappa(),
                              stage < 0 ? ctx->n_if : ctx->halo_if[stage], stage < 0 ? ctx->n_mort : ctx->halo_mort[stage],
                              ni, nm, ctx->d_if_sorted.p, ctx->d_mort_sorted.p,
                              stage < 0 ? ctx->n_elem : ctx->halo_el[stage], ne, ctx->d_elem_sorted.p,
                              ctx->d_level.p, ctx->d_method.p, 2.0 / ctx->length, sa, ctx->d_wsurf.p, ctx->d_q.p,
                              ctx->d_vsurf.p, d_K, nullptr));
  return PERK_OK;
}

perk_status perk_rhs_full(perk_ctx* ctx, const double* d_Y, double* d_K) {
  if (!ctx) return PERK_E_INVALID_ARG;
  return rhs_given(ctx, -1, d_Y, d_K);
}

perk_status perk_rhs_active(perk_ctx* ctx, int stage, const double* d_Y, double* d_K) {
  if (!ctx) return PERK_E_INVALID_ARG;
  if (!ctx->has_tab) return fail(ctx, PERK_E_NOT_READY, "no tableau");
  if (stage < 0 || stage >= ctx->S) return fail(ctx, PERK_E_INVALID_ARG, "stage %d outside [0, %d)", stage, ctx->S);
  return rhs_given(ctx, stage, d_Y, d_K);
}

// device memory a step needs beyond the mesh buffers (allocated outside any graph capture)
static perk_status prepare_step(perk_ctx* ctx) {
  if (ctx->pattern_mode) {
    if (ctx->ws_base && (!ctx->d_Kpat.ext || ctx->d_Kpat.cap < (size_t)ctx->n_elem * ELEM * ctx->S))
      return fail(ctx, PERK_E_OOM,
                  "a stage pattern keeps all S stages, which the bound workspace does not hold: query "
                  "perk_workspace_bytes after setting the tableau and bind again");
    PERK_CUDA(ctx, ctx->d_Kpat.ensure((size_t)ctx->n_elem * ELEM * ctx->S));
  }
  return PERK_OK;
}

static perk_status step_impl(perk_ctx* ctx, double* d_U) {
  {
    perk_status s = prepare_step(ctx);
    if (s != PERK_OK) return s;
  }
  if (ctx->prob.use_graph) {
    if (!ctx->graph_valid || ctx->graph_U != d_U) {
      cudaGraph_t g = nullptr;
      PERK_CUDA(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
      perk_status s = enqueue_step(ctx, ctx->cap_stream, d_U);
      cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &g);
      if (s != PERK_OK) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();   // the failed capture's error is reported once, not by later calls
        return s;
      }
      PERK_CUDA(ctx, ce);
      // a re-captured step usually differs from the previous one only in launch sizes and
      // pointers: update the executable graph in place, instantiate only if that fails
      bool updated = false;
      if (ctx->graph) {
        cudaGraphExecUpdateResultInfo info;
        updated = cudaGraphExecUpdate(ctx->graph, g, &info) == cudaSuccess;
        if (!updated) {
          cudaGetLastError();
          cudaGraphExecDestroy(ctx->graph);
          ctx->graph = nullptr;
        }
      }
      cudaError_t ie = updated ? cudaSuccess : cudaGraphInstantiate(&ctx->graph, g, 0);
      cudaGraphDestroy(g);
      PERK_CUDA(ctx, ie);
      ctx->graph_U = d_U;
      ctx->graph_valid = true;
    }
    PERK_CUDA(ctx, cudaGraphLaunch(ctx->graph, ctx->stream));
  } else {
    perk_status s = enqueue_step(ctx, ctx->stream, d_U);
    if (s != PERK_OK) return s;
  }
  ctx->counters.steps += 1;
  for (int i = 0; i < ctx->S; ++i) {
    ctx->counters.element_stage_evaluations += ctx->act_el[i];
    ctx->counters.dof_stage_updates += ctx->act_el[i] * NODES;
  }
  return PERK_OK;
}

static perk_status step_ready(perk_ctx* ctx, double* d_U) {
  if (!ctx->has_mesh || !ctx->has_tab || !ctx->partitioned || ctx->part_S != ctx->S)
    return fail(ctx, PERK_E_NOT_READY, "mesh or tableau missing");
  if (!d_U) return fail(ctx, PERK_E_INVALID_ARG, "null U");
  if (((uintptr_t)d_U & 15) != 0) return fail(ctx, PERK_E_INVALID_ARG, "U must be 16-byte aligned");
  return PERK_OK;
}

perk_status perk_step(perk_ctx* ctx, double* d_U, double dt) {
  if (!ctx) return PERK_E_INVALID_ARG;
  perk_status s = step_ready(ctx, d_U);
  if (s != PERK_OK) return s;
  s = set_dts(ctx, nullptr, dt);
  if (s != PERK_OK) return s;
  return step_impl(ctx, d_U);
}

perk_status perk_step_profiled(perk_ctx* ctx, double* d_U, double dt, perk_kernel_times* acc) {
  if (!ctx || !acc) return PERK_E_INVALID_ARG;
  if (!ctx->has_mesh || !ctx->has_tab || !ctx->partitioned || ctx->part_S != ctx->S)
    return fail(ctx, PERK_E_NOT_READY, "mesh or tableau missing");
  if (!d_U || !std::isfinite(dt) || !(dt > 0.0)) return fail(ctx, PERK_E_INVALID_ARG, "bad U or dt");
  {
    perk_status s = set_dts(ctx, nullptr, dt);
    if (s != PERK_OK) return s;
  }
  {
    perk_status s = prepare_step(ctx);
    if (s != PERK_OK) return s;
  }
  LaunchTimer timer;
  perk_status s = enqueue_step(ctx, ctx->stream, d_U, &timer);
  if (s != PERK_OK) return s;
  PERK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (size_t q = 0; q < timer.stop.size(); ++q) {
    float ms = 0.f;
    PERK_CUDA(ctx, cudaEventElapsedTime(&ms, timer.start[q], timer.stop[q]));
    acc->ms[timer.kind[q]] += ms;
    acc->launches[timer.kind[q]] += 1;
  }
  for (int i = 0; i < ctx->S; ++i) acc->element_stages += ctx->act_el[i];
  ctx->counters.steps += 1;
  for (int i = 0; i < ctx->S; ++i) {
    ctx->counters.element_stage_evaluations += ctx->act_el[i];
    ctx->counters.dof_stage_updates += ctx->act_el[i] * NODES;
  }
  return PERK_OK;
}

perk_status perk_step_dts(perk_ctx* ctx, double* d_U, const double* dts) {
  if (!ctx) return PERK_E_INVALID_ARG;
  if (!dts) return fail(ctx, PERK_E_INVALID_ARG, "null dts");
  perk_status s = step_ready(ctx, d_U);
  if (s != PERK_OK) return s;
  s = set_dts(ctx, dts, 0.0);
  if (s != PERK_OK) return s;
  return step_impl(ctx, d_U);
}

perk_status perk_compute_dt_members(perk_ctx* ctx, const double* d_U, double cfl, double* dts) {
  if (!ctx || !dts) return PERK_E_INVALID_ARG;
  if (!ctx->has_mesh) return fail(ctx, PERK_E_NOT_READY, "no mesh");
  if (!d_U || !(cfl > 0.0)) return fail(ctx, PERK_E_INVALID_ARG, "bad U or cfl");
  PERK_CUDA(ctx, ctx->d_block_min.ensure((size_t)std::max(ctx->n_members, DT_MAX_BLOCKS)));
  PERK_CUDA(ctx, launch_dt_members(ctx->stream, ctx->n_elem, d_U, ctx->d_level.p, ctx->d_member.p, ctx->n_members,
                                   ctx->length, ctx->ops.gamma, ctx->d_block_min.p));
  std::vector<double> m(ctx->n_members);
  PERK_CUDA(ctx, cudaMemcpyAsync(m.data(), ctx->d_block_min.p, m.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                 ctx->stream));
  PERK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (int q = 0; q < ctx->n_members; ++q)
    if (!std::isfinite(m[q]) || !(m[q] > 0.0))
      return fail(ctx, PERK_E_NONFINITE, "member %d: a node has no admissible wave speed (rho or p <= 0, or NaN)", q);
  for (int q = 0; q < ctx->n_members; ++q) dts[q] = cfl * m[q] / (double)NN;
  return PERK_OK;
}

perk_status perk_check(perk_ctx* ctx) {
  if (!ctx) return PERK_E_INVALID_ARG;
  PERK_CUDA(ctx, cudaMemcpyAsync(&ctx->h_pin->flag, ctx->d_flag.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  PERK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const int flag = ctx->h_pin->flag;
  if (flag) {
    PERK_CUDA(ctx, cudaMemsetAsync(ctx->d_flag.p, 0, sizeof(int), ctx->stream));
    PERK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->counters.rejected_steps_checked += 1;
    if (flag & 2)
      return fail(ctx, PERK_E_TIMEOUT, "a stage's volume work gave up waiting for its face fluxes; the step was "
                                       "not committed");
    return fail(ctx, PERK_E_NONFINITE, "a step produced a non-admissible state and was not committed");
  }
  return PERK_OK;
}

perk_status perk_set_stage_fusion(perk_ctx* ctx, int enabled) {
  if (!ctx) return PERK_E_INVALID_ARG;
  if (enabled < 0 || enabled > 2) return fail(ctx, PERK_E_INVALID_ARG, "fusion mode must be 0, 1 or 2");
  if (ctx->fuse_stage != (enabled != 0) || ctx->fuse_step != (enabled == 2)) {
    ctx->fuse_stage = enabled != 0;
    ctx->fuse_step = enabled == 2;
    drop_graph(ctx);
  }
  return PERK_OK;
}

perk_status perk_compute_dt(perk_ctx* ctx, const double* d_U, double cfl, double* dt) {
  if (!ctx || !dt) return PERK_E_INVALID_ARG;
  if (!ctx->has_mesh) return fail(ctx, PERK_E_NOT_READY, "no mesh");
  if (!d_U || !(cfl > 0.0)) return fail(ctx, PERK_E_INVALID_ARG, "bad U or cfl");
  const int nb = (int)std::min<int64_t>(DT_MAX_BLOCKS, (ctx->n_elem * NODES + DT_THREADS - 1) / DT_THREADS);
  if (ctx->d_block_min.cap < (size_t)nb) return fail(ctx, PERK_E_INVALID_ARG, "internal: step-size scratch too small");
  PERK_CUDA(ctx, launch_dt(ctx->stream, ctx->n_elem, d_U, ctx->d_level.p, ctx->length, ctx->ops.gamma,
                           ctx->d_block_min.p, nb, ctx->d_dt_out.p));
  PERK_CUDA(ctx, cudaMemcpyAsync(&ctx->h_pin->dt, ctx->d_dt_out.p, sizeof(double), cudaMemcpyDeviceToHost,
                                 ctx->stream));
  PERK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const double m = ctx->h_pin->dt;
  if (!std::isfinite(m) || !(m > 0.0))
    return fail(ctx, PERK_E_NONFINITE, "a node has no admissible wave speed (rho or p <= 0, or NaN)");
  *dt = cfl * m / (double)NN;
  return PERK_OK;
}

// smallest member active at a stage (members are active from the finest down): K_1 everywhere,
// otherwise members with E >= S - stage + 1
static int min_active_member(const perk_ctx* ctx, int stage) {
  if (stage <= 0 || !ctx->has_tab) return 0;
  return ctx->stage_minmem[stage];
}

perk_status perk_rhs_jvp(perk_ctx* ctx, int stage, const double* d_Y, const double* d_V, double* d_Kd) {
  if (!ctx) return PERK_E_INVALID_ARG;
  if (!ctx->differentiable())
    return fail(ctx, PERK_E_INVALID_ARG, "derivatives are built for HLL, HLLC and EC surface fluxes without shock capturing");
  if (ctx->viscous()) return fail(ctx, PERK_E_INVALID_ARG, "derivatives are built for the Euler equations");
  if (!ctx->has_mesh || !ctx->partitioned) return fail(ctx, PERK_E_NOT_READY, "no mesh");
  if (!d_Y || !d_V || !d_Kd) return fail(ctx, PERK_E_INVALID_ARG, "null array");
  if (stage >= 0 && (!ctx->has_tab || stage >= ctx->S)) return fail(ctx, PERK_E_INVALID_ARG, "bad stage %d", stage);
  const int64_t ne = stage < 0 ? ctx->n_elem : ctx->act_el[stage];
  const int64_t ni = stage < 0 ? ctx->n_if : ctx->act_if[stage];
  const int64_t nm = stage < 0 ? ctx->n_mort : ctx->act_mort[stage];
  PERK_CUDA(ctx, ctx->d_surf_d.ensure((size_t)ctx->n_elem * ELEM));
  PERK_CUDA(ctx, launch_jvp(ctx->stream, ctx->ops, ni, ctx->d_if_sorted.p, nm, ctx->d_mort_sorted.p, ne,
                            ctx->d_elem_sorted.p, ctx->d_level.p, 2.0 / ctx->length, d_Y, d_V, ctx->d_logtab.p,
                            ctx->d_surf.p, ctx->d_surf_d.p, nullptr, d_Kd));
  return PERK_OK;
}

perk_status perk_rhs_vjp(perk_ctx* ctx, int stage, const double* d_Y, const double* d_lam, double* d_g) {
  if (!ctx) return PERK_E_INVALID_ARG;
  if (!ctx->differentiable())
    return fail(ctx, PERK_E_INVALID_ARG, "derivatives are built for HLL, HLLC and EC surface fluxes without shock capturing");
  if (ctx->viscous()) return fail(ctx, PERK_E_INVALID_ARG, "derivatives are built for the Euler equations");
  if (!ctx->has_mesh || !ctx->partitioned) return fail(ctx, PERK_E_NOT_READY, "no mesh");
  if (!d_Y || !d_lam || !d_g) return fail(ctx, PERK_E_INVALID_ARG, "null array");
  if (stage >= 0 && (!ctx->has_tab || stage >= ctx->S)) return fail(ctx, PERK_E_INVALID_ARG, "bad stage %d", stage);
  const int64_t na = stage < 0 ? ctx->n_elem : ctx->act_el[stage];
  const int64_t ni = stage < 0 ? ctx->n_if : ctx->act_if[stage];
  const int64_t nm = stage < 0 ? ctx->n_mort : ctx->act_mort[stage];
  PERK_CUDA(ctx, ctx->d_surf_d.ensure((size_t)ctx->n_elem * ELEM));
  StageArgs sa{};
  sa.Y = d_Y;
  const int mm = min_active_member(ctx, stage);
  PERK_CUDA(ctx, ctx->d_rctl.ensure(2 * MAX_S));
  PERK_CUDA(ctx, cudaMemsetAsync(ctx->d_surf_d.p, 0, (size_t)ctx->n_elem * ELEM * sizeof(double), ctx->stream));
  PERK_CUDA(ctx, cudaMemsetAsync(ctx->d_rctl.p, 0, sizeof(unsigned long long), ctx->stream));
  PERK_CUDA(ctx, launch_vjp_stage(ctx->stream, Y_GIVEN, ctx->ops, na, ctx->d_elem_sorted.p, ni, ctx->d_if_sorted.p, nm,
                                  ctx->d_mort_sorted.p, ctx->d_level.p, ctx->d_method.p, mm, 2.0 / ctx->length, sa,
                                  d_lam, ctx->d_logtab.p, d_g, ctx->d_surf_d.p, ctx->d_rctl.p));
  PERK_CUDA(ctx, launch_vjp_gather(ctx->stream, ctx->n_elem, ctx->d_method.p, mm, ctx->d_surf_d.p, d_g));
  return PERK_OK;
}

static perk_status step_ready_adjoint(perk_ctx* ctx, const double* d_Un, double dt) {
  if (ctx->viscous()) return fail(ctx, PERK_E_INVALID_ARG, "derivatives are built for the Euler equations");
  if (!ctx->differentiable())
    return fail(ctx, PERK_E_INVALID_ARG, "derivatives are built for HLL, HLLC and EC surface fluxes without shock capturing");
  if (!ctx->has_mesh || !ctx->has_tab || !ctx->partitioned || ctx->part_S != ctx->S)
    return fail(ctx, PERK_E_NOT_READY, "mesh or tableau missing");
  if (ctx->n_members != 1) return fail(ctx, PERK_E_INVALID_ARG, "the step adjoint takes single-member contexts");
  if (!d_Un || !(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, PERK_E_INVALID_ARG, "bad U or dt");
  if (ctx->order == 3 && ctx->S < 3) return fail(ctx, PERK_E_INVALID_ARG, "third order needs S >= 3");
  return set_dts(ctx, nullptr, dt);
}

// the stages of one step from U_n, stage i stored in K + i * n_elem * 64; when d_U is given,
// all S stages are evaluated, the last one checks admissibility and the commit updates d_U (as
// perk_step does); without d_U only K_1 .. K_{S-1} are evaluated: the reverse sweep needs the
// stage states Y_1 .. Y_S, and none of them is formed from K_S
static perk_status enqueue_stages(perk_ctx* ctx, cudaStream_t st, const double* d_Un, double* K, double* d_U) {
  const size_t nd = (size_t)ctx->n_elem * ELEM;
  UpdateArgs ua{};
  ua.b1 = ctx->w_b1;
  ua.bp = ctx->w_bp;
  ua.bs = ctx->w_bs;
  ua.U = d_U;
  ua.K1 = K;
  ua.Kp = K + (size_t)(ctx->S > 1 ? ctx->S - 2 : 0) * nd;   // K_{S-1}
  ua.flag = ctx->d_flag.p;
  const int n_stages = d_U ? ctx->S : ctx->S - 1;
  const bool fused = d_U && ctx->stage_fused();
  for (int i = 0; i < n_stages; ++i) {
    StageArgs sa{};
    sa.U = d_Un;
    sa.K1 = K;
    sa.Kp = K + (size_t)(i > 0 ? i - 1 : 0) * nd;
    sa.coef = ctx->d_coef.p + (size_t)i * MAX_R;
    sa.dt = ctx->d_dt.p;
    const bool check = d_U && i == ctx->S - 1;
    // one launch per stage only when the final update follows (it restarts the stage counters)
    if (fused) {
      PERK_CUDA(ctx, launch_stage(st, i, ctx->ops, ctx->act_if[i], ctx->d_if_sorted.p, ctx->act_mort[i],
                                  ctx->d_mort_sorted.p, ctx->act_el[i], ctx->d_elem_sorted.p, ctx->d_level.p,
                                  ctx->d_method.p, 2.0 / ctx->length, sa, ctx->d_surf.p, K + (size_t)i * nd,
                                  check ? &ua : nullptr, ctx->d_logtab.p, ctx->d_ctl.p, ctx->d_stamp.p,
                                  ctx->d_flag.p));
      continue;
    }
    PERK_CUDA(ctx, launch_faces(st, Y_COMBINE, ctx->ops, ctx->act_if[i], ctx->d_if_sorted.p, ctx->act_mort[i],
                                ctx->d_mort_sorted.p, ctx->d_method.p, sa, ctx->d_surf.p));
    PERK_CUDA(ctx, launch_volume(st, Y_COMBINE, ctx->ops, ctx->act_el[i], ctx->d_elem_sorted.p, ctx->d_level.p,
                                 ctx->d_method.p, 2.0 / ctx->length, sa, ctx->d_surf.p, K + (size_t)i * nd,
                                 check ? &ua : nullptr, ctx->d_logtab.p, ctx->vol_epb));
  }
  ua.stage_ctl = fused ? ctx->d_ctl.p : nullptr;
  if (d_U) PERK_CUDA(ctx, launch_commit(st, ctx->n_elem, ua, K + (size_t)(ctx->S - 1) * nd, ctx->d_dt.p, d_U));
  return PERK_OK;
}

// buffers, the second stream and its events of the reverse sweep (allocated outside any capture)
static perk_status prepare_reverse(perk_ctx* ctx) {
  const size_t nd = (size_t)ctx->n_elem * ELEM;
  PERK_CUDA(ctx, ctx->d_g.ensure(nd));
  PERK_CUDA(ctx, ctx->d_lamK1.ensure(nd));
  PERK_CUDA(ctx, ctx->d_lamKa.ensure(nd));
  PERK_CUDA(ctx, ctx->d_lamKb.ensure(nd));
  PERK_CUDA(ctx, ctx->d_surf_d.ensure(nd));
  PERK_CUDA(ctx, ctx->d_rctl.ensure(2 * MAX_S));
  if (!ctx->aux_stream) {
    PERK_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking));
    PERK_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    PERK_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
  }
  return PERK_OK;
}

// the reverse sweep of one step whose stages K (from U_n) are stored (prepare_reverse first)
static perk_status enqueue_reverse(perk_ctx* ctx, cudaStream_t st, const double* d_Un, double dt, const double* K,
                                   const double* d_lam_np1, double* d_lam_n) {
  const int S = ctx->S;
  const size_t nd = (size_t)ctx->n_elem * ELEM;
  // seed with the final update U_{n+1} = U_n + dt (b1 K_1 + b_{S-1} K_{S-1} + b_S K_S)
  const double b1 = ctx->w_b1, bp = ctx->w_bp, bs = ctx->w_bs;
  double* lam_cur = ctx->d_lamKa.p;    // adjoint of K_i at the current stage i
  double* lam_prev = ctx->d_lamKb.p;   // adjoint of K_{i-1}, being accumulated
  double* lamK1 = ctx->d_lamK1.p;
  // face adjoints start from zero; each stage's accumulation clears what it gathers
  PERK_CUDA(ctx, cudaMemsetAsync(ctx->d_surf_d.p, 0, nd * sizeof(double), st));
  const bool fused = ctx->stage_fused();
  // item counters of the reverse stage launches (two per stage when faces and volume run apart)
  PERK_CUDA(ctx, cudaMemsetAsync(ctx->d_rctl.p, 0, 2 * MAX_S * sizeof(unsigned long long), st));
  if (S == 1) {
    PERK_CUDA(ctx, launch_adj_seed(st, ctx->n_elem, dt, 0.0, 0.0, b1 + bp + bs, d_lam_np1, d_lam_n, lam_prev, nullptr,
                                   lamK1));
  } else {
    PERK_CUDA(ctx, launch_adj_seed(st, ctx->n_elem, dt, b1, bp, bs, d_lam_np1, d_lam_n, lamK1,
                                   S - 1 > 1 ? lam_prev : nullptr, lam_cur));
  }
  for (int i = S - 1; i >= 0; --i) {
    // adjoint of K_i is in lam_cur (for i == 0 it is the accumulated lamK1); the stage state
    // Y_i = U_n + dt (alpha K_1 + beta K_{i-1}) is formed inside the VJP kernels
    double* lam_i = (i == 0) ? lamK1 : lam_cur;
    const StageCoef* coef = (i == 0) ? nullptr : ctx->d_coef.p + (size_t)i * MAX_R;
    const int mm = min_active_member(ctx, i);
    StageArgs sa{};
    sa.U = d_Un;
    sa.K1 = K;
    sa.Kp = K + (size_t)(i > 0 ? i - 1 : 0) * nd;
    sa.coef = coef;
    sa.dt = ctx->d_dt.p;
    if (fused) {
      // face and volume adjoints in one launch
      PERK_CUDA(ctx, launch_vjp_stage(st, Y_COMBINE, ctx->ops, ctx->act_el[i], ctx->d_elem_sorted.p, ctx->act_if[i],
                                      ctx->d_if_sorted.p, ctx->act_mort[i], ctx->d_mort_sorted.p, ctx->d_level.p,
                                      ctx->d_method.p, mm, 2.0 / ctx->length, sa, lam_i, ctx->d_logtab.p, ctx->d_g.p,
                                      ctx->d_surf_d.p, ctx->d_rctl.p + i));
    } else {
      // the face items on the second stream, beside the volume items (the same kernel, so the
      // results do not depend on the mode)
      PERK_CUDA(ctx, cudaEventRecord(ctx->ev_fork, st));
      PERK_CUDA(ctx, cudaStreamWaitEvent(ctx->aux_stream, ctx->ev_fork, 0));
      PERK_CUDA(ctx, launch_vjp_stage(ctx->aux_stream, Y_COMBINE, ctx->ops, 0, ctx->d_elem_sorted.p, ctx->act_if[i],
                                      ctx->d_if_sorted.p, ctx->act_mort[i], ctx->d_mort_sorted.p, ctx->d_level.p,
                                      ctx->d_method.p, mm, 2.0 / ctx->length, sa, lam_i, ctx->d_logtab.p, ctx->d_g.p,
                                      ctx->d_surf_d.p, ctx->d_rctl.p + MAX_S + i));
      PERK_CUDA(ctx, cudaEventRecord(ctx->ev_join, ctx->aux_stream));
      PERK_CUDA(ctx, launch_vjp_stage(st, Y_COMBINE, ctx->ops, ctx->act_el[i], ctx->d_elem_sorted.p, 0,
                                      ctx->d_if_sorted.p, 0, ctx->d_mort_sorted.p, ctx->d_level.p, ctx->d_method.p, mm,
                                      2.0 / ctx->length, sa, lam_i, ctx->d_logtab.p, ctx->d_g.p, ctx->d_surf_d.p,
                                      ctx->d_rctl.p + i));
      PERK_CUDA(ctx, cudaStreamWaitEvent(st, ctx->ev_join, 0));
    }
    // the stage's halo: its active elements and their face neighbours (a prefix of the sorted list)
    const int64_t halo = ctx->halo_el[i];
    if (i == 0) {
      PERK_CUDA(ctx, launch_adj_accum(st, halo, ctx->d_elem_sorted.p, ctx->d_method.p, mm, nullptr, dt, ctx->d_g.p,
                                      ctx->d_surf_d.p, d_lam_n, nullptr, nullptr, 0));
    } else {
      // contributions to K_{i-1}: into lamK1 when i - 1 == 0; else into lam_prev, which holds the
      // final-update seed only for K_{S-1} (i == S-1) and is otherwise assigned here
      double* target = (i - 1 == 0) ? lamK1 : lam_prev;
      const int assign = (i - 1 == 0 || i == S - 1) ? 0 : 1;
      PERK_CUDA(ctx, launch_adj_accum(st, halo, ctx->d_elem_sorted.p, ctx->d_method.p, mm, coef, dt, ctx->d_g.p,
                                      ctx->d_surf_d.p, d_lam_n, lamK1, target, assign));
      if (i - 1 > 0) std::swap(lam_cur, lam_prev);   // lam_cur <- adjoint of K_{i-1}
    }
  }
  return PERK_OK;
}

// Replays the graph exec of the work enqueue(stream) issues, capturing it again (and updating the
// executable graph in place where it can) when valid is false; without graphs the work is issued
// on the context's stream directly.
extern "C++" {   // (a template, inside the C-linkage block)
template <class F>
static perk_status run_captured(perk_ctx* ctx, cudaGraphExec_t& exec, bool& valid, F&& enqueue) {
  if (!ctx->prob.use_graph) return enqueue(ctx->stream);
  if (!valid) {
    cudaGraph_t g = nullptr;
    PERK_CUDA(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    perk_status s = enqueue(ctx->cap_stream);
    cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &g);
    if (s != PERK_OK) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return s;
    }
    PERK_CUDA(ctx, ce);
    bool updated = false;
    if (exec) {
      cudaGraphExecUpdateResultInfo info;
      updated = cudaGraphExecUpdate(exec, g, &info) == cudaSuccess;
      if (!updated) {
        cudaGetLastError();
        cudaGraphExecDestroy(exec);
        exec = nullptr;
      }
    }
    cudaError_t ie = updated ? cudaSuccess : cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    PERK_CUDA(ctx, ie);
    valid = true;
  }
  PERK_CUDA(ctx, cudaGraphLaunch(exec, ctx->stream));
  return PERK_OK;
}
}  // extern "C++"

perk_status perk_step_store(perk_ctx* ctx, double* d_U, double dt, double* d_K) {
  if (!ctx) return PERK_E_INVALID_ARG;
  perk_status s = step_ready_adjoint(ctx, d_U, dt);
  if (s != PERK_OK) return s;
  if (!d_K) return fail(ctx, PERK_E_INVALID_ARG, "null stage array");
  if (ctx->store_key[0] != d_U || ctx->store_key[1] != d_K) {
    ctx->store_valid = false;
    ctx->store_key[0] = d_U;
    ctx->store_key[1] = d_K;
  }
  s = run_captured(ctx, ctx->graph_store, ctx->store_valid,
                   [&](cudaStream_t st) { return enqueue_stages(ctx, st, d_U, d_K, d_U); });
  if (s != PERK_OK) return s;
  ctx->counters.steps += 1;
  for (int i = 0; i < ctx->S; ++i) {
    ctx->counters.element_stage_evaluations += ctx->act_el[i];
    ctx->counters.dof_stage_updates += ctx->act_el[i] * NODES;
  }
  return PERK_OK;
}

// the reverse step (with the stages recomputed into the context's array first when recompute)
static perk_status run_reverse(perk_ctx* ctx, const double* d_Un, double dt, const double* K, bool recompute,
                               const double* d_lam_np1, double* d_lam_n) {
  perk_status s = prepare_reverse(ctx);
  if (s != PERK_OK) return s;
  const void* key[4] = {d_Un, K, d_lam_np1, d_lam_n};
  if (!std::equal(key, key + 4, ctx->rev_key) || ctx->rev_dt != dt || ctx->rev_recompute != recompute) {
    ctx->rev_valid = false;
    std::copy(key, key + 4, ctx->rev_key);
    ctx->rev_dt = dt;
    ctx->rev_recompute = recompute;
  }
  return run_captured(ctx, ctx->graph_rev, ctx->rev_valid, [&](cudaStream_t st) {
    if (recompute) {
      perk_status r = enqueue_stages(ctx, st, d_Un, const_cast<double*>(K), nullptr);
      if (r != PERK_OK) return r;
    }
    return enqueue_reverse(ctx, st, d_Un, dt, K, d_lam_np1, d_lam_n);
  });
}

perk_status perk_step_vjp_stored(perk_ctx* ctx, const double* d_Un, double dt, const double* d_K,
                                 const double* d_lam_np1, double* d_lam_n) {
  if (!ctx) return PERK_E_INVALID_ARG;
  perk_status s = step_ready_adjoint(ctx, d_Un, dt);
  if (s != PERK_OK) return s;
  if (!d_K || !d_lam_np1 || !d_lam_n || d_lam_n == d_lam_np1)
    return fail(ctx, PERK_E_INVALID_ARG, "bad arguments (lam_n and lam_np1 must be distinct)");
  return run_reverse(ctx, d_Un, dt, d_K, false, d_lam_np1, d_lam_n);
}

perk_status perk_step_vjp(perk_ctx* ctx, const double* d_Un, double dt, const double* d_lam_np1, double* d_lam_n) {
  if (!ctx) return PERK_E_INVALID_ARG;
  perk_status s = step_ready_adjoint(ctx, d_Un, dt);
  if (s != PERK_OK) return s;
  if (!d_lam_np1 || !d_lam_n || d_lam_n == d_lam_np1)
    return fail(ctx, PERK_E_INVALID_ARG, "bad arguments (lam_n and lam_np1 must be distinct)");
  PERK_CUDA(ctx, ctx->d_Kall.ensure((size_t)ctx->n_elem * ELEM * ctx->S));
  return run_reverse(ctx, d_Un, dt, ctx->d_Kall.p, true, d_lam_np1, d_lam_n);
}

perk_status perk_set_volume_blocks(perk_ctx* ctx, int32_t elems_per_block) {
  if (!ctx) return PERK_E_INVALID_ARG;
  if (elems_per_block != 2 && elems_per_block != 4 && elems_per_block != 8)
    return fail(ctx, PERK_E_INVALID_ARG, "elements per block must be 2, 4 or 8");
  if (elems_per_block != ctx->vol_epb) {
    ctx->vol_epb = elems_per_block;
    drop_graph(ctx);
  }
  return PERK_OK;
}

perk_status perk_autotune_volume(perk_ctx* ctx, const double* d_U, int32_t* elems_per_block) {
  if (!ctx) return PERK_E_INVALID_ARG;
  if (!ctx->has_mesh || !ctx->partitioned) return fail(ctx, PERK_E_NOT_READY, "no mesh");
  if (!d_U) return fail(ctx, PERK_E_INVALID_ARG, "null U");
  const size_t nd = (size_t)ctx->n_elem * ELEM;
  PERK_CUDA(ctx, ctx->d_Ka.ensure(nd));   // scratch output: a stage buffer, free between steps
  DevBuf<double>& K = ctx->d_Ka;
  StageArgs sa{};
  sa.Y = d_U;
  cudaStream_t st = ctx->stream;
  PERK_CUDA(ctx, launch_faces(st, Y_GIVEN, ctx->ops, ctx->n_if, ctx->d_if_sorted.p, ctx->n_mort,
                              ctx->d_mort_sorted.p, ctx->d_method.p, sa, ctx->d_surf.p));
  cudaEvent_t a = nullptr, b = nullptr;
  PERK_CUDA(ctx, cudaEventCreate(&a));
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return fail(ctx, PERK_E_CUDA, "event creation failed");
  }
  const int cand[3] = {2, 4, 8};
  float best_ms = 0.f;
  int best = VOL_EPB_DEFAULT;
  cudaError_t err = cudaSuccess;
  for (int k = 0; k < 3 && err == cudaSuccess; ++k) {
    // one untimed launch, then five timed ones over every element of the mesh
    err = launch_volume(st, Y_GIVEN, ctx->ops, ctx->n_elem, ctx->d_elem_sorted.p, ctx->d_level.p, ctx->d_method.p,
                        2.0 / ctx->length, sa, ctx->d_surf.p, K.p, nullptr, ctx->d_logtab.p, cand[k]);
    if (err == cudaSuccess) err = cudaEventRecord(a, st);
    for (int r = 0; r < 5 && err == cudaSuccess; ++r)
      err = launch_volume(st, Y_GIVEN, ctx->ops, ctx->n_elem, ctx->d_elem_sorted.p, ctx->d_level.p, ctx->d_method.p,
                          2.0 / ctx->length, sa, ctx->d_surf.p, K.p, nullptr, ctx->d_logtab.p, cand[k]);
    if (err == cudaSuccess) err = cudaEventRecord(b, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(b);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, a, b);
    if (err == cudaSuccess && (k == 0 || ms < best_ms)) {
      best_ms = ms;
      best = cand[k];
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  PERK_CUDA(ctx, err);
  if (best != ctx->vol_epb) {
    ctx->vol_epb = best;
    drop_graph(ctx);   // the next step re-captures its launches
  }
  if (elems_per_block) *elems_per_block = best;
  return PERK_OK;
}

perk_status perk_autotune_step(perk_ctx* ctx, const double* d_U, const double* dts, int32_t* mode) {
  if (!ctx) return PERK_E_INVALID_ARG;
  if (!ctx->has_mesh || !ctx->has_tab || !ctx->partitioned || ctx->part_S != ctx->S)
    return fail(ctx, PERK_E_NOT_READY, "mesh or tableau missing");
  if (!d_U || !dts) return fail(ctx, PERK_E_INVALID_ARG, "null U or dt");
  perk_status s = set_dts(ctx, dts, 0.0);
  if (s != PERK_OK) return s;
  s = prepare_step(ctx);
  if (s != PERK_OK) return s;
  cudaStream_t st = ctx->stream;
  PERK_CUDA(ctx, cudaMemcpyAsync(&ctx->h_pin->flag, ctx->d_flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  PERK_CUDA(ctx, cudaStreamSynchronize(st));
  if (ctx->h_pin->flag != 0) return fail(ctx, PERK_E_NOT_READY, "a rejected step is pending: call perk_check first");
  const bool old_stage = ctx->fuse_stage, old_step = ctx->fuse_step;
  int cand[3], nc = 0;
  ctx->fuse_stage = true;
  if (ctx->stage_fused()) {
    cand[nc++] = 1;
    ctx->fuse_step = true;
    if (ctx->step_fused()) cand[nc++] = 2;
  }
  cand[nc++] = 0;
  int best = cand[0];
  float best_ms = 0.f;
  cudaError_t err = cudaSuccess;
  cudaEvent_t a = nullptr, b = nullptr;
  if (nc > 1) {
    err = cudaEventCreate(&a);
    if (err == cudaSuccess) err = cudaEventCreate(&b);
    for (int k = 0; k < nc && err == cudaSuccess; ++k) {
      ctx->fuse_stage = cand[k] != 0;
      ctx->fuse_step = cand[k] == 2;
      // one untimed and five timed steps from the same U: the admissibility flag is raised
      // before each, so the final update (which still restarts the stage counters and
      // advances the step count) leaves U unchanged
      for (int r = 0; r < 6 && err == cudaSuccess; ++r) {
        err = cudaMemsetAsync(ctx->d_flag.p, 1, sizeof(int), st);
        if (err == cudaSuccess && r == 1) err = cudaEventRecord(a, st);
        if (err == cudaSuccess && enqueue_step(ctx, st, const_cast<double*>(d_U)) != PERK_OK) err = cudaErrorUnknown;
      }
      if (err == cudaSuccess) err = cudaEventRecord(b, st);
      if (err == cudaSuccess) err = cudaEventSynchronize(b);
      float ms = 0.f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, a, b);
      if (err == cudaSuccess && (k == 0 || ms < best_ms)) {
        best_ms = ms;
        best = cand[k];
      }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
  ctx->fuse_stage = best != 0;
  ctx->fuse_step = best == 2;
  if (ctx->fuse_stage != old_stage || ctx->fuse_step != old_step) drop_graph(ctx);
  const cudaError_t clear = cudaMemsetAsync(ctx->d_flag.p, 0, sizeof(int), st);
  const cudaError_t sync = cudaStreamSynchronize(st);
  PERK_CUDA(ctx, err);
  PERK_CUDA(ctx, clear);
  PERK_CUDA(ctx, sync);
  if (mode) *mode = best;
  return PERK_OK;
}

perk_status perk_selftest_math(perk_ctx* ctx, int64_t n, const double* d_x, double* d_out) {
  if (!ctx || !d_x || !d_out || n < 0) return PERK_E_INVALID_ARG;
  PERK_CUDA(ctx, launch_selftest_math(ctx->stream, n, d_x, d_out, ctx->d_logtab.p));
  return PERK_OK;
}

perk_status perk_amr_indicator(perk_ctx* ctx, int32_t indicator, const double* d_U, double* d_eta) {
  if (!ctx || !d_U || !d_eta) return PERK_E_INVALID_ARG;
  if (!ctx->has_mesh) return fail(ctx, PERK_E_NOT_READY, "no mesh");
  if (indicator != PERK_INDICATOR_DENSITY && indicator != PERK_INDICATOR_LOHNER_VX)
    return fail(ctx, PERK_E_INVALID_ARG, "unknown indicator %d", indicator);
  std::vector<double> x, w;
  lgl(NN - 1, x, w);
  PERK_CUDA(ctx, launch_indicator(ctx->stream, ctx->n_elem, d_U, ctx->ops, w[0], w[1], indicator, d_eta));
  return PERK_OK;
}

// perk_adapt_plan on the device (a mesh in member-major Morton order): desired levels from the
// indicator (or the caller's), balance, and the new leaves' offsets; only the new cell count and
// whether anything changes come back to the host.
static perk_status adapt_plan_device(perk_ctx* ctx, const perk_amr_params* prm, const int32_t* desired,
                                     const double* d_U, int64_t* n_new) {
  const int64_t n = ctx->n_elem;
  cudaStream_t st = ctx->stream;
  PERK_CUDA(ctx, ctx->d_des.ensure((size_t)n));
  PERK_CUDA(ctx, ctx->d_off.ensure((size_t)n + 1));
  PERK_CUDA(ctx, ctx->d_info.ensure(8));
  AmrPlanArgs a{0, 0, 0.0, 0.0};
  const double* eta = nullptr;
  if (desired) {
    PERK_CUDA(ctx, cudaMemcpyAsync(ctx->d_des.p, desired, n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  } else {
    std::vector<double> x, w;
    lgl(NN - 1, x, w);
    PERK_CUDA(ctx, launch_indicator(st, n, d_U, ctx->ops, w[0], w[1], prm->indicator, ctx->d_eta.p));
    a = AmrPlanArgs{prm->level_min, prm->level_max, prm->refine_above, prm->coarsen_below};
    eta = ctx->d_eta.p;
  }
  PERK_CUDA(ctx, launch_amr_plan(st, n, ctx->d_cells.p, eta, a, ctx->n_if, ctx->d_if_raw.p, ctx->n_mort,
                                 ctx->d_mort_raw.p, ctx->d_des.p, ctx->d_off.p, ctx->d_info.p));
  const int64_t* info = ctx->h_pin->info;
  PERK_CUDA(ctx, cudaMemcpyAsync(ctx->h_pin->info, ctx->d_info.p, 5 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  PERK_CUDA(ctx, cudaStreamSynchronize(st));
  if (info[4] != 0) return fail(ctx, PERK_E_CUDA, "AMR balance did not settle within its pass bound");
  ctx->plan_device = true;
  ctx->plan_n_new = info[0];
  ctx->plan_identity = info[1] == 0;
  ctx->has_plan = true;
  *n_new = info[0];
  return PERK_OK;
}

perk_status perk_adapt_plan(perk_ctx* ctx, const perk_amr_params* prm, const int32_t* desired, const double* d_U,
                            int64_t* n_new) {
  if (!ctx || !n_new) return PERK_E_INVALID_ARG;
  if (!ctx->has_mesh) return fail(ctx, PERK_E_NOT_READY, "no mesh");
  ctx->has_plan = false;
  ctx->plan_device = false;
  const int64_t n = ctx->n_elem;
  if (desired || ctx->host_stale || !ctx->mesh_morton) {
    perk_status s = sync_host_mesh(ctx);   // the desired levels are checked against the host's levels
    if (s != PERK_OK) return s;
  }
  const int32_t* c = ctx->h_cells.data();
  if (desired) {
    for (int64_t e = 0; e < n; ++e)
      if (desired[e] < c[3 * e] - 1 || desired[e] > c[3 * e] + 1 || desired[e] < 0 || desired[e] > 27)
        return fail(ctx, PERK_E_INVALID_ARG, "desired level of cell %lld must differ by at most one", (long long)e);
  } else {
    if (!prm || !d_U) return fail(ctx, PERK_E_INVALID_ARG, "need AMR parameters and U");
    if (prm->indicator != PERK_INDICATOR_DENSITY && prm->indicator != PERK_INDICATOR_LOHNER_VX)
      return fail(ctx, PERK_E_INVALID_ARG, "unknown indicator %d", prm->indicator);
  }
  if (ctx->mesh_morton) return adapt_plan_device(ctx, prm, desired, d_U, n_new);
  std::vector<int32_t> d(n);
  if (desired) {
    for (int64_t e = 0; e < n; ++e) d[e] = desired[e];
  } else {
    std::vector<double> x, w;
    lgl(NN - 1, x, w);
    PERK_CUDA(ctx, launch_indicator(ctx->stream, n, d_U, ctx->ops, w[0], w[1], prm->indicator, ctx->d_eta.p));
    std::vector<double> eta(n);
    PERK_CUDA(ctx, cudaMemcpyAsync(eta.data(), ctx->d_eta.p, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    PERK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int64_t e = 0; e < n; ++e) {
      const int l = c[3 * e];
      d[e] = l;
      if (eta[e] > prm->refine_above && l < prm->level_max)
        d[e] = l + 1;
      else if (eta[e] < prm->coarsen_below && l > prm->level_min && !(eta[e] > prm->refine_above))
        d[e] = l - 1;
    }
  }
  balance_levels(ctx, d);
  bool identity = true;
  for (int64_t e = 0; e < n && identity; ++e) identity = d[e] == c[3 * e];
  ctx->plan_identity = identity;
  // new leaves (member by member, Morton order within a member) and transfer records
  const int32_t* mb = ctx->h_member.data();
  FlatMap old((size_t)n);
  for (int64_t e = 0; e < n; ++e) old.insert(key_of(mb[e], c[3 * e], c[3 * e + 1], c[3 * e + 2]).v, (int32_t)e);
  struct NewCell {
    int32_t m, l, ix, iy;
  };
  std::vector<NewCell> nc;
  nc.reserve((size_t)n * 2);
  FlatMap seen((size_t)n);
  std::vector<int> lmax(ctx->n_members, 0);
  for (int64_t e = 0; e < n; ++e) {
    const int l = c[3 * e], ix = c[3 * e + 1], iy = c[3 * e + 2], me = mb[e];
    if (d[e] == l + 1) {
      for (int cy = 0; cy < 2; ++cy)
        for (int cx = 0; cx < 2; ++cx) nc.push_back({me, l + 1, 2 * ix + cx, 2 * iy + cy});
    } else if (d[e] == l) {
      nc.push_back({me, l, ix, iy});
    } else if (seen.insert(key_of(me, l - 1, ix >> 1, iy >> 1).v, 1)) {
      nc.push_back({me, l - 1, ix >> 1, iy >> 1});
    }
    lmax[me] = std::max(lmax[me], d[e]);
  }
  struct Ord {
    int32_t m;
    uint64_t z;
    int64_t k;
    bool operator<(const Ord& o) const { return m != o.m ? m < o.m : z < o.z; }
  };
  std::vector<Ord> order(nc.size());
  for (size_t k = 0; k < nc.size(); ++k)
    order[k] = {nc[k].m, morton_key(nc[k].l, nc[k].ix, nc[k].iy, lmax[nc[k].m]), (int64_t)k};
  // leaves generated from a Morton-ordered mesh are already in order
  if (!std::is_sorted(order.begin(), order.end())) std::sort(order.begin(), order.end());
  const int64_t m = (int64_t)nc.size();
  ctx->plan_cells.resize(3 * m);
  ctx->plan_member.resize(m);
  ctx->plan_map.resize(5 * m);
  for (int64_t k = 0; k < m; ++k) {
    const NewCell& q = nc[order[k].k];
    ctx->plan_cells[3 * k] = q.l;
    ctx->plan_cells[3 * k + 1] = q.ix;
    ctx->plan_cells[3 * k + 2] = q.iy;
    ctx->plan_member[k] = q.m;
    int32_t* r = &ctx->plan_map[5 * k];
    const int32_t it = old.find(key_of(q.m, q.l, q.ix, q.iy).v);
    if (it >= 0) {
      r[0] = 0;
      r[1] = it;
      r[2] = r[3] = r[4] = 0;
      continue;
    }
    const int32_t par = q.l > 0 ? old.find(key_of(q.m, q.l - 1, q.ix >> 1, q.iy >> 1).v) : -1;
    if (par >= 0) {
      r[0] = 1 | ((q.ix & 1) << 2) | ((q.iy & 1) << 3);
      r[1] = par;
      r[2] = r[3] = r[4] = 0;
      continue;
    }
    r[0] = 2;
    for (int cc = 0; cc < 4; ++cc) {
      const int32_t ch = old.find(key_of(q.m, q.l + 1, 2 * q.ix + (cc & 1), 2 * q.iy + (cc >> 1)).v);
      if (ch < 0) return fail(ctx, PERK_E_INVALID_ARG, "internal: missing child in AMR plan");
      r[1 + cc] = ch;
    }
  }
  ctx->has_plan = true;
  *n_new = m;
  return PERK_OK;
}

// perk_adapt_commit of a device plan: new leaves, transfer, connectivity and partition on the
// device; the host receives the counts the launches need (one synchronisation)
static perk_status adapt_commit_device(perk_ctx* ctx, const double* d_Uold, double* d_Unew) {
  const int64_t n = ctx->n_elem, m = ctx->plan_n_new;
  cudaStream_t st = ctx->stream;
  if (ctx->ws_base && m > ctx->ws_cells)
    return fail(ctx, PERK_E_OOM,
                "the adapted mesh has %lld cells, the bound workspace serves up to %lld: bind a larger one "
                "(perk_workspace_bytes) and commit again", (long long)m, (long long)ctx->ws_cells);
  // Every buffer of the new mesh is sized before the first launch of this call (the plan left the
  // stream empty, so no reallocation frees memory that queued work still reads).  The old leaves
  // (d_cells), desired levels and offsets keep their sizes: the new-leaf kernel reads them.
  const size_t mm = (size_t)m;
  PERK_CUDA(ctx, grow(ctx->d_newcells, mm));
  PERK_CUDA(ctx, grow(ctx->d_key, mm));
  PERK_CUDA(ctx, grow(ctx->d_map, 5 * mm));
  PERK_CUDA(ctx, grow(ctx->d_level, mm));
  PERK_CUDA(ctx, grow(ctx->d_member, mm));
  PERK_CUDA(ctx, grow(ctx->d_method, mm));
  PERK_CUDA(ctx, grow(ctx->d_elem_sorted, mm));
  PERK_CUDA(ctx, grow(ctx->d_if_raw, 2 * mm));
  PERK_CUDA(ctx, grow(ctx->d_if_sorted, 2 * mm));
  PERK_CUDA(ctx, grow(ctx->d_mort_raw, 2 * mm));
  PERK_CUDA(ctx, grow(ctx->d_mort_sorted, 2 * mm));
  PERK_CUDA(ctx, grow(ctx->d_cnt_if, mm));
  PERK_CUDA(ctx, grow(ctx->d_cnt_mort, mm));
  PERK_CUDA(ctx, grow(ctx->d_off_if, mm));
  PERK_CUDA(ctx, grow(ctx->d_off_mort, mm));
  PERK_CUDA(ctx, grow(ctx->d_surf, mm * ELEM));
  PERK_CUDA(ctx, grow(ctx->d_K1, mm * ELEM));
  PERK_CUDA(ctx, grow(ctx->d_Ka, mm * ELEM));
  PERK_CUDA(ctx, grow(ctx->d_Kb, mm * ELEM));
  PERK_CUDA(ctx, grow(ctx->d_eta, mm));
  if (ctx->viscous()) {
    PERK_CUDA(ctx, grow(ctx->d_wsurf, mm * 64));
    PERK_CUDA(ctx, grow(ctx->d_q, mm * 128));
    PERK_CUDA(ctx, grow(ctx->d_vsurf, mm * 64));
  }
  PERK_CUDA(ctx, grow(ctx->d_stamp, 4 * mm));
  PERK_CUDA(ctx, cudaMemsetAsync(ctx->d_stamp.p, 0, 4 * mm * sizeof(unsigned long long), st));
  PERK_CUDA(ctx, grow(ctx->d_prog, mm));
  PERK_CUDA(ctx, cudaMemsetAsync(ctx->d_prog.p, 0, mm * sizeof(unsigned long long), st));
  PERK_CUDA(ctx, launch_amr_leaves(st, n, ctx->d_cells.p, ctx->d_des.p, ctx->d_off.p, ctx->d_newcells.p,
                                   ctx->d_key.p, ctx->d_map.p));
  PERK_CUDA(ctx, launch_transfer(st, m, ctx->d_map.p, d_Uold, ctx->ops, d_Unew));
  std::swap(ctx->d_cells, ctx->d_newcells);
  PERK_CUDA(ctx, launch_amr_install(st, m, ctx->d_cells.p, ctx->d_level.p, ctx->d_member.p));
  PERK_CUDA(ctx, launch_connect(st, m, ctx->d_cells.p, ctx->d_key.p, ctx->d_cnt_if.p, ctx->d_cnt_mort.p,
                                ctx->d_off_if.p, ctx->d_off_mort.p, ctx->d_if_raw.p, ctx->d_mort_raw.p, ctx->d_info.p));
  drop_graph(ctx);
  ctx->has_plan = false;
  ctx->plan_device = false;
  ctx->n_elem = m;
  ctx->n_if = 2 * m;     // upper bounds until the partition brings the counts back
  ctx->n_mort = 2 * m;
  ctx->host_stale = true;
  ctx->mesh_morton = true;
  return run_partition(ctx, true);
}

perk_status perk_adapt_commit_dt(perk_ctx* ctx, const double* d_Uold, double* d_Unew, double cfl, double* dt) {
  if (!ctx) return PERK_E_INVALID_ARG;
  if (!dt || !(cfl > 0.0)) return fail(ctx, PERK_E_INVALID_ARG, "bad cfl or null dt");
  ctx->pending_dt_U = d_Unew;
  ctx->dt_folded = false;
  const perk_status s = perk_adapt_commit(ctx, d_Uold, d_Unew);
  const bool folded = ctx->dt_folded;
  ctx->pending_dt_U = nullptr;
  ctx->dt_folded = false;
  if (s != PERK_OK) return s;
  if (!folded) return perk_compute_dt(ctx, d_Unew, cfl, dt);   // the commit read nothing back
  const double m = ctx->h_pin->dt;
  if (!std::isfinite(m) || !(m > 0.0))
    return fail(ctx, PERK_E_NONFINITE, "a node has no admissible wave speed (rho or p <= 0, or NaN)");
  *dt = cfl * m / (double)NN;
  return PERK_OK;
}

perk_status perk_adapt_commit(perk_ctx* ctx, const double* d_Uold, double* d_Unew) {
  if (!ctx) return PERK_E_INVALID_ARG;
  if (!ctx->has_plan) return fail(ctx, PERK_E_NOT_READY, "no AMR plan");
  if (!d_Uold || !d_Unew || d_Uold == d_Unew) return fail(ctx, PERK_E_INVALID_ARG, "need distinct old and new U");
  if (ctx->plan_device && !ctx->plan_identity) return adapt_commit_device(ctx, d_Uold, d_Unew);
  const int64_t m = ctx->plan_device ? ctx->plan_n_new : (int64_t)ctx->plan_cells.size() / 3;
  if (ctx->plan_identity) {
    // nothing changes: the new state is a copy and the mesh, partition and graph stay
    PERK_CUDA(ctx, cudaMemcpyAsync(d_Unew, d_Uold, (size_t)m * ELEM * sizeof(double), cudaMemcpyDeviceToDevice,
                                   ctx->stream));
    ctx->has_plan = false;
    ctx->plan_device = false;
    ctx->plan_cells.clear();
    ctx->plan_member.clear();
    return PERK_OK;
  }
  if (ctx->ws_base && m > ctx->ws_cells)
    return fail(ctx, PERK_E_OOM,
                "the adapted mesh has %lld cells, the bound workspace serves up to %lld: bind a larger one "
                "(perk_workspace_bytes) and commit again", (long long)m, (long long)ctx->ws_cells);
  PERK_CUDA(ctx, ctx->d_map.ensure((size_t)5 * m));
  PERK_CUDA(ctx, cudaMemcpyAsync(ctx->d_map.p, ctx->plan_map.data(), ctx->plan_map.size() * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, ctx->stream));
  // (the pageable upload above is staged before the call returns, so plan_map may be reused)
  PERK_CUDA(ctx, launch_transfer(ctx->stream, m, ctx->d_map.p, d_Uold, ctx->ops, d_Unew));
  ctx->has_plan = false;
  const std::vector<int32_t> cells = std::move(ctx->plan_cells);
  const std::vector<int32_t> members = std::move(ctx->plan_member);
  ctx->plan_cells.clear();
  ctx->plan_member.clear();
  return set_mesh(ctx, m, cells.data(), ctx->n_members > 1 ? members.data() : nullptr, ctx->x0, ctx->length);
}

perk_status perk_amr_balance(int64_t n_cells, const int32_t* cells, const int32_t* desired, int32_t* levels) {
  if (n_cells <= 0 || !cells || !desired || !levels) return fail(nullptr, PERK_E_INVALID_ARG, "bad arguments");
  // the host state balance_levels reads, in a context that owns no device memory
  perk_ctx tmp;
  std::vector<int4> ifs, morts;
  if (build_connectivity(nullptr, n_cells, cells, nullptr, ifs, morts) != PERK_OK) return PERK_E_INVALID_ARG;
  tmp.n_elem = n_cells;
  tmp.h_cells.assign(cells, cells + 3 * n_cells);
  tmp.h_member.assign(n_cells, 0);
  tmp.h_if = std::move(ifs);
  tmp.h_mort = std::move(morts);
  std::vector<int32_t> d(n_cells);
  for (int64_t e = 0; e < n_cells; ++e) {
    const int l = cells[3 * e];
    if (desired[e] < l - 1 || desired[e] > l + 1 || desired[e] < 0 || desired[e] > 27)
      return fail(nullptr, PERK_E_INVALID_ARG, "desired level of cell %lld must differ by at most one", (long long)e);
    d[e] = desired[e];
  }
  balance_levels(&tmp, d);
  std::copy(d.begin(), d.end(), levels);
  return PERK_OK;
}

perk_status perk_get_cells(const perk_ctx* ctx, int32_t* cells, int64_t cap) {
  if (!ctx || !cells) return PERK_E_INVALID_ARG;
  if (!ctx->has_mesh) return PERK_E_NOT_READY;
  if (cap < ctx->n_elem) return PERK_E_INVALID_ARG;
  {
    perk_status s = sync_host_mesh(const_cast<perk_ctx*>(ctx));
    if (s != PERK_OK) return s;
  }
  std::copy(ctx->h_cells.begin(), ctx->h_cells.end(), cells);
  return PERK_OK;
}

perk_status perk_workspace_bytes(const perk_ctx* ctx, int64_t n_cells, size_t* bytes) {
  if (!ctx || !bytes) return PERK_E_INVALID_ARG;
  perk_ctx* c = const_cast<perk_ctx*>(ctx);   // the layout walk reads the buffers' types only
  if (n_cells < 0 || n_cells > ((int64_t)1 << 30)) return fail(c, PERK_E_INVALID_ARG, "bad cell count");
  if (n_cells == 0) n_cells = std::max<int64_t>(ctx->n_elem, 1);
  *bytes = workspace_layout_bytes(c, n_cells);
  return PERK_OK;
}

perk_status perk_bind_workspace(perk_ctx* ctx, void* d_ws, size_t bytes) {
  if (!ctx) return PERK_E_INVALID_ARG;
  const bool unbind = d_ws == nullptr && bytes == 0;
  if (!unbind && (!d_ws || ((uintptr_t)d_ws % WS_ALIGN) != 0))
    return fail(ctx, PERK_E_INVALID_ARG, "the workspace must be device memory aligned to %d bytes", (int)WS_ALIGN);
  const int64_t need = std::max<int64_t>(ctx->n_elem, 1);
  int64_t cells = need;
  if (!unbind) {
    const size_t need_bytes = workspace_layout_bytes(ctx, need);
    if (bytes < need_bytes)
      return fail(ctx, PERK_E_INVALID_ARG, "workspace of %zu bytes; the current mesh needs %zu", bytes, need_bytes);
    // the largest mesh the block serves (the layout grows with the cell count)
    int64_t lo = need, hi = (int64_t)1 << 30;
    while (lo < hi) {
      const int64_t mid = lo + (hi - lo + 1) / 2;
      if (workspace_layout_bytes(ctx, mid) <= bytes)
        lo = mid;
      else
        hi = mid - 1;
    }
    cells = lo;
  }
  // move every covered buffer's contents to its new place (the workspace, or fresh allocations),
  // then let go of the old memory
  PERK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  struct Old {
    void* p;
    bool ext;
  };
  std::vector<Old> old;
  std::vector<const void*> moved;
  cudaError_t err = cudaSuccess;
  size_t off = 0;
  for_each_workspace_buffer(ctx, cells, [&](auto& b, size_t count) {
    moved.push_back(&b);
    using T = std::remove_reference_t<decltype(*b.p)>;
    if (err != cudaSuccess) return;
    T* np = nullptr;
    if (unbind) {
      err = cudaMalloc(&np, count * sizeof(T));
      if (err != cudaSuccess) return;
      ctx->counters.device_allocations += 1;
    } else {
      off = ws_align(off);
      np = reinterpret_cast<T*>(static_cast<char*>(d_ws) + off);
      off += count * sizeof(T);
    }
    if (b.p && b.cap) err = cudaMemcpyAsync(np, b.p, std::min(b.cap, count) * sizeof(T), cudaMemcpyDeviceToDevice,
                                            ctx->stream);
    old.push_back({b.p, b.ext});
    b.p = np;
    b.cap = count;
    b.ext = !unbind;
  });
  const cudaError_t sync = cudaStreamSynchronize(ctx->stream);
  for (const Old& o : old)
    if (o.p && !o.ext) cudaFree(o.p);
  // buffers of another mode left in a previous block (scratch only): allocated afresh when needed
  for_each_buffer(ctx, [&](auto& b) {
    if (b.ext && std::find(moved.begin(), moved.end(), (const void*)&b) == moved.end()) {
      b.p = nullptr;
      b.cap = 0;
      b.ext = false;
    }
  });
  PERK_CUDA(ctx, err);
  PERK_CUDA(ctx, sync);
  ctx->ws_base = unbind ? nullptr : static_cast<char*>(d_ws);
  ctx->ws_bytes = unbind ? 0 : bytes;
  ctx->ws_cells = unbind ? 0 : cells;
  destroy_graph(ctx);   // the step's buffers moved
  return PERK_OK;
}

perk_status perk_get_counters(const perk_ctx* ctx, perk_counters* out) {
  if (!ctx || !out) return PERK_E_INVALID_ARG;
  *out = ctx->counters;
  return PERK_OK;
}

}  // extern "C"
