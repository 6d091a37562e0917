// Host runtime of the 3D path: the C ABI declared in include/perk3d.h.
//
// Owns the hexahedral reference operators, the octree connectivity built from a
// leaf-cell list (interfaces and 2:1 face mortars with four small cells), the
// device copies of the mesh and of the level partition (the partition kernel of
// the 2D path, with three geometry bits in mortar records), the coefficient
// table and the stage buffers, and drives one P-ERK step as 2S + 1 launches,
// optionally replayed from a CUDA graph.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "perk3d_internal.h"

using namespace perk3;
using perk::MAX_R;
using perk::MAX_S;

namespace {

template <typename T>
struct Buf {
  T* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t n) {
    if (n <= cap && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) cap = std::max<size_t>(n, 1);
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

constexpr int MAX_LEVEL3 = 19;

// Operators of degree N on the hexahedron: the split-form derivative matrix, 1/w_0, and the
// 1D mortar interpolation and exact L2 projection matrices of the two halves of an edge (a face
// mortar applies them along both tangential axes).
bool build_ops3(int N, double gamma, int surface_flux, Ops3& o) {
  const int nn = N + 1;
  o = Ops3{};
  o.nn = nn;
  std::vector<double> x, w;
  perk::lgl(N, x, w);
  std::vector<double> lam(nn);
  for (int j = 0; j < nn; ++j) {
    double p = 1.0;
    for (int k = 0; k < nn; ++k)
      if (k != j) p *= x[j] - x[k];
    lam[j] = 1.0 / p;
  }
  for (int i = 0; i < nn; ++i)
    for (int j = 0; j < nn; ++j) o.dsplit[i][j] = (i == j) ? 0.0 : 2.0 * (lam[j] / lam[i]) / (x[i] - x[j]);
  for (int i = 0; i < nn; ++i) {
    double row = 0.0;
    for (int j = 0; j < nn; ++j)
      if (j != i) {
        o.dmat[i][j] = 0.5 * o.dsplit[i][j];
        row += o.dmat[i][j];
      }
    o.dmat[i][i] = -row;   // a derivative matrix annihilates constants
  }
  o.inv_w0 = 1.0 / w[0];
  for (int k = 0; k < nn; ++k) {
    perk::lagrange_values(x, 0.5 * (x[k] - 1.0), o.p_lo[k]);
    perk::lagrange_values(x, 0.5 * (x[k] + 1.0), o.p_hi[k]);
  }
  // exact mass matrix (nn Gauss points integrate degree 2N exactly) and its inverse
  std::vector<double> xg, wg;
  perk::gauss_legendre(nn, xg, wg);
  double M[MAXNN][MAXNN] = {}, A[MAXNN][2 * MAXNN] = {};
  for (int g = 0; g < nn; ++g) {
    double L[MAXNN];
    perk::lagrange_values(x, xg[g], L);
    for (int a = 0; a < nn; ++a)
      for (int b = 0; b < nn; ++b) M[a][b] += wg[g] * L[a] * L[b];
  }
  for (int a = 0; a < nn; ++a)
    for (int b = 0; b < 2 * nn; ++b) A[a][b] = b < nn ? M[a][b] : (b - nn == a ? 1.0 : 0.0);
  for (int c = 0; c < nn; ++c) {
    int piv = c;
    for (int r = c + 1; r < nn; ++r)
      if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
    if (A[piv][c] == 0.0) return false;
    for (int b = 0; b < 2 * nn; ++b) std::swap(A[c][b], A[piv][b]);
    const double d = A[c][c];
    for (int b = 0; b < 2 * nn; ++b) A[c][b] /= d;
    for (int r = 0; r < nn; ++r)
      if (r != c) {
        const double f = A[r][c];
        for (int b = 0; b < 2 * nn; ++b) A[r][b] -= f * A[c][b];
      }
  }
  // R_h = 1/2 M^{-1} P_h^T M: the L2 projection of a half-edge polynomial onto the edge
  for (int h = 0; h < 2; ++h) {
    const double(*P)[MAXNN] = h ? o.p_hi : o.p_lo;
    double(*R)[MAXNN] = h ? o.r_hi : o.r_lo;
    double PtM[MAXNN][MAXNN] = {};
    for (int a = 0; a < nn; ++a)
      for (int b = 0; b < nn; ++b)
        for (int c = 0; c < nn; ++c) PtM[a][b] += P[c][a] * M[c][b];
    for (int a = 0; a < nn; ++a)
      for (int b = 0; b < nn; ++b) {
        double s = 0.0;
        for (int c = 0; c < nn; ++c) s += A[a][nn + c] * PtM[c][b];
        R[a][b] = 0.5 * s;
      }
  }
  o.gamma = gamma;
  o.gm1 = gamma - 1.0;
  o.inv_gm1 = 1.0 / (gamma - 1.0);
  o.surface_flux = surface_flux;
  return true;
}

// level (5 bits) | ix | iy | iz (19 bits each)
inline uint64_t key3(int l, int64_t x, int64_t y, int64_t z) {
  return ((uint64_t)l << 57) | ((uint64_t)x << 38) | ((uint64_t)y << 19) | (uint64_t)z;
}

// Morton key of a leaf's lower corner at resolution lmax (bits interleaved x, y, z)
uint64_t morton3(int l, int64_t x, int64_t y, int64_t z, int lmax) {
  const int s = lmax - l;
  x <<= s;
  y <<= s;
  z <<= s;
  uint64_t m = 0;
  for (int b = 0; b < 21; ++b) {
    m |= (uint64_t)((x >> b) & 1) << (3 * b);
    m |= (uint64_t)((y >> b) & 1) << (3 * b + 1);
    m |= (uint64_t)((z >> b) & 1) << (3 * b + 2);
  }
  return m;
}

struct Conn {
  std::vector<int4> ifs;      // (left, right, dir, 0)
  std::vector<int4> morts;    // (large, s0, table index, dir | large_side << 2)
  std::vector<int4> msmall;   // four small cells by quadrant q1 + 2 q2
};

// Interfaces and mortars of a periodic, 2:1-balanced octree leaf list by a walk over each
// leaf's six face neighbourhoods.  Returns an empty string on success, else the error.
std::string build_connectivity3(int64_t n, const int32_t* cells, Conn& c) {
  std::unordered_map<uint64_t, int32_t> leaf;
  leaf.reserve((size_t)n * 2);
  int lmax = 0;
  char buf[160];
  for (int64_t e = 0; e < n; ++e) {
    const int l = cells[4 * e];
    if (l < 0 || l > MAX_LEVEL3) {
      snprintf(buf, sizeof buf, "cell %lld: level %d out of range", (long long)e, l);
      return buf;
    }
    const int64_t side = (int64_t)1 << l;
    for (int d = 0; d < 3; ++d) {
      const int64_t v = cells[4 * e + 1 + d];
      if (v < 0 || v >= side) {
        snprintf(buf, sizeof buf, "cell %lld: index outside level %d", (long long)e, l);
        return buf;
      }
    }
    lmax = std::max(lmax, l);
    if (!leaf.emplace(key3(l, cells[4 * e + 1], cells[4 * e + 2], cells[4 * e + 3]), (int32_t)e).second) {
      snprintf(buf, sizeof buf, "cell %lld duplicated", (long long)e);
      return buf;
    }
  }
  // exact tiling: the Morton intervals at the finest level follow each other from 0 to 8^lmax
  {
    std::vector<std::pair<uint64_t, uint64_t>> iv((size_t)n);
    for (int64_t e = 0; e < n; ++e) {
      const int l = cells[4 * e];
      const uint64_t z = morton3(l, cells[4 * e + 1], cells[4 * e + 2], cells[4 * e + 3], lmax);
      iv[e] = {z, z + (1ull << (3 * (lmax - l)))};
    }
    std::sort(iv.begin(), iv.end());
    uint64_t next = 0;
    for (const auto& q : iv) {
      if (q.first != next) return "cells overlap or leave a gap";
      next = q.second;
    }
    if (next != (1ull << (3 * lmax))) return "cells do not tile the cube";
  }
  auto find = [&](int l, int64_t x, int64_t y, int64_t z) -> int32_t {
    if (l < 0 || l > MAX_LEVEL3) return -1;
    auto it = leaf.find(key3(l, x, y, z));
    return it == leaf.end() ? -1 : it->second;
  };
  for (int64_t e = 0; e < n; ++e) {
    const int l = cells[4 * e];
    const int64_t side = (int64_t)1 << l;
    const int64_t p[3] = {cells[4 * e + 1], cells[4 * e + 2], cells[4 * e + 3]};
    for (int d = 0; d < 3; ++d) {
      const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
      for (int s = 0; s < 2; ++s) {   // s = 0: the +d neighbourhood, s = 1: the -d one
        int64_t q[3] = {p[0], p[1], p[2]};
        q[d] = s == 0 ? (p[d] + 1) % side : (p[d] + side - 1) % side;
        const int32_t same = find(l, q[0], q[1], q[2]);
        if (same >= 0) {
          if (s == 0) c.ifs.push_back(make_int4((int)e, same, d, 0));   // built once, from the - side
          continue;
        }
        if (l > 0 && find(l - 1, q[0] >> 1, q[1] >> 1, q[2] >> 1) >= 0) continue;   // small side of a mortar
        // the neighbourhood is refined once: its four children against this face
        int32_t sm[4];
        for (int b = 0; b < 2; ++b)
          for (int a = 0; a < 2; ++a) {
            int64_t ch[3];
            ch[d] = 2 * q[d] + (s == 0 ? 0 : 1);
            ch[t1] = 2 * q[t1] + a;
            ch[t2] = 2 * q[t2] + b;
            sm[a + 2 * b] = find(l + 1, ch[0], ch[1], ch[2]);
          }
        if (sm[0] < 0 || sm[1] < 0 || sm[2] < 0 || sm[3] < 0) {
          snprintf(buf, sizeof buf, "mesh not 2:1 balanced at cell %lld", (long long)e);
          return buf;
        }
        const int idx = (int)c.msmall.size();
        c.msmall.push_back(make_int4(sm[0], sm[1], sm[2], sm[3]));
        c.morts.push_back(make_int4((int)e, sm[0], idx, d | (s << 2)));
      }
    }
  }
  return std::string();
}

}  // namespace

struct perk3d_ctx {
  perk3d_problem prob{};
  Ops3 ops{};
  int nn = 3;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  std::string err;

  bool has_mesh = false;
  int64_t n_elem = 0, n_if = 0, n_mort = 0;
  double x0 = 0.0, length = 1.0;
  std::vector<int32_t> h_level;
  std::vector<int32_t> h_cells;                 // [n_elem][4] (level, ix, iy, iz)
  std::vector<std::pair<int32_t, int32_t>> h_pairs;   // face neighbours (interfaces; large-small of mortars)

  // pending AMR plan (perk3d_adapt_plan -> perk3d_adapt_commit)
  bool has_plan = false, plan_identity = false;
  int64_t plan_n = 0;                           // cells of the planned mesh
  std::vector<int32_t> plan_cells, plan_map;    // [m][4], [m][9]
  Buf<int32_t> d_map;
  Buf<double> d_eta;

  bool has_tab = false;
  int order = 2, S = 0, R = 0;
  int32_t E[MAX_R] = {};
  int32_t stage_minmem[MAX_S] = {};
  std::vector<double> c, a;
  double w_b1 = 0.0, w_bp = 0.0, w_bs = 1.0;

  bool partitioned = false;
  int part_S = 0;
  int32_t lmin = 0, lmax = 0;
  int64_t act_el[MAX_S] = {}, act_if[MAX_S] = {}, act_mort[MAX_S] = {};
  // per stage, the prefixes of the one-level halo of the active members (BR1 gradients)
  int64_t halo_el[MAX_S] = {}, halo_if[MAX_S] = {}, halo_mort[MAX_S] = {};
  bool viscous() const { return prob.equations == PERK_NAVIER_STOKES; }
  double kappa() const { return prob.mu * prob.gamma / ((prob.gamma - 1.0) * prob.prandtl); }
  Buf<double> d_q;   // BR1 viscous fluxes [n_elem][3 axes][5][n^3]

  Buf<int32_t> d_level, d_method, d_elem_sorted, d_minmem, d_minmax, d_member_lmax;
  Buf<int4> d_if_raw, d_mort_raw, d_if_sorted, d_mort_sorted, d_msmall;
  Buf<int64_t> d_counts;
  Buf<double> d_surf, d_K1, d_Ka, d_Kb, d_dt, d_dt_out, d_logtab;
  Buf<StageCoef> d_coef;
  Buf<int> d_flag;

  cudaGraphExec_t graph = nullptr;
  bool graph_valid = false;
  double* graph_U = nullptr;
  double cur_dt = NAN;

  perk_counters counters{};
};

namespace {

thread_local std::string g_err3;

perk_status fail(perk3d_ctx* ctx, perk_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx)
    ctx->err = buf;
  else
    g_err3 = buf;
  return s;
}

#define P3_CUDA(ctx, call)                                                                          \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? PERK_E_OOM : PERK_E_CUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                               \
  } while (0)

perk_status run_partition3(perk3d_ctx* ctx) {
  if (!ctx->has_mesh) return fail(ctx, PERK_E_NOT_READY, "no mesh");
  int R = 1, S = 1;
  int32_t minmem[MAX_S] = {0};
  if (ctx->has_tab) {
    R = ctx->R;
    S = ctx->S;
    std::copy(ctx->stage_minmem, ctx->stage_minmem + MAX_S, minmem);
  }
  P3_CUDA(ctx, cudaMemcpyAsync(ctx->d_minmem.p, minmem, sizeof minmem, cudaMemcpyHostToDevice, ctx->stream));
  P3_CUDA(ctx, perk::launch_partition(ctx->stream, ctx->n_elem, ctx->n_if, ctx->n_mort, ctx->d_level.p,
                                      ctx->d_if_raw.p, ctx->d_mort_raw.p, R, S, ctx->d_minmem.p, nullptr, 1,
                                      ctx->d_member_lmax.p, ctx->d_method.p, ctx->d_elem_sorted.p,
                                      ctx->d_if_sorted.p, ctx->d_mort_sorted.p, ctx->d_counts.p, ctx->d_minmax.p,
                                      MORT_FLAG_BITS));
  int64_t counts[6 * MAX_S];
  int32_t mm[2];
  P3_CUDA(ctx, cudaMemcpyAsync(counts, ctx->d_counts.p, sizeof counts, cudaMemcpyDeviceToHost, ctx->stream));
  P3_CUDA(ctx, cudaMemcpyAsync(mm, ctx->d_minmax.p, sizeof mm, cudaMemcpyDeviceToHost, ctx->stream));
  P3_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
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
  ctx->graph_valid = false;
  return PERK_OK;
}

StageArgs combine_args(perk3d_ctx* ctx, int stage, double* d_U, const double* Kp) {
  StageArgs sa{};
  sa.U = d_U;
  sa.K1 = ctx->d_K1.p;
  sa.Kp = Kp;
  sa.coef = ctx->d_coef.p + (size_t)stage * MAX_R;
  sa.dt = ctx->d_dt.p;
  return sa;
}

// the launches of one step on stream st (also under graph capture); timer: per-kind events
struct Timer3 {
  std::vector<cudaEvent_t> ev;
  std::vector<int> kind;
  ~Timer3() {
    for (auto e : ev) cudaEventDestroy(e);
  }
  cudaError_t mark(cudaStream_t st) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    ev.push_back(e);
    return cudaEventRecord(e, st);
  }
};

#define P3_TIMED(ctx, timer, st, k, call)        \
  do {                                           \
    if (timer) P3_CUDA(ctx, (timer)->mark(st));  \
    P3_CUDA(ctx, call);                          \
    if (timer) {                                 \
      P3_CUDA(ctx, (timer)->mark(st));           \
      (timer)->kind.push_back(k);                \
    }                                            \
  } while (0)

perk_status enqueue_step3(perk3d_ctx* ctx, cudaStream_t st, double* d_U, Timer3* timer = nullptr) {
  const int S = ctx->S;
  double* Kbuf[3] = {ctx->d_K1.p, ctx->d_Ka.p, ctx->d_Kb.p};
  int prev = 0, cur = 0;
  double* K_before_last = ctx->d_K1.p;
  UpdateArgs ua{};
  ua.b1 = ctx->w_b1;
  ua.bp = ctx->w_bp;
  ua.bs = ctx->w_bs;
  ua.U = d_U;
  ua.K1 = ctx->d_K1.p;
  ua.flag = ctx->d_flag.p;
  const double two_over_len = 2.0 / ctx->length;
  for (int i = 0; i < S; ++i) {
    cur = (i == 0) ? 0 : (i % 2 == 1 ? 1 : 2);
    const StageArgs sa = combine_args(ctx, i, d_U, Kbuf[prev]);
    P3_TIMED(ctx, timer, st, 0,
             launch_faces3(st, perk::Y_COMBINE, ctx->ops, ctx->act_if[i], ctx->d_if_sorted.p, ctx->act_mort[i],
                           ctx->d_mort_sorted.p, ctx->d_msmall.p, ctx->d_method.p, sa, ctx->d_logtab.p,
                           ctx->d_surf.p));
    const bool last = i == S - 1;
    if (last) K_before_last = Kbuf[prev];
    UpdateArgs chk = ua;
    chk.Kp = K_before_last;
    const bool visc = ctx->viscous();
    P3_TIMED(ctx, timer, st, 1,
             launch_volume3(st, perk::Y_COMBINE, ctx->ops, ctx->act_el[i], ctx->d_elem_sorted.p, ctx->d_level.p,
                            ctx->d_method.p, two_over_len, sa, ctx->d_surf.p, Kbuf[cur],
                            (last && !visc) ? &chk : nullptr, ctx->d_logtab.p));
    if (visc)
      P3_TIMED(ctx, timer, st, 3,
               launch_br1_3d(st, perk::Y_COMBINE, ctx->ops, ctx->prob.mu, ctx->kappa(), ctx->halo_if[i],
                             ctx->halo_mort[i], ctx->act_if[i], ctx->act_mort[i], ctx->d_if_sorted.p,
                             ctx->d_mort_sorted.p, ctx->d_msmall.p, ctx->halo_el[i], ctx->act_el[i],
                             ctx->d_elem_sorted.p, ctx->d_level.p, ctx->d_method.p, two_over_len, sa, ctx->d_surf.p,
                             ctx->d_q.p, Kbuf[cur], last ? &chk : nullptr));
    prev = cur;
  }
  ua.Kp = K_before_last;
  P3_TIMED(ctx, timer, st, 2,
           launch_commit3(st, ctx->n_elem * elem3(ctx->nn), ua, Kbuf[cur], ctx->d_dt.p, d_U));
  return PERK_OK;
}

perk_status upload_coef3(perk3d_ctx* ctx) {
  std::vector<StageCoef> coef((size_t)MAX_S * MAX_R, StageCoef{0.0, 0.0, 0, 0});
  for (int i = 1; i < ctx->S; ++i)
    for (int r = 0; r < ctx->R; ++r) {
      const double beta = ctx->a[(size_t)r * ctx->S + i];
      coef[(size_t)i * MAX_R + r] = StageCoef{ctx->c[i] - beta, beta, i - 1, 0};
    }
  P3_CUDA(ctx, cudaMemcpyAsync(ctx->d_coef.p, coef.data(), coef.size() * sizeof(StageCoef), cudaMemcpyHostToDevice,
                               ctx->stream));
  P3_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return PERK_OK;
}

perk_status set_dt3(perk3d_ctx* ctx, double dt) {
  if (!std::isfinite(dt) || !(dt > 0.0)) return fail(ctx, PERK_E_INVALID_ARG, "bad dt");
  if (ctx->cur_dt == dt) return PERK_OK;
  ctx->cur_dt = dt;
  // pageable source: the value is staged before the call returns
  P3_CUDA(ctx, cudaMemcpyAsync(ctx->d_dt.p, &ctx->cur_dt, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  return PERK_OK;
}

perk_status step_ready3(perk3d_ctx* ctx, double* d_U) {
  if (!ctx->has_mesh || !ctx->has_tab || !ctx->partitioned || ctx->part_S != ctx->S)
    return fail(ctx, PERK_E_NOT_READY, "mesh or tableau missing");
  if (!d_U) return fail(ctx, PERK_E_INVALID_ARG, "null U");
  if (((uintptr_t)d_U & 15) != 0) return fail(ctx, PERK_E_INVALID_ARG, "U must be 16-byte aligned");
  return PERK_OK;
}

void count_step3(perk3d_ctx* ctx) {
  ctx->counters.steps += 1;
  for (int i = 0; i < ctx->S; ++i) {
    ctx->counters.element_stage_evaluations += ctx->act_el[i];
    ctx->counters.dof_stage_updates += ctx->act_el[i] * nodes3(ctx->nn);
  }
}

// One AMR plan on the host (the part of perk3d_adapt_plan after the desired levels): d (one level
// per cell, within one of the cell's) raised in place to the least fixed point of the sibling rule
// (eight leaves of one parent coarsen together) and the 2:1 rule across the face pairs; the new
// leaves in Morton order (new_cells [m][4]) and their transfer records (map [m][9]: kind | child
// bits, then the source cells).  False only if a coarsened parent misses a child, which a tiling
// of the cube rules out.
bool plan_cells3(int64_t n, const int32_t* c, const std::vector<std::pair<int32_t, int32_t>>& pairs,
                 std::vector<int32_t>& d, bool* identity_out, std::vector<int32_t>& new_cells,
                 std::vector<int32_t>& map) {
  std::unordered_map<uint64_t, int32_t> gid;
  std::vector<int32_t> group_of(n, -1), gcount, gmembers;
  for (int64_t e = 0; e < n; ++e) {
    const int l = c[4 * e];
    if (l == 0) continue;
    const uint64_t k = key3(l, c[4 * e + 1] >> 1, c[4 * e + 2] >> 1, c[4 * e + 3] >> 1);
    auto it = gid.find(k);
    int32_t g;
    if (it == gid.end()) {
      g = (int32_t)gcount.size();
      gid.emplace(k, g);
      gcount.push_back(0);
      gmembers.insert(gmembers.end(), 8, -1);
    } else {
      g = it->second;
    }
    if (gcount[g] < 8) gmembers[8 * g + gcount[g]] = (int32_t)e;
    gcount[g] += 1;
    group_of[e] = g;
  }
  bool changed = true;
  while (changed) {
    changed = false;
    for (int64_t e = 0; e < n; ++e) {
      if (d[e] >= c[4 * e]) continue;
      const int32_t g = group_of[e];
      bool ok = g >= 0 && gcount[g] == 8;
      for (int q = 0; ok && q < 8; ++q) ok = d[gmembers[8 * g + q]] < c[4 * gmembers[8 * g + q]];
      if (ok) continue;
      if (g < 0) {
        d[e] = c[4 * e];
        changed = true;
        continue;
      }
      for (int q = 0; q < 8 && q < gcount[g]; ++q) {
        const int32_t m = gmembers[8 * g + q];
        if (d[m] < c[4 * m]) {
          d[m] = c[4 * m];
          changed = true;
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
  bool identity = true;
  for (int64_t e = 0; e < n && identity; ++e) identity = d[e] == c[4 * e];
  *identity_out = identity;
  // new leaves (Morton order) and transfer records
  std::unordered_map<uint64_t, int32_t> old;
  old.reserve((size_t)n * 2);
  int lmax = 0;
  for (int64_t e = 0; e < n; ++e) {
    old.emplace(key3(c[4 * e], c[4 * e + 1], c[4 * e + 2], c[4 * e + 3]), (int32_t)e);
    lmax = std::max(lmax, d[e]);
  }
  struct NewCell {
    int32_t l, x, y, z;
  };
  std::vector<NewCell> nc;
  nc.reserve((size_t)n * 2);
  std::unordered_map<uint64_t, int32_t> seen;
  for (int64_t e = 0; e < n; ++e) {
    const int l = c[4 * e], x = c[4 * e + 1], y = c[4 * e + 2], z = c[4 * e + 3];
    if (d[e] == l + 1) {
      for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
          for (int cx = 0; cx < 2; ++cx) nc.push_back({l + 1, 2 * x + cx, 2 * y + cy, 2 * z + cz});
    } else if (d[e] == l) {
      nc.push_back({l, x, y, z});
    } else if (seen.emplace(key3(l - 1, x >> 1, y >> 1, z >> 1), 1).second) {
      nc.push_back({l - 1, x >> 1, y >> 1, z >> 1});
    }
  }
  std::vector<std::pair<uint64_t, int64_t>> order(nc.size());
  for (size_t k = 0; k < nc.size(); ++k) order[k] = {morton3(nc[k].l, nc[k].x, nc[k].y, nc[k].z, lmax), (int64_t)k};
  std::sort(order.begin(), order.end());
  const int64_t m = (int64_t)nc.size();
  new_cells.resize(4 * m);
  map.assign(9 * m, 0);
  for (int64_t k = 0; k < m; ++k) {
    const NewCell& q = nc[order[k].second];
    int32_t* cc = &new_cells[4 * k];
    cc[0] = q.l;
    cc[1] = q.x;
    cc[2] = q.y;
    cc[3] = q.z;
    int32_t* r = &map[9 * k];
    auto it = old.find(key3(q.l, q.x, q.y, q.z));
    if (it != old.end()) {
      r[0] = 0;
      r[1] = it->second;
      continue;
    }
    auto par = q.l > 0 ? old.find(key3(q.l - 1, q.x >> 1, q.y >> 1, q.z >> 1)) : old.end();
    if (par != old.end()) {
      r[0] = 1 | ((q.x & 1) << 2) | ((q.y & 1) << 3) | ((q.z & 1) << 4);
      r[1] = par->second;
      continue;
    }
    r[0] = 2;
    for (int ch = 0; ch < 8; ++ch) {
      auto ci = old.find(key3(q.l + 1, 2 * q.x + (ch & 1), 2 * q.y + ((ch >> 1) & 1), 2 * q.z + (ch >> 2)));
      if (ci == old.end()) return false;
      r[1 + ch] = ci->second;
    }
  }
  return true;
}

}  // namespace

extern "C" {

perk_status perk3d_create(const perk3d_problem* prob, perk3d_ctx** out) {
  if (!prob || !out) return fail(nullptr, PERK_E_INVALID_ARG, "null argument");
  *out = nullptr;
  if ((prob->N != 2 && prob->N != 3) || !(prob->gamma > 1.0) || prob->surface_flux < 0 || prob->surface_flux > 3)
    return fail(nullptr, PERK_E_INVALID_ARG, "N must be 2 or 3, gamma > 1, and the surface flux known");
  if (prob->equations != PERK_EULER && prob->equations != PERK_NAVIER_STOKES)
    return fail(nullptr, PERK_E_INVALID_ARG, "unknown equations %d", prob->equations);
  if (prob->equations == PERK_NAVIER_STOKES && (!(prob->mu > 0.0) || !(prob->prandtl > 0.0)))
    return fail(nullptr, PERK_E_INVALID_ARG, "Navier-Stokes needs mu > 0 and Pr > 0");
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) {
    cudaGetLastError();
    return fail(nullptr, PERK_E_CUDA, "no CUDA device");
  }
  perk3d_ctx* ctx = new perk3d_ctx();
  ctx->prob = *prob;
  ctx->nn = prob->N + 1;
  perk::device_sm_count();   // cached before any graph capture
  if (!build_ops3(prob->N, prob->gamma, prob->surface_flux, ctx->ops)) {
    delete ctx;
    return fail(nullptr, PERK_E_INVALID_ARG, "singular mass matrix");
  }
  if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      ctx->d_dt.ensure(1) != cudaSuccess || ctx->d_dt_out.ensure(1) != cudaSuccess ||
      ctx->d_flag.ensure(1) != cudaSuccess || ctx->d_logtab.ensure(2 * perk::LOG_TABLE_SIZE) != cudaSuccess ||
      ctx->d_counts.ensure(6 * MAX_S) != cudaSuccess || ctx->d_minmax.ensure(2) != cudaSuccess ||
      ctx->d_minmem.ensure(MAX_S) != cudaSuccess || ctx->d_member_lmax.ensure(1) != cudaSuccess ||
      ctx->d_coef.ensure((size_t)MAX_S * MAX_R) != cudaSuccess) {
    perk3d_destroy(ctx);
    return fail(nullptr, PERK_E_CUDA, "allocation of the context's buffers failed");
  }
  const std::vector<double> t = perk::log_table();
  if (cudaMemset(ctx->d_flag.p, 0, sizeof(int)) != cudaSuccess ||
      cudaMemcpy(ctx->d_logtab.p, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    perk3d_destroy(ctx);
    return fail(nullptr, PERK_E_CUDA, "initialisation of the context's buffers failed");
  }
  *out = ctx;
  return PERK_OK;
}

void perk3d_destroy(perk3d_ctx* ctx) {
  if (!ctx) return;
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  for (auto* b : {&ctx->d_level, &ctx->d_method, &ctx->d_elem_sorted, &ctx->d_minmem, &ctx->d_minmax,
                  &ctx->d_member_lmax, &ctx->d_map})
    b->release();
  ctx->d_eta.release();
  ctx->d_q.release();
  for (auto* b : {&ctx->d_if_raw, &ctx->d_mort_raw, &ctx->d_if_sorted, &ctx->d_mort_sorted, &ctx->d_msmall})
    b->release();
  for (auto* b : {&ctx->d_surf, &ctx->d_K1, &ctx->d_Ka, &ctx->d_Kb, &ctx->d_dt, &ctx->d_dt_out, &ctx->d_logtab})
    b->release();
  ctx->d_counts.release();
  ctx->d_coef.release();
  ctx->d_flag.release();
  delete ctx;
}

const char* perk3d_last_error(const perk3d_ctx* ctx) { return ctx ? ctx->err.c_str() : g_err3.c_str(); }

perk_status perk3d_set_stream(perk3d_ctx* ctx, void* stream) {
  if (!ctx) return PERK_E_INVALID_ARG;
  ctx->stream = (cudaStream_t)stream;
  return PERK_OK;
}

perk_status perk3d_mesh_faces(int64_t n_cells, const int32_t* cells, int64_t* n_if, int32_t* ifs, int64_t if_cap,
                              int64_t* n_mort, int32_t* morts, int64_t mort_cap) {
  if (n_cells <= 0 || !cells || !n_if || !n_mort) return fail(nullptr, PERK_E_INVALID_ARG, "bad arguments");
  Conn c;
  const std::string e = build_connectivity3(n_cells, cells, c);
  if (!e.empty()) return fail(nullptr, PERK_E_INVALID_ARG, "%s", e.c_str());
  *n_if = (int64_t)c.ifs.size();
  *n_mort = (int64_t)c.morts.size();
  if (ifs && if_cap >= *n_if)
    for (size_t q = 0; q < c.ifs.size(); ++q) {
      ifs[4 * q] = c.ifs[q].x;
      ifs[4 * q + 1] = c.ifs[q].y;
      ifs[4 * q + 2] = c.ifs[q].z;
      ifs[4 * q + 3] = 0;
    }
  if (morts && mort_cap >= *n_mort)
    for (size_t q = 0; q < c.morts.size(); ++q) {
      const int4 s = c.msmall[c.morts[q].z];
      const int32_t rec[6] = {c.morts[q].x, s.x, s.y, s.z, s.w, c.morts[q].w};
      std::copy(rec, rec + 6, morts + 6 * q);
    }
  return PERK_OK;
}

perk_status perk3d_mesh_upload(perk3d_ctx* ctx, int64_t n_cells, const int32_t* cells, double x0, double length) {
  if (!ctx) return PERK_E_INVALID_ARG;
  if (n_cells <= 0 || !cells || !(length > 0.0) || !std::isfinite(x0))
    return fail(ctx, PERK_E_INVALID_ARG, "bad mesh arguments");
  if (n_cells > (int64_t)1 << 30) return fail(ctx, PERK_E_INVALID_ARG, "too many cells");
  Conn c;
  const std::string e = build_connectivity3(n_cells, cells, c);
  if (!e.empty()) return fail(ctx, PERK_E_INVALID_ARG, "%s", e.c_str());
  ctx->graph_valid = false;
  ctx->has_mesh = false;
  ctx->partitioned = false;
  ctx->n_elem = n_cells;
  ctx->n_if = (int64_t)c.ifs.size();
  ctx->n_mort = (int64_t)c.morts.size();
  ctx->x0 = x0;
  ctx->length = length;
  ctx->h_level.resize(n_cells);
  for (int64_t q = 0; q < n_cells; ++q) ctx->h_level[q] = cells[4 * q];
  ctx->h_cells.assign(cells, cells + 4 * n_cells);
  ctx->h_pairs.clear();
  ctx->h_pairs.reserve(c.ifs.size() + 4 * c.morts.size());
  for (const int4& f : c.ifs) ctx->h_pairs.emplace_back(f.x, f.y);
  for (const int4& m : c.morts) {
    const int4 sm = c.msmall[m.z];
    for (int32_t q : {sm.x, sm.y, sm.z, sm.w}) ctx->h_pairs.emplace_back(m.x, q);
  }
  ctx->has_plan = false;
  const size_t ne = (size_t)n_cells;
  P3_CUDA(ctx, ctx->d_level.ensure(ne));
  P3_CUDA(ctx, ctx->d_method.ensure(ne));
  P3_CUDA(ctx, ctx->d_elem_sorted.ensure(ne));
  P3_CUDA(ctx, ctx->d_if_raw.ensure(c.ifs.size()));
  P3_CUDA(ctx, ctx->d_if_sorted.ensure(c.ifs.size()));
  P3_CUDA(ctx, ctx->d_mort_raw.ensure(c.morts.size()));
  P3_CUDA(ctx, ctx->d_mort_sorted.ensure(c.morts.size()));
  P3_CUDA(ctx, ctx->d_msmall.ensure(c.msmall.size()));
  P3_CUDA(ctx, ctx->d_surf.ensure(ne * surf3(ctx->nn)));
  P3_CUDA(ctx, ctx->d_K1.ensure(ne * elem3(ctx->nn)));
  P3_CUDA(ctx, ctx->d_Ka.ensure(ne * elem3(ctx->nn)));
  P3_CUDA(ctx, ctx->d_Kb.ensure(ne * elem3(ctx->nn)));
  P3_CUDA(ctx, ctx->d_eta.ensure(ne));
  if (ctx->viscous()) P3_CUDA(ctx, ctx->d_q.ensure(ne * 15 * nodes3(ctx->nn)));
  P3_CUDA(ctx, cudaMemcpyAsync(ctx->d_level.p, ctx->h_level.data(), ne * sizeof(int32_t), cudaMemcpyHostToDevice,
                               ctx->stream));
  if (!c.ifs.empty())
    P3_CUDA(ctx, cudaMemcpyAsync(ctx->d_if_raw.p, c.ifs.data(), c.ifs.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                 ctx->stream));
  if (!c.morts.empty()) {
    P3_CUDA(ctx, cudaMemcpyAsync(ctx->d_mort_raw.p, c.morts.data(), c.morts.size() * sizeof(int4),
                                 cudaMemcpyHostToDevice, ctx->stream));
    P3_CUDA(ctx, cudaMemcpyAsync(ctx->d_msmall.p, c.msmall.data(), c.msmall.size() * sizeof(int4),
                                 cudaMemcpyHostToDevice, ctx->stream));
  }
  // the host vectors go out of scope: wait for the pageable copies to be consumed
  P3_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->has_mesh = true;
  return run_partition3(ctx);
}

perk_status perk3d_mesh_query(const perk3d_ctx* ctx, perk_mesh_info* info) {
  if (!ctx || !info) return PERK_E_INVALID_ARG;
  std::memset(info, 0, sizeof *info);
  info->n_elem = ctx->n_elem;
  info->n_interfaces = ctx->n_if;
  info->n_mortars = ctx->n_mort;
  info->level_min = ctx->lmin;
  info->level_max = ctx->lmax;
  info->S = ctx->has_tab ? ctx->S : 0;
  for (int i = 0; i < MAX_S && i < ctx->part_S; ++i) {
    info->active_elements[i] = ctx->act_el[i];
    info->active_interfaces[i] = ctx->act_if[i];
    info->active_mortars[i] = ctx->act_mort[i];
    if (i < info->S) info->dof_stage_updates += ctx->act_el[i] * nodes3(ctx->nn);
  }
  info->index_bytes = (int64_t)(ctx->n_elem * 2 * sizeof(int32_t) + ctx->n_if * sizeof(int4) +
                                ctx->n_mort * 2 * sizeof(int4));
  return PERK_OK;
}

perk_status perk3d_set_tableau(perk3d_ctx* ctx, int order, int S, int R, const int32_t* E, const double* c,
                               const double* a) {
  if (!ctx) return PERK_E_INVALID_ARG;
  if ((order != 2 && order != 3) || S < 1 || S > MAX_S || R < 1 || R > MAX_R || !E || !c || !a)
    return fail(ctx, PERK_E_INVALID_ARG, "invalid tableau dimensions");
  if (order == 3 && S < 3) return fail(ctx, PERK_E_INVALID_ARG, "third order needs S >= 3");
  for (int r = 0; r < R; ++r)
    if (E[r] < 1 || E[r] > S || (r > 0 && E[r] < E[r - 1]))
      return fail(ctx, PERK_E_INVALID_ARG, "member evaluations must ascend within [1, S]");
  if (E[R - 1] != S) return fail(ctx, PERK_E_INVALID_ARG, "the largest member must evaluate every stage");
  for (int r = 0; r < R; ++r)
    for (int i0 = 1; i0 < S; ++i0) {
      const bool evaluated = (i0 == 1) || (i0 >= S - E[r] + 2);
      if (!evaluated && a[(size_t)r * S + i0] != 0.0)
        return fail(ctx, PERK_E_INVALID_ARG, "member %d: a_{%d,%d} != 0 but stage %d is not evaluated", r, i0 + 1,
                    i0, i0);
    }
  ctx->order = order;
  ctx->S = S;
  ctx->R = R;
  ctx->w_b1 = order == 3 ? 1.0 / 6.0 : 0.0;
  ctx->w_bp = order == 3 ? 1.0 / 6.0 : 0.0;
  ctx->w_bs = order == 3 ? 2.0 / 3.0 : 1.0;
  std::copy(E, E + R, ctx->E);
  ctx->c.assign(c, c + S);
  ctx->a.assign(a, a + (size_t)R * S);
  // member r is active at stage i >= 1 iff E[r] >= S - i + 1; the coarsest active member per stage
  for (int i = 0; i < MAX_S; ++i) {
    int mm = R;
    for (int r = R - 1; r >= 0; --r)
      if (i == 0 || E[r] >= S - i + 1) mm = r;
    ctx->stage_minmem[i] = i < S ? mm : R;
  }
  ctx->has_tab = true;
  ctx->graph_valid = false;
  perk_status s = upload_coef3(ctx);
  if (s != PERK_OK) return s;
  if (ctx->has_mesh) return run_partition3(ctx);
  return PERK_OK;
}

static perk_status rhs_given3(perk3d_ctx* ctx, int stage, const double* d_Y, double* d_K) {
  if (!ctx->has_mesh || !ctx->partitioned) return fail(ctx, PERK_E_NOT_READY, "no mesh");
  if (!d_Y || !d_K) return fail(ctx, PERK_E_INVALID_ARG, "null array");
  StageArgs sa{};
  sa.Y = d_Y;
  const int64_t ne = stage < 0 ? ctx->n_elem : ctx->act_el[stage];
  const int64_t ni = stage < 0 ? ctx->n_if : ctx->act_if[stage];
  const int64_t nm = stage < 0 ? ctx->n_mort : ctx->act_mort[stage];
  P3_CUDA(ctx, launch_faces3(ctx->stream, perk::Y_GIVEN, ctx->ops, ni, ctx->d_if_sorted.p, nm, ctx->d_mort_sorted.p,
                             ctx->d_msmall.p, ctx->d_method.p, sa, ctx->d_logtab.p, ctx->d_surf.p));
  P3_CUDA(ctx, launch_volume3(ctx->stream, perk::Y_GIVEN, ctx->ops, ne, ctx->d_elem_sorted.p, ctx->d_level.p,
                              ctx->d_method.p, 2.0 / ctx->length, sa, ctx->d_surf.p, d_K, nullptr, ctx->d_logtab.p));
  if (ctx->viscous())
    P3_CUDA(ctx, launch_br1_3d(ctx->stream, perk::Y_GIVEN, ctx->ops, ctx->prob.mu, ctx->kappa(),
                               stage < 0 ? ctx->n_if : ctx->halo_if[stage],
                               stage < 0 ? ctx->n_mort : ctx->halo_mort[stage], ni, nm, ctx->d_if_sorted.p,
                               ctx->d_mort_sorted.p, ctx->d_msmall.p, stage < 0 ? ctx->n_elem : ctx->halo_el[stage],
                               ne, ctx->d_elem_sorted.p, ctx->d_level.p, ctx->d_method.p, 2.0 / ctx->length, sa,
                               ctx->d_surf.p, ctx->d_q.p, d_K, nullptr));
  return PERK_OK;
}

perk_status perk3d_rhs_full(perk3d_ctx* ctx, const double* d_Y, double* d_K) {
  if (!ctx) return PERK_E_INVALID_ARG;
  return rhs_given3(ctx, -1, d_Y, d_K);
}

perk_status perk3d_rhs_active(perk3d_ctx* ctx, int stage, const double* d_Y, double* d_K) {
  if (!ctx) return PERK_E_INVALID_ARG;
  if (!ctx->has_tab) return fail(ctx, PERK_E_NOT_READY, "no tableau");
  if (stage < 0 || stage >= ctx->S) return fail(ctx, PERK_E_INVALID_ARG, "stage %d outside [0, %d)", stage, ctx->S);
  return rhs_given3(ctx, stage, d_Y, d_K);
}

perk_status perk3d_step(perk3d_ctx* ctx, double* d_U, double dt) {
  if (!ctx) return PERK_E_INVALID_ARG;
  perk_status s = step_ready3(ctx, d_U);
  if (s != PERK_OK) return s;
  s = set_dt3(ctx, dt);
  if (s != PERK_OK) return s;
  if (ctx->prob.use_graph) {
    if (!ctx->graph_valid || ctx->graph_U != d_U) {
      cudaGraph_t g = nullptr;
      P3_CUDA(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
      s = enqueue_step3(ctx, ctx->cap_stream, d_U);
      cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &g);
      if (s != PERK_OK) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return s;
      }
      P3_CUDA(ctx, ce);
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
      P3_CUDA(ctx, ie);
      ctx->graph_U = d_U;
      ctx->graph_valid = true;
    }
    P3_CUDA(ctx, cudaGraphLaunch(ctx->graph, ctx->stream));
  } else {
    s = enqueue_step3(ctx, ctx->stream, d_U);
    if (s != PERK_OK) return s;
  }
  count_step3(ctx);
  return PERK_OK;
}

perk_status perk3d_step_profiled(perk3d_ctx* ctx, double* d_U, double dt, perk_kernel_times* acc) {
  if (!ctx || !acc) return PERK_E_INVALID_ARG;
  perk_status s = step_ready3(ctx, d_U);
  if (s != PERK_OK) return s;
  s = set_dt3(ctx, dt);
  if (s != PERK_OK) return s;
  Timer3 timer;
  s = enqueue_step3(ctx, ctx->stream, d_U, &timer);
  if (s != PERK_OK) return s;
  P3_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (size_t q = 0; q < timer.kind.size(); ++q) {
    float ms = 0.0f;
    P3_CUDA(ctx, cudaEventElapsedTime(&ms, timer.ev[2 * q], timer.ev[2 * q + 1]));
    acc->ms[timer.kind[q]] += ms;
    acc->launches[timer.kind[q]] += 1;
  }
  for (int i = 0; i < ctx->S; ++i) acc->element_stages += ctx->act_el[i];
  count_step3(ctx);
  return PERK_OK;
}

perk_status perk3d_check(perk3d_ctx* ctx) {
  if (!ctx) return PERK_E_INVALID_ARG;
  int flag = 0;
  P3_CUDA(ctx, cudaMemcpyAsync(&flag, ctx->d_flag.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  P3_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (flag) {
    P3_CUDA(ctx, cudaMemsetAsync(ctx->d_flag.p, 0, sizeof(int), ctx->stream));
    P3_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->counters.rejected_steps_checked += 1;
    return fail(ctx, PERK_E_NONFINITE, "a step produced an inadmissible state and was not committed");
  }
  return PERK_OK;
}

perk_status perk3d_compute_dt(perk3d_ctx* ctx, const double* d_U, double cfl, double* dt) {
  if (!ctx || !dt) return PERK_E_INVALID_ARG;
  if (!ctx->has_mesh) return fail(ctx, PERK_E_NOT_READY, "no mesh");
  if (!d_U || !(cfl > 0.0)) return fail(ctx, PERK_E_INVALID_ARG, "bad arguments");
  P3_CUDA(ctx, launch_dt3(ctx->stream, ctx->nn, ctx->n_elem, d_U, ctx->d_level.p, ctx->length, ctx->prob.gamma,
                          ctx->d_dt_out.p));
  double m = 0.0;
  P3_CUDA(ctx, cudaMemcpyAsync(&m, ctx->d_dt_out.p, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  P3_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (!std::isfinite(m) || !(m > 0.0)) return fail(ctx, PERK_E_NONFINITE, "no admissible wave speed");
  *dt = cfl * m;
  return PERK_OK;
}

perk_status perk3d_get_counters(const perk3d_ctx* ctx, perk_counters* out) {
  if (!ctx || !out) return PERK_E_INVALID_ARG;
  *out = ctx->counters;
  return PERK_OK;
}

perk_status perk3d_amr_indicator(perk3d_ctx* ctx, const double* d_U, double* d_eta) {
  if (!ctx) return PERK_E_INVALID_ARG;
  if (!ctx->has_mesh) return fail(ctx, PERK_E_NOT_READY, "no mesh");
  if (!d_U || !d_eta) return fail(ctx, PERK_E_INVALID_ARG, "null array");
  P3_CUDA(ctx, launch_enstrophy3(ctx->stream, ctx->ops, ctx->n_elem, d_U, ctx->d_level.p, 2.0 / ctx->length, d_eta));
  return PERK_OK;
}

perk_status perk3d_adapt_plan(perk3d_ctx* ctx, const perk3d_amr_params* prm, const int32_t* desired, const double* d_U,
                              int64_t* n_new) {
  if (!ctx || !n_new) return PERK_E_INVALID_ARG;
  if (!ctx->has_mesh) return fail(ctx, PERK_E_NOT_READY, "no mesh");
  const int64_t n = ctx->n_elem;
  const int32_t* c = ctx->h_cells.data();
  std::vector<int32_t> d(n);
  if (desired) {
    for (int64_t e = 0; e < n; ++e) {
      if (desired[e] < c[4 * e] - 1 || desired[e] > c[4 * e] + 1 || desired[e] < 0 || desired[e] > MAX_LEVEL3)
        return fail(ctx, PERK_E_INVALID_ARG, "desired level of cell %lld must differ by at most one", (long long)e);
      d[e] = desired[e];
    }
  } else {
    if (!prm || !d_U) return fail(ctx, PERK_E_INVALID_ARG, "need AMR parameters and U");
    if (prm->level_min < 0 || prm->level_max > MAX_LEVEL3 || prm->level_min > prm->level_max)
      return fail(ctx, PERK_E_INVALID_ARG, "bad level range");
    P3_CUDA(ctx, launch_enstrophy3(ctx->stream, ctx->ops, n, d_U, ctx->d_level.p, 2.0 / ctx->length, ctx->d_eta.p));
    std::vector<double> eta(n);
    P3_CUDA(ctx, cudaMemcpyAsync(eta.data(), ctx->d_eta.p, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    P3_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int64_t e = 0; e < n; ++e) {
      const int l = c[4 * e];
      d[e] = l;
      if (eta[e] > prm->refine_above && l < prm->level_max)
        d[e] = l + 1;
      else if (eta[e] < prm->coarsen_below && l > prm->level_min && !(eta[e] > prm->refine_above))
        d[e] = l - 1;
    }
  }
  // no cell asks for a change: the current (balanced) mesh is the fixed point, nothing to plan
  {
    bool same = true;
    for (int64_t e = 0; e < n && same; ++e) same = d[e] == c[4 * e];
    if (same) {
      ctx->plan_identity = true;
      ctx->plan_n = n;
      ctx->plan_cells.clear();
      ctx->has_plan = true;
      *n_new = n;
      return PERK_OK;
    }
  }
  bool identity = false;
  if (!plan_cells3(n, c, ctx->h_pairs, d, &identity, ctx->plan_cells, ctx->plan_map))
    return fail(ctx, PERK_E_INVALID_ARG, "internal: missing child in AMR plan");
  ctx->plan_identity = identity;
  const int64_t m = (int64_t)ctx->plan_cells.size() / 4;
  ctx->plan_n = m;
  ctx->has_plan = true;
  *n_new = m;
  return PERK_OK;
}

perk_status perk3d_adapt_commit(perk3d_ctx* ctx, const double* d_Uold, double* d_Unew) {
  if (!ctx) return PERK_E_INVALID_ARG;
  if (!ctx->has_plan) return fail(ctx, PERK_E_NOT_READY, "no AMR plan");
  if (!d_Uold || !d_Unew || d_Uold == d_Unew) return fail(ctx, PERK_E_INVALID_ARG, "need distinct old and new U");
  const int64_t m = ctx->plan_n;
  if (ctx->plan_identity) {
    P3_CUDA(ctx, cudaMemcpyAsync(d_Unew, d_Uold, (size_t)m * elem3(ctx->nn) * sizeof(double),
                                 cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->has_plan = false;
    return PERK_OK;
  }
  P3_CUDA(ctx, ctx->d_map.ensure((size_t)9 * m));
  P3_CUDA(ctx, cudaMemcpyAsync(ctx->d_map.p, ctx->plan_map.data(), ctx->plan_map.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, ctx->stream));
  P3_CUDA(ctx, launch_transfer3(ctx->stream, ctx->ops, m, ctx->d_map.p, d_Uold, d_Unew));
  ctx->has_plan = false;
  const std::vector<int32_t> cells = std::move(ctx->plan_cells);
  ctx->plan_cells.clear();
  return perk3d_mesh_upload(ctx, m, cells.data(), ctx->x0, ctx->length);
}

perk_status perk3d_amr_plan_cells(int64_t n_cells, const int32_t* cells, const int32_t* desired, int32_t* levels,
                                  int64_t* n_new, int32_t* new_cells, int32_t* map, int64_t cap) {
  if (n_cells <= 0 || !cells || !desired || !levels || !n_new) return fail(nullptr, PERK_E_INVALID_ARG, "bad arguments");
  Conn conn;
  const std::string e = build_connectivity3(n_cells, cells, conn);
  if (!e.empty()) return fail(nullptr, PERK_E_INVALID_ARG, "%s", e.c_str());
  std::vector<int32_t> d(n_cells);
  for (int64_t q = 0; q < n_cells; ++q) {
    const int l = cells[4 * q];
    if (desired[q] < l - 1 || desired[q] > l + 1 || desired[q] < 0 || desired[q] > MAX_LEVEL3)
      return fail(nullptr, PERK_E_INVALID_ARG, "desired level of cell %lld must differ by at most one", (long long)q);
    d[q] = desired[q];
  }
  std::vector<std::pair<int32_t, int32_t>> pairs;
  pairs.reserve(conn.ifs.size() + 4 * conn.morts.size());
  for (const int4& f : conn.ifs) pairs.emplace_back(f.x, f.y);
  for (const int4& m : conn.morts) {
    const int4 sm = conn.msmall[m.z];
    for (int32_t q : {sm.x, sm.y, sm.z, sm.w}) pairs.emplace_back(m.x, q);
  }
  bool identity = false;
  std::vector<int32_t> nc, mp;
  if (!plan_cells3(n_cells, cells, pairs, d, &identity, nc, mp))
    return fail(nullptr, PERK_E_INVALID_ARG, "internal: missing child in AMR plan");
  std::copy(d.begin(), d.end(), levels);
  const int64_t m = (int64_t)nc.size() / 4;
  *n_new = m;
  if (cap >= m) {
    if (new_cells) std::copy(nc.begin(), nc.end(), new_cells);
    if (map) std::copy(mp.begin(), mp.end(), map);
  }
  return PERK_OK;
}

perk_status perk3d_get_cells(const perk3d_ctx* ctx, int32_t* cells, int64_t cap) {
  if (!ctx || !cells) return PERK_E_INVALID_ARG;
  if (cap < ctx->n_elem) return PERK_E_INVALID_ARG;
  std::copy(ctx->h_cells.begin(), ctx->h_cells.end(), cells);
  return PERK_OK;
}

}  // extern "C"
