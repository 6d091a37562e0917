// BR1 viscous terms of the compressible Navier-Stokes equations (Bassi-Rebay 1,
// strong form; the paper's viscous cases, Sec. 7.1), added to the Euler
// right-hand side of the same stage:
//
//   k_grad_faces   central face values w* = (w_L + w_R)/2 of w = (v1, v2, T = p/rho)
//                  at every face node (mortars: small side averages with the
//                  interpolated large trace; large side takes the L2 projection)
//   k_grad         q = (2/h) [D w + lifting of (w* - w)] at every node of every
//                  element (inactive elements included: active neighbours need
//                  their traces; this covers the one-ring halo), and from it and the
//                  stage state the viscous fluxes f_v along x and y, stored per node
//   k_visc_faces   central viscous face flux f* = (f_v,L + f_v,R)/2 (normal component),
//                  from the stored fluxes
//   k_visc_volume  K += (2/h) [D f_v + lifting of (f* - f_v)] on the active elements,
//                  from the stored fluxes; on the last stage also the admissibility
//                  check of the step
//
// Stage states are formed on the fly exactly as in the inviscid kernels.

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "perk.h"
#include "perk_internal.h"
#include "perk_devmath.cuh"

namespace perk {
namespace br1 {

constexpr int FSTRIDE = 128;  // doubles of viscous fluxes per element: [direction][variable][node]
constexpr int WSTRIDE = 64;   // doubles of face data per element: [face][variable][node]
// one-warp blocks: 8 interfaces (4 threads each) or 4 mortars (8 threads each) per face block,
// 2 elements (16 threads each) per element block, so that the few thousand elements of a stage
// spread over all SMs
constexpr int BR1_THREADS = 32, BR1_IF = BR1_THREADS / 4, BR1_MORT = BR1_THREADS / 8, BR1_ELEMS = BR1_THREADS / 16;

__device__ __forceinline__ int face_node(int face, int k) {
  return face == 0 ? 4 * k : face == 1 ? 4 * k + 3 : face == 2 ? k : 12 + k;
}

template <int YS>
__device__ __forceinline__ void state(const StageArgs& sa, int64_t e, int m, int node, double y[4]) {
  const int64_t base = e * ELEM + node;
  if (YS == Y_GIVEN) {
    for (int v = 0; v < 4; ++v) y[v] = __ldg(sa.Y + base + v * NODES);
  } else {
    const StageCoef c = sa.coef[m];
    const double dt = sa.dt[sa.member ? sa.member[e] : 0];
    for (int v = 0; v < 4; ++v) y[v] = __ldg(sa.U + base + v * NODES);
    if (__double_as_longlong(c.alpha) != 0)
      for (int v = 0; v < 4; ++v) y[v] = fma(dt * c.alpha, __ldg(sa.K1 + base + v * NODES), y[v]);
    if (__double_as_longlong(c.beta) != 0) {
      const double* Kp = coupled_stage(sa, c);
      for (int v = 0; v < 4; ++v) y[v] = fma(dt * c.beta, __ldg(Kp + base + v * NODES), y[v]);
    }
  }
}

// the gradient variables (v1, v2, T = p/rho) of a state (1/rho by the Newton-refined reciprocal)
__device__ __forceinline__ void grad_vars(const double u[4], double gm1, double w[3]) {
  const double ir = rcp_nr(u[0]);
  w[0] = u[1] * ir;
  w[1] = u[2] * ir;
  const double p = gm1 * (u[3] - 0.5 * (u[1] * w[0] + u[2] * w[1]));
  w[2] = p * ir;
}

// normal viscous flux (direction dir) from the velocities (v1, v2) and the gradients
// (dvars/dx, dvars/dy)
__device__ __forceinline__ void visc_flux(double v1, double v2, const double qx[3], const double qy[3], int dir,
                                          double mu, double kappa, double f[4]) {
  const double div = qx[0] + qy[1];
  if (dir == 0) {
    const double txx = mu * (2.0 * qx[0] - (2.0 / 3.0) * div);
    const double txy = mu * (qy[0] + qx[1]);
    f[0] = 0.0;
    f[1] = txx;
    f[2] = txy;
    f[3] = v1 * txx + v2 * txy + kappa * qx[2];
  } else {
    const double tyy = mu * (2.0 * qy[1] - (2.0 / 3.0) * div);
    const double txy = mu * (qy[0] + qx[1]);
    f[0] = 0.0;
    f[1] = txy;
    f[2] = tyy;
    f[3] = v1 * txy + v2 * tyy + kappa * qy[2];
  }
}


// ---------------------------------------------------------------------------
template <int YS, int PHASE>
__global__ void __launch_bounds__(BR1_THREADS) k_faces(Ops ops, int64_t n_if, const int4* __restrict__ ifs, int64_t n_mort,
                                                const int4* __restrict__ morts, int64_t if_blocks,
                                                const int32_t* __restrict__ method, StageArgs sa,
                                                const double* __restrict__ q, double mu, double kappa,
                                                double* __restrict__ out) {
  // PHASE 0: central w* (3 variables); PHASE 1: central viscous flux (4 variables)
  constexpr int NVAR = PHASE == 0 ? 3 : 4;
  __shared__ double s_half[BR1_MORT][2][4][NN];
  auto value = [&](int64_t e, int m, int node, int dir, double r[4]) {
    if (PHASE == 0) {
      double u[4];
      state<YS>(sa, e, m, node, u);
      grad_vars(u, ops.gm1, r);
    } else {
      // the flux along the face's direction, stored by k_grad
      for (int v = 0; v < 4; ++v) r[v] = __ldg(q + e * FSTRIDE + dir * 64 + v * NODES + node);
    }
  };
  if (blockIdx.x < if_blocks) {
    const int64_t idx = (int64_t)blockIdx.x * BR1_IF + (threadIdx.x >> 2);
    const int k = threadIdx.x & 3;
    if (idx >= n_if) return;
    const int4 r = ifs[idx];
    const int dir = r.z;
    double a[4], b[4];
    value(r.x, r.w, face_node(2 * dir + 1, k), dir, a);
    value(r.y, r.w, face_node(2 * dir, k), dir, b);
    for (int v = 0; v < NVAR; ++v) {
      const double avg = 0.5 * (a[v] + b[v]);
      out[(int64_t)r.x * WSTRIDE + (2 * dir + 1) * 16 + 4 * v + k] = avg;
      out[(int64_t)r.y * WSTRIDE + (2 * dir) * 16 + 4 * v + k] = avg;
    }
    return;
  }
  const int lm = threadIdx.x >> 3;
  const int64_t idx = (int64_t)(blockIdx.x - if_blocks) * BR1_MORT + lm;
  const int half = (threadIdx.x >> 2) & 1, k = threadIdx.x & 3;
  const bool valid = idx < n_mort;
  int4 r = valid ? morts[idx] : make_int4(0, 0, 0, 0);
  const int dir = r.w & 1, large_side = (r.w >> 1) & 1, m_fine = r.w >> 2;
  const int large_face = large_side == 0 ? 2 * dir + 1 : 2 * dir;
  const int small_face = large_side == 0 ? 2 * dir : 2 * dir + 1;
  const int small = half ? r.z : r.y;
  if (valid) {
    const int m_large = method[r.x];
    double li[4] = {0.0, 0.0, 0.0, 0.0};
    for (int l = 0; l < NN; ++l) {
      double a[4];
      value(r.x, m_large, face_node(large_face, l), dir, a);
      const double w = half ? ops.p_hi[k][l] : ops.p_lo[k][l];
      for (int v = 0; v < NVAR; ++v) li[v] = fma(w, a[v], li[v]);
    }
    double b[4];
    value(small, m_fine, face_node(small_face, k), dir, b);
    for (int v = 0; v < NVAR; ++v) {
      const double avg = 0.5 * (b[v] + li[v]);
      out[(int64_t)small * WSTRIDE + small_face * 16 + 4 * v + k] = avg;
      s_half[lm][half][v][k] = avg;
    }
  }
  __syncwarp();
  if (valid) {
    for (int vv = 0; vv < 2; ++vv) {
      const int v = 2 * half + vv;
      if (v >= NVAR) continue;
      double acc = 0.0;
      for (int l = 0; l < NN; ++l) {
        acc = fma(ops.r_lo[k][l], s_half[lm][0][v][l], acc);
        acc = fma(ops.r_hi[k][l], s_half[lm][1][v][l], acc);
      }
      out[(int64_t)r.x * WSTRIDE + large_face * 16 + 4 * v + k] = acc;
    }
  }
}

// q = (2/h) [D w + (1/w_N)(w* - w)|_N - (1/w_0)(w* - w)|_0] along x and y, then the viscous
// fluxes f_v,x and f_v,y at the node, stored in fv[e][direction][variable][node]
template <int YS>
__global__ void __launch_bounds__(BR1_THREADS) k_grad(Ops ops, int64_t n, const int32_t* __restrict__ elems,
                                               const int32_t* __restrict__ level, const int32_t* __restrict__ method,
                                               double two_over_len, StageArgs sa, const double* __restrict__ wsurf,
                                               double mu, double kappa, double* __restrict__ fv) {
  __shared__ double s_w[BR1_ELEMS][3][NODES];
  const int le = threadIdx.x >> 4, t = threadIdx.x & 15, i = t & 3, j = t >> 2;
  const int64_t slot = (int64_t)blockIdx.x * BR1_ELEMS + le;
  const bool valid = slot < n;
  const int64_t e = valid ? elems[slot] : 0;
  double u[4] = {1.0, 0.0, 0.0, 2.5}, w[3];
  if (valid) state<YS>(sa, e, method[e], t, u);
  grad_vars(u, ops.gm1, w);
  for (int v = 0; v < 3; ++v) s_w[le][v][t] = w[v];
  __syncwarp();
  if (!valid) return;
  const double s = ldexp(two_over_len, level[e]);
  const double iw = ops.inv_w0;
  const double* ws = wsurf + e * WSTRIDE;
  double qx[3], qy[3];
  for (int v = 0; v < 3; ++v) {
    double gx = 0.0, gy = 0.0;
    for (int m = 0; m < NN; ++m) {
      gx = fma(ops.dmat[i][m], s_w[le][v][j * 4 + m], gx);
      gy = fma(ops.dmat[j][m], s_w[le][v][m * 4 + i], gy);
    }
    const double wv = s_w[le][v][t];
    if (i == 0) gx = fma(-iw, ws[0 * 16 + 4 * v + j] - wv, gx);
    if (i == 3) gx = fma(iw, ws[1 * 16 + 4 * v + j] - wv, gx);
    if (j == 0) gy = fma(-iw, ws[2 * 16 + 4 * v + i] - wv, gy);
    if (j == 3) gy = fma(iw, ws[3 * 16 + 4 * v + i] - wv, gy);
    qx[v] = s * gx;
    qy[v] = s * gy;
  }
  double fx[4], fy[4];
  visc_flux(w[0], w[1], qx, qy, 0, mu, kappa, fx);
  visc_flux(w[0], w[1], qx, qy, 1, mu, kappa, fy);
  for (int v = 0; v < 4; ++v) {
    fv[e * FSTRIDE + v * NODES + t] = fx[v];
    fv[e * FSTRIDE + 64 + v * NODES + t] = fy[v];
  }
}

// K += (2/h) [D f_v,x + D f_v,y + lifting of (f* - f_v)] on the active elements
template <int YS, bool CHECK>
__global__ void __launch_bounds__(BR1_THREADS) k_visc_volume(Ops ops, int64_t n, const int32_t* __restrict__ elems,
                                                      const int32_t* __restrict__ level,
                                                      const int32_t* __restrict__ method, double two_over_len,
                                                      StageArgs sa, const double* __restrict__ fv,
                                                      const double* __restrict__ vsurf, double* __restrict__ K,
                                                      UpdateArgs ua) {
  __shared__ double s_f[BR1_ELEMS][2][4][NODES];
  const int le = threadIdx.x >> 4, t = threadIdx.x & 15, i = t & 3, j = t >> 2;
  const int64_t slot = (int64_t)blockIdx.x * BR1_ELEMS + le;
  const bool valid = slot < n;
  const int64_t e = valid ? elems[slot] : 0;
  double fx[4] = {0.0, 0.0, 0.0, 0.0}, fy[4] = {0.0, 0.0, 0.0, 0.0};
  if (valid) {
    for (int v = 0; v < 4; ++v) {
      fx[v] = __ldg(fv + e * FSTRIDE + v * NODES + t);
      fy[v] = __ldg(fv + e * FSTRIDE + 64 + v * NODES + t);
    }
  }
  for (int v = 0; v < 4; ++v) {
    s_f[le][0][v][t] = fx[v];
    s_f[le][1][v][t] = fy[v];
  }
  __syncwarp();
  if (!valid) return;
  const double s = ldexp(two_over_len, level[e]);
  const double iw = ops.inv_w0;
  const double* vs = vsurf + e * WSTRIDE;
  double kv[4];
  for (int v = 0; v < 4; ++v) {
    double acc = 0.0;
    for (int m = 0; m < NN; ++m) {
      acc = fma(ops.dmat[i][m], s_f[le][0][v][j * 4 + m], acc);
      acc = fma(ops.dmat[j][m], s_f[le][1][v][m * 4 + i], acc);
    }
    if (i == 0) acc = fma(-iw, vs[0 * 16 + 4 * v + j] - fx[v], acc);
    if (i == 3) acc = fma(iw, vs[1 * 16 + 4 * v + j] - fx[v], acc);
    if (j == 0) acc = fma(-iw, vs[2 * 16 + 4 * v + i] - fy[v], acc);
    if (j == 3) acc = fma(iw, vs[3 * 16 + 4 * v + i] - fy[v], acc);
    const int64_t at = e * ELEM + v * NODES + t;
    kv[v] = K[at] + s * acc;
    K[at] = kv[v];
  }
  if (CHECK) {
    const double dt = sa.dt[sa.member ? sa.member[e] : 0];
    const int64_t base = e * ELEM + t;
    double un[4];
    for (int v = 0; v < 4; ++v) {
      double inc = ua.bs * kv[v];
      if (ua.b1 != 0.0) inc = fma(ua.b1, ua.K1[base + v * NODES], inc);
      if (ua.bp != 0.0) inc = fma(ua.bp, ua.Kp[base + v * NODES], inc);
      un[v] = fma(dt, inc, ua.U[base + v * NODES]);
    }
    const double p = ops.gm1 * (un[3] - 0.5 * (un[1] * un[1] + un[2] * un[2]) / un[0]);
    const bool ok = isfinite(un[0]) && isfinite(un[1]) && isfinite(un[2]) && isfinite(un[3]) && un[0] > 0.0 &&
                    p > 0.0 && isfinite(p);
    if (!ok) *ua.flag = 1;
  }
}

}  // namespace br1

cudaError_t launch_br1(cudaStream_t st, YSource ysrc, const Ops& ops, double mu, double kappa, int64_t n_if_all,
                       int64_t n_mort_all, int64_t n_if_act, int64_t n_mort_act, const int4* ifs, const int4* morts,
                       int64_t n_all, int64_t n_act, const int32_t* elems, const int32_t* level, const int32_t* method,
                       double two_over_len, const StageArgs& sa, double* wsurf, double* q, double* vsurf, double* K,
                       const UpdateArgs* check) {
  const int64_t bi = (n_if_all + br1::BR1_IF - 1) / br1::BR1_IF, bm = (n_mort_all + br1::BR1_MORT - 1) / br1::BR1_MORT;
  const int64_t bia = (n_if_act + br1::BR1_IF - 1) / br1::BR1_IF, bma = (n_mort_act + br1::BR1_MORT - 1) / br1::BR1_MORT;
  UpdateArgs ua{};
  if (check) ua = *check;
  if (ysrc == Y_GIVEN) {
    if (bi + bm) br1::k_faces<Y_GIVEN, 0><<<(unsigned)(bi + bm), br1::BR1_THREADS, 0, st>>>(ops, n_if_all, ifs, n_mort_all, morts,
                                                                               bi, method, sa, q, mu, kappa, wsurf);
    if (n_all) br1::k_grad<Y_GIVEN><<<(unsigned)((n_all + br1::BR1_ELEMS - 1) / br1::BR1_ELEMS), br1::BR1_THREADS, 0, st>>>(ops, n_all, elems, level, method,
                                                                                 two_over_len, sa, wsurf, mu, kappa, q);
    if (bia + bma) br1::k_faces<Y_GIVEN, 1><<<(unsigned)(bia + bma), br1::BR1_THREADS, 0, st>>>(
        ops, n_if_act, ifs, n_mort_act, morts, bia, method, sa, q, mu, kappa, vsurf);
    if (n_act) br1::k_visc_volume<Y_GIVEN, false><<<(unsigned)((n_act + br1::BR1_ELEMS - 1) / br1::BR1_ELEMS), br1::BR1_THREADS, 0, st>>>(
        ops, n_act, elems, level, method, two_over_len, sa, q, vsurf, K, ua);
  } else {
    if (bi + bm) br1::k_faces<Y_COMBINE, 0><<<(unsigned)(bi + bm), br1::BR1_THREADS, 0, st>>>(
        ops, n_if_all, ifs, n_mort_all, morts, bi, method, sa, q, mu, kappa, wsurf);
    if (n_all) br1::k_grad<Y_COMBINE><<<(unsigned)((n_all + br1::BR1_ELEMS - 1) / br1::BR1_ELEMS), br1::BR1_THREADS, 0, st>>>(ops, n_all, elems, level, method,
                                                                                   two_over_len, sa, wsurf, mu, kappa, q);
    if (bia + bma) br1::k_faces<Y_COMBINE, 1><<<(unsigned)(bia + bma), br1::BR1_THREADS, 0, st>>>(
        ops, n_if_act, ifs, n_mort_act, morts, bia, method, sa, q, mu, kappa, vsurf);
    if (n_act) {
      if (check)
        br1::k_visc_volume<Y_COMBINE, true><<<(unsigned)((n_act + br1::BR1_ELEMS - 1) / br1::BR1_ELEMS), br1::BR1_THREADS, 0, st>>>(
            ops, n_act, elems, level, method, two_over_len, sa, q, vsurf, K, ua);
      else
        br1::k_visc_volume<Y_COMBINE, false><<<(unsigned)((n_act + br1::BR1_ELEMS - 1) / br1::BR1_ELEMS), br1::BR1_THREADS, 0, st>>>(
            ops, n_act, elems, level, method, two_over_len, sa, q, vsurf, K, ua);
    }
  }
  return cudaGetLastError();
}

}  // namespace perk
