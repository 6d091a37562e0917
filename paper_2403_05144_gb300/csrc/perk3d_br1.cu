// BR1 viscous terms of the 3D compressible Navier-Stokes equations (Bassi-Rebay 1, strong form;
// the viscous Taylor-Green run of Sec. 7.1.3), added to the Euler right-hand side of the same
// stage.  Four launches per stage, after the inviscid volume kernel (whose face-flux buffer they
// reuse):
//
//   k3b_faces<0>    central face values w* = (w_L + w_R)/2 of w = (v1, v2, v3, T = p/rho) on the
//                   one-level halo of the active members (mortars: the small side averages with
//                   the interpolated large trace, the large side takes the four-quadrant L2
//                   projection)
//   k3b_grad        q_d = (2/h) [D_d w + lifting of (w* - w)] at every node of the halo elements,
//                   and from it and the stage state the viscous fluxes f_v,d along the three axes,
//                   stored per node (the state and the gradients are not needed again)
//   k3b_faces<1>    central viscous face flux f* = (f_v,L + f_v,R)/2 (normal component) on the
//                   active faces, from the stored fluxes
//   k3b_visc_volume K += (2/h) sum_d [D_d f_v,d + lifting of (f* - f_v,d)] on the active
//                   elements, from the stored fluxes; on the last stage also the admissibility
//                   check of the step
//
// Face neighbours differ by at most one level, hence by at most one member, so the halo of
// the active members is a prefix of the level-sorted lists (the partition's halo counts).

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "perk3d_device.cuh"
#include "perk3d_internal.h"
#include "perk_devmath.cuh"

namespace perk3 {
namespace br1 {

using perk::Y_COMBINE;
using perk::Y_GIVEN;

__device__ __forceinline__ void grad_vars3(const double u[5], double gm1, double w[5]) {
  const double ir = perk::rcp_nr(u[0]);
  w[0] = u[1] * ir;
  w[1] = u[2] * ir;
  w[2] = u[3] * ir;
  const double p = gm1 * (u[4] - 0.5 * (u[1] * w[0] + u[2] * w[1] + u[3] * w[2]));
  w[3] = p * ir;
  w[4] = 0.0;
}

// viscous flux along axis d from the velocity v and q[a][var] = d w_var / d x_a
__device__ __forceinline__ void visc_flux3(const double v[3], const double q[3][4], int d, double mu, double kappa,
                                           double f[5]) {
  const double div = q[0][0] + q[1][1] + q[2][2];
  double tau[3];   // tau_{a d} = mu (dv_a/dx_d + dv_d/dx_a) - (2/3) mu div delta_ad
#pragma unroll
  for (int a = 0; a < 3; ++a) tau[a] = mu * (q[d][a] + q[a][d] - (a == d ? (2.0 / 3.0) * div : 0.0));
  f[0] = 0.0;
  f[1] = tau[0];
  f[2] = tau[1];
  f[3] = tau[2];
  f[4] = fma(v[0], tau[0], fma(v[1], tau[1], fma(v[2], tau[2], kappa * q[d][3])));
}


constexpr int THREADS = 128;

// PHASE 0: central w* (4 variables); PHASE 1: central viscous flux (5 variables); face data in
// surf[e][face][variable][face node] (the inviscid kernels' layout)
template <int NN, int YS, int PHASE>
__global__ void __launch_bounds__(THREADS) k3b_faces(Ops3 ops, int64_t n_if, const int4* __restrict__ ifs,
                                                      int64_t n_mort, const int4* __restrict__ morts,
                                                      const int4* __restrict__ msmall, int64_t if_blocks,
                                                      const int32_t* __restrict__ method, StageArgs sa,
                                                      const double* __restrict__ q, double mu, double kappa,
                                                      double* __restrict__ surf) {
  constexpr int FN = G<NN>::FN, SURF = G<NN>::SURF;
  constexpr int IFB = THREADS / FN, MB = THREADS / (4 * FN);
  constexpr int NVAR = PHASE == 0 ? 4 : 5;
  __shared__ double s_l[MB][5][FN];
  __shared__ double s_a[MB][4][5][FN];
  auto value = [&](int64_t e, int m, int node, int d, double r[5]) {
    if (PHASE == 0) {
      double u[5];
      stage_state3<NN, YS>(sa, e, m, node, u);
      grad_vars3(u, ops.gm1, r);
    } else {
      // the flux along the face's axis, stored by k3b_grad
#pragma unroll
      for (int v = 0; v < 5; ++v) r[v] = __ldg(q + e * G<NN>::F + (d * 5 + v) * G<NN>::NODES + node);
    }
  };
  if (blockIdx.x < if_blocks) {
    const int li = threadIdx.x / FN, k = threadIdx.x - li * FN;
    const int64_t idx = (int64_t)blockIdx.x * IFB + li;
    if (li >= IFB || idx >= n_if) return;
    const int4 r = ifs[idx];
    const int d = r.z;
    double a[5], b[5];
    value(r.x, r.w, face_node3<NN>(2 * d + 1, k), d, a);
    value(r.y, r.w, face_node3<NN>(2 * d, k), d, b);
#pragma unroll
    for (int v = 0; v < NVAR; ++v) {
      const double avg = 0.5 * (a[v] + b[v]);
      surf[(int64_t)r.x * SURF + (2 * d + 1) * 5 * FN + v * FN + k] = avg;
      surf[(int64_t)r.y * SURF + (2 * d) * 5 * FN + v * FN + k] = avg;
    }
    return;
  }
  const int lm = threadIdx.x / (4 * FN);
  const int rem = threadIdx.x - lm * 4 * FN;
  const int quad = rem / FN, k = rem - quad * FN;
  const int64_t idx = (int64_t)(blockIdx.x - if_blocks) * MB + lm;
  const bool valid = lm < MB && idx < n_mort;
  int4 r = make_int4(0, 0, 0, 0);
  if (valid) r = morts[idx];
  const int d = r.w & 3, large_side = (r.w >> 2) & 1, m_fine = r.w >> MORT_FLAG_BITS;
  const int large_face = large_side == 0 ? 2 * d + 1 : 2 * d;
  const int small_face = large_side == 0 ? 2 * d : 2 * d + 1;
  const int t1 = k % NN, t2 = k / NN, q1 = quad & 1, q2 = quad >> 1;
  if (valid && quad == 0) {
    double a[5];
    value(r.x, method[r.x], face_node3<NN>(large_face, k), d, a);
#pragma unroll
    for (int v = 0; v < NVAR; ++v) s_l[lm][v][k] = a[v];
  }
  __syncthreads();
  if (valid) {
    double w1[NN];
#pragma unroll
    for (int l1 = 0; l1 < NN; ++l1) w1[l1] = q1 ? ops.p_hi[t1][l1] : ops.p_lo[t1][l1];
    double li[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int l2 = 0; l2 < NN; ++l2) {
      const double w2 = q2 ? ops.p_hi[t2][l2] : ops.p_lo[t2][l2];
#pragma unroll
      for (int v = 0; v < NVAR; ++v) {
        double row = 0.0;
#pragma unroll
        for (int l1 = 0; l1 < NN; ++l1) row = fma(w1[l1], s_l[lm][v][l2 * NN + l1], row);
        li[v] = fma(w2, row, li[v]);
      }
    }
    const int4 sm = msmall[r.z];
    const int small = quad == 0 ? sm.x : quad == 1 ? sm.y : quad == 2 ? sm.z : sm.w;
    double b[5];
    value(small, m_fine, face_node3<NN>(small_face, k), d, b);
#pragma unroll
    for (int v = 0; v < NVAR; ++v) {
      const double avg = 0.5 * (b[v] + li[v]);
      surf[(int64_t)small * SURF + small_face * 5 * FN + v * FN + k] = avg;
      s_a[lm][quad][v][k] = avg;
    }
  }
  __syncthreads();
  if (valid) {
    for (int vv = 0; vv < 2; ++vv) {
      const int v = vv ? 4 : quad;
      if (v >= NVAR || (vv && quad != 0)) continue;
      double acc = 0.0;
#pragma unroll
      for (int qq = 0; qq < 4; ++qq)
#pragma unroll
        for (int l2 = 0; l2 < NN; ++l2) {
          double row = 0.0;
#pragma unroll
          for (int l1 = 0; l1 < NN; ++l1)
            row = fma((qq & 1) ? ops.r_hi[t1][l1] : ops.r_lo[t1][l1], s_a[lm][qq][v][l2 * NN + l1], row);
          acc = fma((qq >> 1) ? ops.r_hi[t2][l2] : ops.r_lo[t2][l2], row, acc);
        }
      surf[(int64_t)r.x * SURF + large_face * 5 * FN + v * FN + k] = acc;
    }
  }
}

template <int NN>
struct Cfg {
  static constexpr int VE = THREADS / G<NN>::NODES;   // 4 (N = 2) or 2 (N = 3)
};

// q_d = (2/h) [D_d w + (1/w_N)(w* - w)|_N - (1/w_0)(w* - w)|_0] along the three axes, then the
// viscous fluxes f_v,d(u, q) at the node, stored in fv[e][d][variable][node]
template <int NN, int YS>
__global__ void __launch_bounds__(THREADS) k3b_grad(Ops3 ops, int64_t n, const int32_t* __restrict__ elems,
                                                     const int32_t* __restrict__ level,
                                                     const int32_t* __restrict__ method, double two_over_len,
                                                     StageArgs sa, const double* __restrict__ surf, double mu,
                                                     double kappa, double* __restrict__ fv) {
  constexpr int FN = G<NN>::FN, NODES = G<NN>::NODES, SURF = G<NN>::SURF, VE = Cfg<NN>::VE;
  __shared__ double s_w[VE][4][NODES];
  const int t = threadIdx.x, le = t / NODES, node = t - le * NODES;
  const int64_t slot = (int64_t)blockIdx.x * VE + le;
  const bool valid = le < VE && slot < n;
  const int64_t e = valid ? elems[slot] : 0;
  const int i = node % NN, j = (node / NN) % NN, k = node / FN;
  double w[5];
  if (valid) {
    double u[5];
    stage_state3<NN, YS>(sa, e, method[e], node, u);
    grad_vars3(u, ops.gm1, w);
#pragma unroll
    for (int v = 0; v < 4; ++v) s_w[le][v][node] = w[v];
  }
  __syncthreads();
  if (!valid) return;
  const double s = ldexp(two_over_len, level[e]);
  const double iw = ops.inv_w0;
  const double* ws = surf + e * SURF;
  double qq[3][4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    double gx = 0.0, gy = 0.0, gz = 0.0;
#pragma unroll
    for (int m = 0; m < NN; ++m) {
      gx = fma(ops.dmat[i][m], s_w[le][v][(k * NN + j) * NN + m], gx);
      gy = fma(ops.dmat[j][m], s_w[le][v][(k * NN + m) * NN + i], gy);
      gz = fma(ops.dmat[k][m], s_w[le][v][(m * NN + j) * NN + i], gz);
    }
    const double wv = s_w[le][v][node];
    if (i == 0) gx = fma(-iw, ws[0 * 5 * FN + v * FN + k * NN + j] - wv, gx);
    if (i == NN - 1) gx = fma(iw, ws[1 * 5 * FN + v * FN + k * NN + j] - wv, gx);
    if (j == 0) gy = fma(-iw, ws[2 * 5 * FN + v * FN + k * NN + i] - wv, gy);
    if (j == NN - 1) gy = fma(iw, ws[3 * 5 * FN + v * FN + k * NN + i] - wv, gy);
    if (k == 0) gz = fma(-iw, ws[4 * 5 * FN + v * FN + j * NN + i] - wv, gz);
    if (k == NN - 1) gz = fma(iw, ws[5 * 5 * FN + v * FN + j * NN + i] - wv, gz);
    qq[0][v] = s * gx;
    qq[1][v] = s * gy;
    qq[2][v] = s * gz;
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double f[5];
    visc_flux3(w, qq, d, mu, kappa, f);   // w[0..2] is the velocity
#pragma unroll
    for (int v = 0; v < 5; ++v) fv[e * G<NN>::F + (d * 5 + v) * NODES + node] = f[v];
  }
}

// K += (2/h) sum_d [D_d f_v,d + lifting of (f* - f_v,d)] on the active elements
template <int NN, int YS, bool CHECK>
__global__ void __launch_bounds__(THREADS) k3b_visc_volume(Ops3 ops, int64_t n, const int32_t* __restrict__ elems,
                                                            const int32_t* __restrict__ level,
                                                            const int32_t* __restrict__ method,
                                                            double two_over_len, StageArgs sa,
                                                            const double* __restrict__ fv,
                                                            const double* __restrict__ surf,
                                                            double* __restrict__ K, UpdateArgs ua) {
  constexpr int FN = G<NN>::FN, NODES = G<NN>::NODES, ELEM = G<NN>::ELEM, SURF = G<NN>::SURF;
  constexpr int VE = Cfg<NN>::VE;
  __shared__ double s_f[VE][3][5][NODES];
  const int t = threadIdx.x, le = t / NODES, node = t - le * NODES;
  const int64_t slot = (int64_t)blockIdx.x * VE + le;
  const bool valid = le < VE && slot < n;
  const int64_t e = valid ? elems[slot] : 0;
  const int i = node % NN, j = (node / NN) % NN, k = node / FN;
  double f[3][5];
  if (valid) {
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        f[d][v] = __ldg(fv + e * G<NN>::F + (d * 5 + v) * NODES + node);
        s_f[le][d][v][node] = f[d][v];
      }
  }
  __syncthreads();
  if (!valid) return;
  const double s = ldexp(two_over_len, level[e]);
  const double iw = ops.inv_w0;
  const double* vs = surf + e * SURF;
  double kv[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < NN; ++m) {
      acc = fma(ops.dmat[i][m], s_f[le][0][v][(k * NN + j) * NN + m], acc);
      acc = fma(ops.dmat[j][m], s_f[le][1][v][(k * NN + m) * NN + i], acc);
      acc = fma(ops.dmat[k][m], s_f[le][2][v][(m * NN + j) * NN + i], acc);
    }
    if (i == 0) acc = fma(-iw, vs[0 * 5 * FN + v * FN + k * NN + j] - f[0][v], acc);
    if (i == NN - 1) acc = fma(iw, vs[1 * 5 * FN + v * FN + k * NN + j] - f[0][v], acc);
    if (j == 0) acc = fma(-iw, vs[2 * 5 * FN + v * FN + k * NN + i] - f[1][v], acc);
    if (j == NN - 1) acc = fma(iw, vs[3 * 5 * FN + v * FN + k * NN + i] - f[1][v], acc);
    if (k == 0) acc = fma(-iw, vs[4 * 5 * FN + v * FN + j * NN + i] - f[2][v], acc);
    if (k == NN - 1) acc = fma(iw, vs[5 * 5 * FN + v * FN + j * NN + i] - f[2][v], acc);
    const int64_t at = e * ELEM + v * NODES + node;
    kv[v] = fma(s, acc, K[at]);
    K[at] = kv[v];
  }
  if (CHECK) {
    const double dt = sa.dt[0];
    const int64_t base = e * ELEM + node;
    double un[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      double inc = ua.bs * kv[v];
      if (ua.b1 != 0.0) inc = fma(ua.b1, __ldg(ua.K1 + base + v * NODES), inc);
      if (ua.bp != 0.0) inc = fma(ua.bp, __ldg(ua.Kp + base + v * NODES), inc);
      un[v] = fma(dt, inc, __ldg(ua.U + base + v * NODES));
    }
    const double p = ops.gm1 * (un[4] - 0.5 * (un[1] * un[1] + un[2] * un[2] + un[3] * un[3]) / un[0]);
    bool ok = un[0] > 0.0 && p > 0.0 && isfinite(p);
#pragma unroll
    for (int v = 0; v < 5; ++v) ok = ok && isfinite(un[v]);
    if (!ok) *ua.flag = 1;
  }
}

template <int NN, int YS>
static void br1_launches(cudaStream_t st, const Ops3& ops, double mu, double kappa, int64_t n_if_h, int64_t n_mort_h,
                         int64_t n_if_a, int64_t n_mort_a, const int4* ifs, const int4* morts, const int4* msmall,
                         int64_t n_el_h, int64_t n_el_a, const int32_t* elems, const int32_t* level,
                         const int32_t* method, double two_over_len, const StageArgs& sa, double* surf, double* q,
                         double* K, const UpdateArgs* check) {
  constexpr int FN = NN * NN, IFB = THREADS / FN, MB = THREADS / (4 * FN), VE = Cfg<NN>::VE;
  const int64_t bi = (n_if_h + IFB - 1) / IFB, bm = (n_mort_h + MB - 1) / MB;
  const int64_t bia = (n_if_a + IFB - 1) / IFB, bma = (n_mort_a + MB - 1) / MB;
  const UpdateArgs ua = check ? *check : UpdateArgs{};
  if (bi + bm)
    k3b_faces<NN, YS, 0><<<(unsigned)(bi + bm), THREADS, 0, st>>>(ops, n_if_h, ifs, n_mort_h, morts, msmall, bi,
                                                                  method, sa, q, mu, kappa, surf);
  if (n_el_h)
    k3b_grad<NN, YS><<<(unsigned)((n_el_h + VE - 1) / VE), THREADS, 0, st>>>(ops, n_el_h, elems, level, method,
                                                                             two_over_len, sa, surf, mu, kappa, q);
  if (bia + bma)
    k3b_faces<NN, YS, 1><<<(unsigned)(bia + bma), THREADS, 0, st>>>(ops, n_if_a, ifs, n_mort_a, morts, msmall, bia,
                                                                    method, sa, q, mu, kappa, surf);
  if (n_el_a) {
    const unsigned g = (unsigned)((n_el_a + VE - 1) / VE);
    if (check)
      k3b_visc_volume<NN, YS, true><<<g, THREADS, 0, st>>>(ops, n_el_a, elems, level, method, two_over_len, sa, q,
                                                           surf, K, ua);
    else
      k3b_visc_volume<NN, YS, false><<<g, THREADS, 0, st>>>(ops, n_el_a, elems, level, method, two_over_len, sa, q,
                                                            surf, K, ua);
  }
}

}  // namespace br1

cudaError_t launch_br1_3d(cudaStream_t st, YSource ys, const Ops3& ops, double mu, double kappa, int64_t n_if_halo,
                          int64_t n_mort_halo, int64_t n_if_act, int64_t n_mort_act, const int4* ifs,
                          const int4* morts, const int4* msmall, int64_t n_el_halo, int64_t n_el_act,
                          const int32_t* elems, const int32_t* level, const int32_t* method, double two_over_len,
                          const StageArgs& sa, double* surf, double* q, double* K, const UpdateArgs* check) {
#define P3B_ARGS                                                                                              \
  st, ops, mu, kappa, n_if_halo, n_mort_halo, n_if_act, n_mort_act, ifs, morts, msmall, n_el_halo, n_el_act, \
      elems, level, method, two_over_len, sa, surf, q, K, check
  if (ops.nn == 3) {
    if (ys == perk::Y_GIVEN)
      br1::br1_launches<3, perk::Y_GIVEN>(P3B_ARGS);
    else
      br1::br1_launches<3, perk::Y_COMBINE>(P3B_ARGS);
  } else if (ops.nn == 4) {
    if (ys == perk::Y_GIVEN)
      br1::br1_launches<4, perk::Y_GIVEN>(P3B_ARGS);
    else
      br1::br1_launches<4, perk::Y_COMBINE>(P3B_ARGS);
  } else {
    return cudaErrorInvalidValue;
  }
#undef P3B_ARGS
  return cudaGetLastError();
}

}  // namespace perk3
