// Derivatives of the partitioned DGSEM right-hand side: Jacobian-vector
// products (JVP) and vector-Jacobian products (VJP), the building blocks of the
// discrete adjoint of the P-ERK step.
//
// Both differentiate exactly the discrete operator of perk_kernels.cu (same
// logarithm table, reciprocals and branch decisions, which are taken on the
// values).  Forward-mode dual numbers carry the derivatives:
//   * JVP: one tangent per value (Dual<1>): K and dK = J(Y) v in one pass.
//   * VJP: hand-written reverse sweeps of the two-point volume flux, the node
//     quantities and the surface fluxes, applied to the adjoint weight of every
//     pair and face-node flux, so that J(Y)^T lambda is assembled pair by pair
//     and face by face without ever forming a Jacobian.

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "perk.h"
#include "perk_internal.h"
#include "perk_devmath.cuh"

namespace perk {
namespace ad {

template <int N>
struct Dual {
  double v;
  double d[N];
};

template <int N>
__device__ __forceinline__ Dual<N> cst(double a) {
  Dual<N> r;
  r.v = a;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = 0.0;
  return r;
}

// ---- arithmetic on doubles and dual numbers (same names, overloaded) ----
__device__ __forceinline__ double val(double a) { return a; }
template <int N>
__device__ __forceinline__ double val(const Dual<N>& a) { return a.v; }

template <int N>
__device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = fma(a.v, b.d[k], a.d[k] * b.v);
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(double a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a * b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a * b.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(const Dual<N>& b, double a) {
  return a * b;
}
template <int N>
__device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, double b) {
  Dual<N> r = a;
  r.v += b;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator+(double b, const Dual<N>& a) {
  return a + b;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, double b) {
  Dual<N> r = a;
  r.v -= b;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(double b, const Dual<N>& a) {
  return -(a - b);
}
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
template <int N>
__device__ __forceinline__ Dual<N> fma_(const Dual<N>& a, const Dual<N>& b, const Dual<N>& c) {
  Dual<N> r;
  r.v = fma(a.v, b.v, c.v);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = fma(a.v, b.d[k], fma(a.d[k], b.v, c.d[k]));
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> fma_(double a, const Dual<N>& b, const Dual<N>& c) {
  Dual<N> r;
  r.v = fma(a, b.v, c.v);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = fma(a, b.d[k], c.d[k]);
  return r;
}

// 1/x by the primal's Newton-Raphson reciprocal; d(1/x) = -dx / x^2
__device__ __forceinline__ double rcp_val(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}
__device__ __forceinline__ double rcp_(double x) { return rcp_val(x); }
template <int N>
__device__ __forceinline__ Dual<N> rcp_(const Dual<N>& x) {
  const double y = rcp_val(x.v);
  const double m = -y * y;
  Dual<N> r;
  r.v = y;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = m * x.d[k];
  return r;
}

// the primal's table logarithm; d ln x = dx / x
__device__ __forceinline__ double log_val(double x, const double* inv_c, const double* ln_c) {
  const long long bits = __double_as_longlong(x);
  const int hi = (int)(bits >> 32);
  const int j = (hi >> 13) & (LOG_TABLE_SIZE - 1);
  const long long eb = (bits >> 52) & 0x7FF;
  const double m = __longlong_as_double((bits & 0x000FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
  const double kd = __longlong_as_double(0x4330000000000000LL | eb) - (4503599627370496.0 + 1023.0);
  const double r = fma(m, inv_c[j], -1.0);
  double q = -1.0 / 8.0;
  q = fma(q, r, 1.0 / 7.0);
  q = fma(q, r, -1.0 / 6.0);
  q = fma(q, r, 1.0 / 5.0);
  q = fma(q, r, -1.0 / 4.0);
  q = fma(q, r, 1.0 / 3.0);
  q = fma(q, r, -0.5);
  const double l1p = fma(r * r, q, r);
  const double v = fma(kd, 0.6931471805599453, ln_c[j] + fma(kd, 2.3190468138462996e-17, l1p));
  return x > 0.0 ? v : __longlong_as_double(0x7FF8000000000000LL);
}
__device__ __forceinline__ double log_(double x, const double* ic, const double* lc) { return log_val(x, ic, lc); }
template <int N>
__device__ __forceinline__ Dual<N> log_(const Dual<N>& x, const double* ic, const double* lc) {
  Dual<N> r;
  r.v = log_val(x.v, ic, lc);
  const double ix = rcp_val(x.v);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = x.d[k] * ix;
  return r;
}

__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
template <int N>
__device__ __forceinline__ Dual<N> sqrt_(const Dual<N>& x) {
  Dual<N> r;
  r.v = sqrt(x.v);
  const double h = 0.5 / r.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = h * x.d[k];
  return r;
}
template <class T>
__device__ __forceinline__ T min_(const T& a, const T& b) {
  return val(a) <= val(b) ? a : b;
}
template <class T>
__device__ __forceinline__ T max_(const T& a, const T& b) {
  return val(a) >= val(b) ? a : b;
}

__device__ __forceinline__ double cst_like(double, double c) { return c; }
template <int N>
__device__ __forceinline__ Dual<N> cst_like(const Dual<N>&, double c) {
  return cst<N>(c);
}

// ---- the discrete operator, generic in the scalar type ----
template <class T>
struct NodeQ {
  T rho, lnrho, beta, lnbeta, v1, v2, hv1, hv2, hp;
};

template <class T>
__device__ __forceinline__ NodeQ<T> node_q(const T u[4], double gm1, const double* ic, const double* lc) {
  NodeQ<T> q;
  const T rp = gm1 * fma_(u[0], u[3], -0.5 * fma_(u[1], u[1], u[2] * u[2]));
  const T r = rcp_(u[0] * rp);
  const T ir = rp * r;
  q.rho = u[0];
  q.v1 = u[1] * ir;
  q.v2 = u[2] * ir;
  q.hp = 0.5 * (rp * ir);
  q.beta = (u[0] * u[0]) * (u[0] * r);
  q.hv1 = 0.5 * q.v1;
  q.hv2 = 0.5 * q.v2;
  q.lnrho = log_(u[0], ic, lc);
  q.lnbeta = log_(q.beta, ic, lc);
  return q;
}

template <class T>
__device__ __forceinline__ T series_H(const T& u) {
  T r = cst_like(u, -214.0 / 14175.0);
  r = fma_(r, u, cst_like(u, -22.0 / 945.0));
  r = fma_(r, u, cst_like(u, -2.0 / 45.0));
  r = fma_(r, u, cst_like(u, -1.0 / 6.0));
  return fma_(r, u, cst_like(u, 0.5));
}
template <class T>
__device__ __forceinline__ T series_2A(const T& u) {
  T r = cst_like(u, 2.0 / 9.0);
  r = fma_(r, u, cst_like(u, 2.0 / 7.0));
  r = fma_(r, u, cst_like(u, 2.0 / 5.0));
  r = fma_(r, u, cst_like(u, 2.0 / 3.0));
  return fma_(r, u, cst_like(u, 2.0));
}

template <class T>
__device__ __forceinline__ void ec_flux(const NodeQ<T>& A, const NodeQ<T>& B, int dir, double inv_gm1, T f[4]) {
  const T dr = B.rho - A.rho, sr = A.rho + B.rho;
  const T db = B.beta - A.beta, sb = A.beta + B.beta;
  const bool ser_r = near_pair(val(A.rho), val(B.rho));
  const bool ser_b = near_pair(val(A.beta), val(B.beta));
  const T den_r = ser_r ? sr : B.lnrho - A.lnrho;
  const T den_b = ser_b ? sb : db;
  const T r = rcp_(den_r * den_b);
  const T qr = den_b * r;
  const T qb = den_r * r;
  const T fr = dr * qr;
  const T rho_ln = ser_r ? sr * series_H(fr * fr) : fr;
  T ibeta;
  if (ser_b) {
    const T fb = db * qb;
    ibeta = qb * series_2A(fb * fb);
  } else {
    ibeta = (B.lnbeta - A.lnbeta) * qb;
  }
  const T v1m = A.hv1 + B.hv1;
  const T v2m = A.hv2 + B.hv2;
  const T pm = A.hp + B.hp;
  const T vnA = dir ? A.v2 : A.v1;
  const T vnB = dir ? B.v2 : B.v1;
  const T frho = rho_ln * (dir ? v2m : v1m);
  f[0] = frho;
  f[1] = dir ? frho * v1m : fma_(frho, v1m, pm);
  f[2] = dir ? fma_(frho, v2m, pm) : frho * v2m;
  const T kin = fma_(A.hv1, B.v1, A.hv2 * B.v2);
  f[3] = fma_(frho, fma_(ibeta, cst_like(ibeta, inv_gm1), kin), fma_(A.hp, vnB, B.hp * vnA));
}

template <class T>
__device__ __forceinline__ void phys_flux(const T u[4], const T& vn, const T& p, int dir, T f[4]) {
  f[0] = u[0] * vn;
  f[1] = dir ? u[1] * vn : fma_(u[1], vn, p);
  f[2] = dir ? fma_(u[2], vn, p) : u[2] * vn;
  f[3] = (u[3] + p) * vn;
}

template <class T>
__device__ void flux_hll(const T uL[4], const T uR[4], int dir, const Ops& ops, T f[4]) {
  const T irL = rcp_(uL[0]), irR = rcp_(uR[0]);
  const T pL = ops.gm1 * (uL[3] - 0.5 * (uL[1] * uL[1] + uL[2] * uL[2]) * irL);
  const T pR = ops.gm1 * (uR[3] - 0.5 * (uR[1] * uR[1] + uR[2] * uR[2]) * irR);
  const T vL = uL[1 + dir] * irL, vR = uR[1 + dir] * irR;
  const T cL = sqrt_(ops.gamma * (pL * irL)), cR = sqrt_(ops.gamma * (pR * irR));
  const T SL = min_(vL - cL, vR - cR), SR = max_(vL + cL, vR + cR);
  T fL[4], fR[4];
  phys_flux(uL, vL, pL, dir, fL);
  phys_flux(uR, vR, pR, dir, fR);
  if (val(SL) >= 0.0) {
    for (int v = 0; v < 4; ++v) f[v] = fL[v];
  } else if (val(SR) <= 0.0) {
    for (int v = 0; v < 4; ++v) f[v] = fR[v];
  } else {
    const T inv = rcp_(SR - SL);
    const T SLSR = SL * SR;
    for (int v = 0; v < 4; ++v) f[v] = (SR * fL[v] - SL * fR[v] + SLSR * (uR[v] - uL[v])) * inv;
  }
}

template <class T>
__device__ void flux_hllc(const T uL[4], const T uR[4], int dir, const Ops& ops, T f[4]) {
  const T irL = rcp_(uL[0]), irR = rcp_(uR[0]);
  const T pL = ops.gm1 * (uL[3] - 0.5 * (uL[1] * uL[1] + uL[2] * uL[2]) * irL);
  const T pR = ops.gm1 * (uR[3] - 0.5 * (uR[1] * uR[1] + uR[2] * uR[2]) * irR);
  const T vL = uL[1 + dir] * irL, vR = uR[1 + dir] * irR;
  const T cL = sqrt_(ops.gamma * (pL * irL)), cR = sqrt_(ops.gamma * (pR * irR));
  const T SL = min_(vL - cL, vR - cR), SR = max_(vL + cL, vR + cR);
  if (val(SL) >= 0.0) {
    phys_flux(uL, vL, pL, dir, f);
    return;
  }
  if (val(SR) <= 0.0) {
    phys_flux(uR, vR, pR, dir, f);
    return;
  }
  const T mL = uL[0] * (SL - vL), mR = uR[0] * (SR - vR);
  const T Ss = (pR - pL + mL * vL - mR * vR) * rcp_(mL - mR);
  const bool left = val(Ss) >= 0.0;
  const T* u = left ? uL : uR;
  const T S = left ? SL : SR;
  const T vn = left ? vL : vR;
  const T p = left ? pL : pR;
  const T m = left ? mL : mR;
  const T ir = left ? irL : irR;
  T fk[4];
  phys_flux(u, vn, p, dir, fk);
  const T fac = m * rcp_(S - Ss);
  T us[4];
  us[0] = fac;
  us[1 + dir] = fac * Ss;
  us[2 - dir] = fac * (u[2 - dir] * ir);
  us[3] = fac * (u[3] * ir + (Ss - vn) * (Ss + p * rcp_(m)));
  for (int v = 0; v < 4; ++v) f[v] = fk[v] + S * (us[v] - u[v]);
}

template <class T>
__device__ void flux_ec_surface(const T uL[4], const T uR[4], int dir, const Ops& ops, const double* ic,
                                const double* lc, T f[4]) {
  const NodeQ<T> A = node_q(uL, ops.gm1, ic, lc), B = node_q(uR, ops.gm1, ic, lc);
  ec_flux(A, B, dir, ops.inv_gm1, f);
}

template <class T>
__device__ __forceinline__ void surface_flux(const T uL[4], const T uR[4], int dir, const Ops& ops, const double* ic,
                                             const double* lc, T f[4]) {
  if (ops.surface_flux == PERK_SURFACE_HLLC)
    flux_hllc(uL, uR, dir, ops, f);
  else if (ops.surface_flux == PERK_SURFACE_EC)
    flux_ec_surface(uL, uR, dir, ops, ic, lc, f);
  else
    flux_hll(uL, uR, dir, ops, f);
}

__device__ __forceinline__ int face_node(int face, int k) {
  return face == 0 ? 4 * k : face == 1 ? 4 * k + 3 : face == 2 ? k : 12 + k;
}

// stage state at one node: given, or U + dt (alpha K1 + beta Kp) with the element's member coefficients
template <int YS>
__device__ __forceinline__ void stage_y(const StageArgs& sa, const int32_t* method, int64_t e, int node, double y[4]) {
  const int64_t base = e * ELEM + node;
  if (YS == Y_GIVEN) {
    for (int v = 0; v < 4; ++v) y[v] = sa.Y[base + v * NODES];
  } else {
    const StageCoef c = sa.coef ? sa.coef[method[e]] : StageCoef{0.0, 0.0, 0, 0};
    const double dt = sa.dt[sa.member ? sa.member[e] : 0];
    for (int v = 0; v < 4; ++v) y[v] = sa.U[base + v * NODES];
    if (__double_as_longlong(c.alpha) != 0)
      for (int v = 0; v < 4; ++v) y[v] = fma(dt * c.alpha, sa.K1[base + v * NODES], y[v]);
    if (__double_as_longlong(c.beta) != 0) {
      const double* Kp = coupled_stage(sa, c);
      for (int v = 0; v < 4; ++v) y[v] = fma(dt * c.beta, Kp[base + v * NODES], y[v]);
    }
  }
}
__device__ __forceinline__ int pair_slot(int a, int b) { return (a * (7 - a)) / 2 + b - a - 1; }

// ===========================================================================
// JVP: surface fluxes and their tangents (value in surf, tangent in surf_d)
__global__ void __launch_bounds__(128) k_jvp_faces(Ops ops, int64_t n_if, const int4* __restrict__ ifs,
                                                    int64_t n_mort, const int4* __restrict__ morts, int64_t if_blocks,
                                                    const double* __restrict__ Y, const double* __restrict__ V,
                                                    const double* __restrict__ logt, double* __restrict__ surf,
                                                    double* __restrict__ surf_d) {
  using D1 = Dual<1>;
  __shared__ double s_half[16][2][4][2][NN];   // [mortar][half][var][value, tangent][node]
  const double* ic = logt;
  const double* lc = logt + LOG_TABLE_SIZE;
  auto load = [&](int64_t e, int node, D1 u[4]) {
    for (int v = 0; v < 4; ++v) {
      u[v].v = Y[e * ELEM + v * NODES + node];
      u[v].d[0] = V[e * ELEM + v * NODES + node];
    }
  };
  if (blockIdx.x < if_blocks) {
    const int64_t idx = (int64_t)blockIdx.x * 32 + (threadIdx.x >> 2);
    const int k = threadIdx.x & 3;
    if (idx >= n_if) return;
    const int4 r = ifs[idx];
    const int dir = r.z;
    D1 uL[4], uR[4], f[4];
    load(r.x, face_node(2 * dir + 1, k), uL);
    load(r.y, face_node(2 * dir, k), uR);
    surface_flux(uL, uR, dir, ops, ic, lc, f);
    for (int v = 0; v < 4; ++v) {
      surf[(int64_t)r.x * ELEM + (2 * dir + 1) * 16 + 4 * v + k] = f[v].v;
      surf_d[(int64_t)r.x * ELEM + (2 * dir + 1) * 16 + 4 * v + k] = f[v].d[0];
      surf[(int64_t)r.y * ELEM + (2 * dir) * 16 + 4 * v + k] = f[v].v;
      surf_d[(int64_t)r.y * ELEM + (2 * dir) * 16 + 4 * v + k] = f[v].d[0];
    }
    return;
  }
  const int lm = threadIdx.x >> 3;
  const int64_t idx = (int64_t)(blockIdx.x - if_blocks) * 16 + lm;
  const int half = (threadIdx.x >> 2) & 1, k = threadIdx.x & 3;
  const bool valid = idx < n_mort;
  int4 r = valid ? morts[idx] : make_int4(0, 0, 0, 0);
  const int dir = r.w & 1, large_side = (r.w >> 1) & 1;
  const int large_face = large_side == 0 ? 2 * dir + 1 : 2 * dir;
  const int small_face = large_side == 0 ? 2 * dir : 2 * dir + 1;
  const int small = half ? r.z : r.y;
  if (valid) {
    D1 ui[4];
    for (int v = 0; v < 4; ++v) ui[v] = cst<1>(0.0);
    for (int l = 0; l < NN; ++l) {
      D1 ul[4];
      load(r.x, face_node(large_face, l), ul);
      const double w = half ? ops.p_hi[k][l] : ops.p_lo[k][l];
      for (int v = 0; v < 4; ++v) ui[v] = fma_(w, ul[v], ui[v]);
    }
    D1 us[4], f[4];
    load(small, face_node(small_face, k), us);
    if (large_side == 0)
      surface_flux(ui, us, dir, ops, ic, lc, f);
    else
      surface_flux(us, ui, dir, ops, ic, lc, f);
    for (int v = 0; v < 4; ++v) {
      surf[(int64_t)small * ELEM + small_face * 16 + 4 * v + k] = f[v].v;
      surf_d[(int64_t)small * ELEM + small_face * 16 + 4 * v + k] = f[v].d[0];
      s_half[lm][half][v][0][k] = f[v].v;
      s_half[lm][half][v][1][k] = f[v].d[0];
    }
  }
  __syncthreads();
  if (valid) {
    for (int vv = 0; vv < 2; ++vv) {
      const int v = 2 * half + vv;
      double a0 = 0.0, a1 = 0.0;
      for (int l = 0; l < NN; ++l) {
        a0 = fma(ops.r_lo[k][l], s_half[lm][0][v][0][l], fma(ops.r_hi[k][l], s_half[lm][1][v][0][l], a0));
        a1 = fma(ops.r_lo[k][l], s_half[lm][0][v][1][l], fma(ops.r_hi[k][l], s_half[lm][1][v][1][l], a1));
      }
      surf[(int64_t)r.x * ELEM + large_face * 16 + 4 * v + k] = a0;
      surf_d[(int64_t)r.x * ELEM + large_face * 16 + 4 * v + k] = a1;
    }
  }
}

// JVP: volume integral + lifting in dual numbers; writes K (value) and dK (tangent)
__global__ void __launch_bounds__(128) k_jvp_volume(Ops ops, int64_t n, const int32_t* __restrict__ elems,
                                                     const int32_t* __restrict__ level, double two_over_len,
                                                     const double* __restrict__ Y, const double* __restrict__ V,
                                                     const double* __restrict__ surf,
                                                     const double* __restrict__ surf_d,
                                                     const double* __restrict__ logt, double* __restrict__ K,
                                                     double* __restrict__ Kd) {
  using D1 = Dual<1>;
  __shared__ NodeQ<D1> s_q[8][NODES];
  __shared__ double s_f[8][4][2][48];
  __shared__ double s_log[2 * LOG_TABLE_SIZE];
  for (int q = threadIdx.x; q < 2 * LOG_TABLE_SIZE; q += 128) s_log[q] = logt[q];
  __syncthreads();
  const int le = threadIdx.x >> 4, t = threadIdx.x & 15, i = t & 3, j = t >> 2;
  const int64_t slot = (int64_t)blockIdx.x * 8 + le;
  const bool valid = slot < n;
  const int64_t e = valid ? elems[slot] : 0;
  D1 y[4];
  for (int v = 0; v < 4; ++v) {
    y[v].v = valid ? Y[e * ELEM + v * NODES + t] : (v == 0 ? 1.0 : v == 3 ? 2.5 : 0.0);
    y[v].d[0] = valid ? V[e * ELEM + v * NODES + t] : 0.0;
  }
  s_q[le][t] = node_q(y, ops.gm1, s_log, s_log + LOG_TABLE_SIZE);
  __syncwarp();
  for (int kk = 0; kk < 3; ++kk) {
    const int p = t + 16 * kk;
    const int dir = p >= 24;
    const int q = dir ? p - 24 : p;
    const int line = q / 6, qq = q - 6 * line;
    const int a = (qq >= 3) + (qq >= 5);
    const int b = qq + 1 - (a * (5 - a)) / 2;
    const int na = dir ? a * 4 + line : line * 4 + a;
    const int nb = dir ? b * 4 + line : line * 4 + b;
    D1 f[4];
    ec_flux(s_q[le][na], s_q[le][nb], dir, ops.inv_gm1, f);
    for (int v = 0; v < 4; ++v) {
      s_f[le][v][0][p] = f[v].v;
      s_f[le][v][1][p] = f[v].d[0];
    }
  }
  __syncwarp();
  double acc[4][2] = {};
  for (int mm = 0; mm < 4; ++mm) {
    if (mm != i) {
      const int p = j * 6 + pair_slot(min(i, mm), max(i, mm));
      for (int v = 0; v < 4; ++v)
        for (int c = 0; c < 2; ++c) acc[v][c] = fma(ops.dsplit[i][mm], s_f[le][v][c][p], acc[v][c]);
    }
    if (mm != j) {
      const int p = 24 + i * 6 + pair_slot(min(j, mm), max(j, mm));
      for (int v = 0; v < 4; ++v)
        for (int c = 0; c < 2; ++c) acc[v][c] = fma(ops.dsplit[j][mm], s_f[le][v][c][p], acc[v][c]);
    }
  }
  if (!valid) return;
  const double iw = ops.inv_w0;
  for (int c = 0; c < 2; ++c) {
    const double* sf = (c ? surf_d : surf) + e * ELEM;
    for (int v = 0; v < 4; ++v) {
      if (i == 0) acc[v][c] = fma(-iw, sf[0 * 16 + 4 * v + j], acc[v][c]);
      if (i == 3) acc[v][c] = fma(iw, sf[1 * 16 + 4 * v + j], acc[v][c]);
      if (j == 0) acc[v][c] = fma(-iw, sf[2 * 16 + 4 * v + i], acc[v][c]);
      if (j == 3) acc[v][c] = fma(iw, sf[3 * 16 + 4 * v + i], acc[v][c]);
    }
  }
  const double scale = -ldexp(two_over_len, level[e]);
  for (int v = 0; v < 4; ++v) {
    if (K) K[e * ELEM + v * NODES + t] = scale * acc[v][0];
    Kd[e * ELEM + v * NODES + t] = scale * acc[v][1];
  }
}

// ===========================================================================
// VJP.  lam is the adjoint of K (zero outside the active elements); g receives
// J(Y)^T lam.  Face kernel: for every active face node, the adjoint weight of
// the numerical flux (its lifting coefficients times lam on both sides) times
// the flux Jacobian gives the adjoint of the two traces, written to
// gsurf[e][face][var][node] (each element face is owned by one face record).
__device__ __forceinline__ double lift_coef(int face, double two_over_len, int level, double iw) {
  // K += -(2/h) (+iw f* on faces 1, 3; -iw f* on faces 0, 2)
  const double s = ldexp(two_over_len, level);
  return (face & 1) ? -s * iw : s * iw;
}

// ---------------------------------------------------------------------------
// Reverse (adjoint) sweep of the volume term, written out by hand.
//
// Field order of the node quantities and of their adjoints:
//   0 rho, 1 ln rho, 2 beta = rho/p, 3 ln beta, 4 v1, 5 v2, 6 v1/2, 7 v2/2, 8 p/2
enum { Q_RHO = 0, Q_LNRHO, Q_BETA, Q_LNBETA, Q_V1, Q_V2, Q_HV1, Q_HV2, Q_HP, NQ };

// derivatives of the log-mean series in u
__device__ __forceinline__ double series_H_d(double u) {   // H'(u)
  double r = 4.0 * (-214.0 / 14175.0);
  r = fma(r, u, 3.0 * (-22.0 / 945.0));
  r = fma(r, u, 2.0 * (-2.0 / 45.0));
  return fma(r, u, -1.0 / 6.0);
}
__device__ __forceinline__ double series_2A_d(double u) {  // (2A)'(u)
  double r = 4.0 * (2.0 / 9.0);
  r = fma(r, u, 3.0 * (2.0 / 7.0));
  r = fma(r, u, 2.0 * (2.0 / 5.0));
  return fma(r, u, 2.0 / 3.0);
}

// Given the adjoint g of the flux f#(A, B) in direction dir, accumulate the
// adjoints of A's and B's node quantities into gA, gB (the forward
// intermediates are recomputed; branch decisions as in the forward flux).
__device__ __forceinline__ void ec_flux_rev(const NodeQ<double>& A, const NodeQ<double>& B, int dir, double inv_gm1,
                                            const double g[4], double gA[NQ], double gB[NQ]) {
  // forward
  const double dr = B.rho - A.rho, sr = A.rho + B.rho;
  const double db = B.beta - A.beta, sb = A.beta + B.beta;
  const bool ser_r = near_pair(A.rho, B.rho);
  const bool ser_b = near_pair(A.beta, B.beta);
  const double den_r = ser_r ? sr : B.lnrho - A.lnrho;
  const double den_b = ser_b ? sb : db;
  const double r = rcp_val(den_r * den_b);
  const double qr = den_b * r, qb = den_r * r;
  const double fr = dr * qr;
  const double ur = fr * fr;
  const double Hr = ser_r ? series_H(ur) : 0.0;
  const double rho_ln = ser_r ? sr * Hr : fr;
  const double fb = db * qb;
  const double ub = fb * fb;
  const double A2 = ser_b ? series_2A(ub) : 0.0;
  const double dlb = B.lnbeta - A.lnbeta;
  const double ibeta = ser_b ? qb * A2 : dlb * qb;
  const double v1m = A.hv1 + B.hv1, v2m = A.hv2 + B.hv2;
  const double vnA = dir ? A.v2 : A.v1, vnB = dir ? B.v2 : B.v1;
  const double vnm = dir ? v2m : v1m;
  const double frho = rho_ln * vnm;
  const double kin = fma(A.hv1, B.v1, A.hv2 * B.v2);
  const double T = fma(ibeta, inv_gm1, kin);
  // reverse
  double g_v1m = g[1] * frho, g_v2m = g[2] * frho;
  const double g_frho = g[0] + g[1] * v1m + g[2] * v2m + g[3] * T;
  const double g_pm = dir ? g[2] : g[1];
  const double g_T = g[3] * frho;
  const double g_ibeta = g_T * inv_gm1;
  const double g_kin = g_T;
  gA[Q_HP] += g[3] * vnB + g_pm;
  gB[Q_HP] += g[3] * vnA + g_pm;
  const double g_vnB = g[3] * A.hp, g_vnA = g[3] * B.hp;
  gA[Q_HV1] += g_kin * B.v1;
  gB[Q_V1] += g_kin * A.hv1;
  gA[Q_HV2] += g_kin * B.v2;
  gB[Q_V2] += g_kin * A.hv2;
  const double g_rho_ln = g_frho * vnm;
  const double g_vnm = g_frho * rho_ln;
  if (dir) {
    g_v2m += g_vnm;
    gA[Q_V2] += g_vnA;
    gB[Q_V2] += g_vnB;
  } else {
    g_v1m += g_vnm;
    gA[Q_V1] += g_vnA;
    gB[Q_V1] += g_vnB;
  }
  gA[Q_HV1] += g_v1m;
  gB[Q_HV1] += g_v1m;
  gA[Q_HV2] += g_v2m;
  gB[Q_HV2] += g_v2m;
  // 1 / {{beta}}_ln
  double g_qb = 0.0, g_db = 0.0, g_sb = 0.0;
  if (ser_b) {
    g_qb += g_ibeta * A2;
    const double g_fb = 2.0 * fb * (g_ibeta * qb * series_2A_d(ub));
    g_db += g_fb * qb;
    g_qb += g_fb * db;
  } else {
    gB[Q_LNBETA] += g_ibeta * qb;
    gA[Q_LNBETA] -= g_ibeta * qb;
    g_qb += g_ibeta * dlb;
  }
  // {{rho}}_ln
  double g_sr = 0.0, g_fr;
  if (ser_r) {
    g_sr += g_rho_ln * Hr;
    g_fr = 2.0 * fr * (g_rho_ln * sr * series_H_d(ur));
  } else {
    g_fr = g_rho_ln;
  }
  const double g_dr = g_fr * qr;
  const double g_qr = g_fr * dr;
  // qr = 1/den_r, qb = 1/den_b
  const double g_den_r = -g_qr * qr * qr;
  const double g_den_b = -g_qb * qb * qb;
  if (ser_r) {
    g_sr += g_den_r;
  } else {
    gB[Q_LNRHO] += g_den_r;
    gA[Q_LNRHO] -= g_den_r;
  }
  if (ser_b)
    g_sb += g_den_b;
  else
    g_db += g_den_b;
  gA[Q_RHO] += g_sr - g_dr;
  gB[Q_RHO] += g_sr + g_dr;
  gA[Q_BETA] += g_sb - g_db;
  gB[Q_BETA] += g_sb + g_db;
}

// adjoint of the node quantities with respect to the conserved state u
__device__ __forceinline__ void node_q_rev(const double u[4], const NodeQ<double>& q, double gm1, const double gq[NQ],
                                           double gu[4]) {
  const double rho = q.rho, ir = rcp_val(rho);
  const double beta = q.beta;
  const double ip = beta * ir;                 // 1/p = (rho/p)/rho
  double g_rho = gq[Q_RHO] + gq[Q_LNRHO] * ir;
  const double g_beta = gq[Q_BETA] + gq[Q_LNBETA] * rcp_val(beta);
  const double g_v1 = gq[Q_V1] + 0.5 * gq[Q_HV1];
  const double g_v2 = gq[Q_V2] + 0.5 * gq[Q_HV2];
  double g_p = 0.5 * gq[Q_HP];
  g_rho += g_beta * ip;                        // beta = rho / p
  g_p -= g_beta * beta * ip;
  const double v1 = q.v1, v2 = q.v2;
  gu[0] = g_rho - (g_v1 * v1 + g_v2 * v2) * ir + g_p * gm1 * 0.5 * (v1 * v1 + v2 * v2);
  gu[1] = g_v1 * ir - g_p * gm1 * v1;
  gu[2] = g_v2 * ir - g_p * gm1 * v2;
  gu[3] = g_p * gm1;
}

// ---------------------------------------------------------------------------
// Reverse sweeps of the surface fluxes (HLL, HLLC, EC), written out by hand.
// Everything happens in the face frame (rho, m_n, m_t, E); the adjoint of the
// rotated flux comes in, the adjoints of both rotated states go out.
struct SideF {
  double rho, mn, mt, E, ir, v, p, c;
};
struct SideG {
  double rho = 0, mn = 0, mt = 0, E = 0, ir = 0, v = 0, p = 0, c = 0;
};

__device__ __forceinline__ void side_fwd(const double u[4], int dir, const Ops& ops, SideF& s) {
  s.rho = u[0];
  s.mn = dir ? u[2] : u[1];
  s.mt = dir ? u[1] : u[2];
  s.E = u[3];
  s.ir = rcp_val(s.rho);
  s.v = s.mn * s.ir;
  s.p = ops.gm1 * (s.E - 0.5 * s.ir * (s.mn * s.mn + s.mt * s.mt));
  s.c = sqrt(ops.gamma * s.p * s.ir);
}

// adjoints of (ir, v, p, c) -> adjoints of (rho, mn, mt, E), then rotated back to u's order
__device__ __forceinline__ void side_rev(const SideF& s, SideG& g, int dir, const Ops& ops, double gu[4]) {
  if (s.c > 0.0) {
    const double h = 0.5 * ops.gamma / s.c;
    g.p += g.c * h * s.ir;
    g.ir += g.c * h * s.p;
  }
  g.E += ops.gm1 * g.p;
  g.ir -= 0.5 * ops.gm1 * (s.mn * s.mn + s.mt * s.mt) * g.p;
  const double g_e2 = -0.5 * ops.gm1 * s.ir * g.p;
  g.mn += 2.0 * s.mn * g_e2 + s.ir * g.v;
  g.mt += 2.0 * s.mt * g_e2;
  g.ir += s.mn * g.v;
  g.rho -= s.ir * s.ir * g.ir;
  gu[0] = g.rho;
  gu[1] = dir ? g.mt : g.mn;
  gu[2] = dir ? g.mn : g.mt;
  gu[3] = g.E;
}

// physical flux F = (mn, mn v + p, mt v, (E + p) v) of one side: adjoint G -> side adjoints
__device__ __forceinline__ void phys_rev(const SideF& s, const double G[4], SideG& g) {
  g.mn += G[0] + G[1] * s.v;
  g.v += G[1] * s.mn + G[2] * s.mt + G[3] * (s.E + s.p);
  g.p += G[1] + G[3] * s.v;
  g.mt += G[2] * s.v;
  g.E += G[3] * s.v;
}
__device__ __forceinline__ void phys_fwd(const SideF& s, double F[4]) {
  F[0] = s.mn;
  F[1] = s.mn * s.v + s.p;
  F[2] = s.mt * s.v;
  F[3] = (s.E + s.p) * s.v;
}

// Davis speeds: route the adjoints of S_L = min(..), S_R = max(..) to the chosen arguments
__device__ __forceinline__ void speeds_rev(const SideF& L, const SideF& R, double gSL, double gSR, SideG& gl,
                                           SideG& gr) {
  if (L.v - L.c <= R.v - R.c) {
    gl.v += gSL;
    gl.c -= gSL;
  } else {
    gr.v += gSL;
    gr.c -= gSL;
  }
  if (L.v + L.c >= R.v + R.c) {
    gl.v += gSR;
    gl.c += gSR;
  } else {
    gr.v += gSR;
    gr.c += gSR;
  }
}

__device__ void hll_rev(const double uL[4], const double uR[4], int dir, const Ops& ops, const double gf[4],
                        double guL[4], double guR[4]) {
  SideF L, R;
  side_fwd(uL, dir, ops, L);
  side_fwd(uR, dir, ops, R);
  const double G[4] = {gf[0], dir ? gf[2] : gf[1], dir ? gf[1] : gf[2], gf[3]};
  SideG gl, gr;
  const double SL = fmin(L.v - L.c, R.v - R.c), SR = fmax(L.v + L.c, R.v + R.c);
  if (SL >= 0.0) {
    phys_rev(L, G, gl);
  } else if (SR <= 0.0) {
    phys_rev(R, G, gr);
  } else {
    double FL[4], FR[4], F[4];
    phys_fwd(L, FL);
    phys_fwd(R, FR);
    const double iD = rcp_val(SR - SL);
    const double dU[4] = {R.rho - L.rho, R.mn - L.mn, R.mt - L.mt, R.E - L.E};
    double gSL = 0.0, gSR = 0.0, GL[4], GR[4];
    for (int v = 0; v < 4; ++v) {
      F[v] = (SR * FL[v] - SL * FR[v] + SL * SR * dU[v]) * iD;
      GL[v] = G[v] * SR * iD;
      GR[v] = -G[v] * SL * iD;
      gSR += G[v] * (FL[v] + SL * dU[v] - F[v]) * iD;
      gSL += G[v] * (-FR[v] + SR * dU[v] + F[v]) * iD;
    }
    phys_rev(L, GL, gl);
    phys_rev(R, GR, gr);
    const double w = SL * SR * iD;   // adjoint of dU
    gr.rho += G[0] * w; gl.rho -= G[0] * w;
    gr.mn += G[1] * w;  gl.mn -= G[1] * w;
    gr.mt += G[2] * w;  gl.mt -= G[2] * w;
    gr.E += G[3] * w;   gl.E -= G[3] * w;
    speeds_rev(L, R, gSL, gSR, gl, gr);
  }
  side_rev(L, gl, dir, ops, guL);
  side_rev(R, gr, dir, ops, guR);
}

__device__ void hllc_rev(const double uL[4], const double uR[4], int dir, const Ops& ops, const double gf[4],
                         double guL[4], double guR[4]) {
  SideF L, R;
  side_fwd(uL, dir, ops, L);
  side_fwd(uR, dir, ops, R);
  const double G[4] = {gf[0], dir ? gf[2] : gf[1], dir ? gf[1] : gf[2], gf[3]};
  SideG gl, gr;
  const double SL = fmin(L.v - L.c, R.v - R.c), SR = fmax(L.v + L.c, R.v + R.c);
  if (SL >= 0.0) {
    phys_rev(L, G, gl);
  } else if (SR <= 0.0) {
    phys_rev(R, G, gr);
  } else {
    const double mL = L.rho * (SL - L.v), mR = R.rho * (SR - R.v);
    const double num = R.p - L.p + mL * L.v - mR * R.v, den = mL - mR;
    const double iden = rcp_val(den);
    const double Ss = num * iden;
    const bool left = Ss >= 0.0;
    const SideF& K = left ? L : R;
    SideG& gk = left ? gl : gr;
    const double S = left ? SL : SR;
    const double m = left ? mL : mR;
    const double iSmS = rcp_val(S - Ss), im = rcp_val(m);
    const double fac = m * iSmS;
    const double pm = K.p * im;
    const double X = K.E * K.ir + (Ss - K.v) * (Ss + pm);
    const double Us[4] = {fac, fac * Ss, fac * K.mt * K.ir, fac * X};
    const double Uk[4] = {K.rho, K.mn, K.mt, K.E};
    // F = F_K + S (Us - U_K)
    phys_rev(K, G, gk);
    double gS = 0.0;
    for (int v = 0; v < 4; ++v) gS += G[v] * (Us[v] - Uk[v]);
    gk.rho -= S * G[0];
    gk.mn -= S * G[1];
    gk.mt -= S * G[2];
    gk.E -= S * G[3];
    const double gUs[4] = {S * G[0], S * G[1], S * G[2], S * G[3]};
    double g_fac = gUs[0] + gUs[1] * Ss + gUs[2] * K.mt * K.ir + gUs[3] * X;
    double g_Ss = gUs[1] * fac;
    gk.mt += gUs[2] * fac * K.ir;
    gk.ir += gUs[2] * fac * K.mt;
    const double gX = gUs[3] * fac;
    gk.E += gX * K.ir;
    gk.ir += gX * K.E;
    g_Ss += gX * ((Ss + pm) + (Ss - K.v));
    gk.v -= gX * (Ss + pm);
    const double g_pm = gX * (Ss - K.v);
    gk.p += g_pm * im;
    double g_m = -g_pm * pm * im;
    // fac = m / (S - S*)
    g_m += g_fac * iSmS;
    gS -= g_fac * fac * iSmS;
    g_Ss += g_fac * fac * iSmS;
    // S* = num / den
    const double g_num = g_Ss * iden, g_den = -g_Ss * Ss * iden;
    double g_mL = (left ? g_m : 0.0) + g_num * L.v + g_den;
    double g_mR = (left ? 0.0 : g_m) - g_num * R.v - g_den;
    gr.p += g_num;
    gl.p -= g_num;
    gl.v += g_num * mL;
    gr.v -= g_num * mR;
    // m_K = rho_K (S_K - v_K)
    double gSL = left ? gS : 0.0, gSR = left ? 0.0 : gS;
    gl.rho += g_mL * (SL - L.v);
    gSL += g_mL * L.rho;
    gl.v -= g_mL * L.rho;
    gr.rho += g_mR * (SR - R.v);
    gSR += g_mR * R.rho;
    gr.v -= g_mR * R.rho;
    speeds_rev(L, R, gSL, gSR, gl, gr);
  }
  side_rev(L, gl, dir, ops, guL);
  side_rev(R, gr, dir, ops, guR);
}

__device__ void ec_surface_rev(const double uL[4], const double uR[4], int dir, const Ops& ops, const double* ic,
                               const double* lc, const double gf[4], double guL[4], double guR[4]) {
  const NodeQ<double> A = node_q(uL, ops.gm1, ic, lc), B = node_q(uR, ops.gm1, ic, lc);
  double gA[NQ] = {}, gB[NQ] = {};
  ec_flux_rev(A, B, dir, ops.inv_gm1, gf, gA, gB);
  node_q_rev(uL, A, ops.gm1, gA, guL);
  node_q_rev(uR, B, ops.gm1, gB, guR);
}

__device__ __forceinline__ void surface_flux_rev(const double uL[4], const double uR[4], int dir, const Ops& ops,
                                                 const double* ic, const double* lc, const double gf[4],
                                                 double guL[4], double guR[4]) {
  if (ops.surface_flux == PERK_SURFACE_HLLC)
    hllc_rev(uL, uR, dir, ops, gf, guL, guR);
  else if (ops.surface_flux == PERK_SURFACE_EC)
    ec_surface_rev(uL, uR, dir, ops, ic, lc, gf, guL, guR);
  else
    hll_rev(uL, uR, dir, ops, gf, guL, guR);
}

// Faces: the adjoint weight of every face-node flux (its lifting coefficients times
// lam on both sides) through the hand-written reverse sweeps.
// face reverse blocks: 4 threads per interface, 8 per mortar
constexpr int FREV_THREADS = 64, FREV_IF = FREV_THREADS / 4, FREV_MORT = FREV_THREADS / 8;

template <int YS>
__global__ void __launch_bounds__(FREV_THREADS) k_vjp_faces_rev(Ops ops, int64_t n_if, const int4* __restrict__ ifs,
                                                        int64_t n_mort, const int4* __restrict__ morts,
                                                        int64_t if_blocks, const int32_t* __restrict__ level,
                                                        const int32_t* __restrict__ method, int min_member,
                                                        double two_over_len, StageArgs sa,
                                                        const double* __restrict__ lam,
                                                        const double* __restrict__ logt, double* __restrict__ gsurf) {
  __shared__ double s_gphi[FREV_MORT][4][NN];
  __shared__ double s_gui[FREV_MORT][2][4][NN];
  const double* ic = logt;
  const double* lc = logt + LOG_TABLE_SIZE;
  const double iw = ops.inv_w0;
  auto load = [&](int64_t e, int node, double u[4]) { stage_y<YS>(sa, method, e, node, u); };
  if (blockIdx.x < if_blocks) {
    const int64_t idx = (int64_t)blockIdx.x * FREV_IF + (threadIdx.x >> 2);
    const int k = threadIdx.x & 3;
    if (idx >= n_if) return;
    const int4 r = ifs[idx];
    const int dir = r.z;
    const int fL = 2 * dir + 1, fR = 2 * dir;
    double uL[4], uR[4], gl[4], gr[4];
    load(r.x, face_node(fL, k), uL);
    load(r.y, face_node(fR, k), uR);
    const double cL = lift_coef(fL, two_over_len, level[r.x], iw);
    const double cR = lift_coef(fR, two_over_len, level[r.y], iw);
    double gf[4];
    for (int v = 0; v < 4; ++v)
      gf[v] = cL * lam[(int64_t)r.x * ELEM + v * NODES + face_node(fL, k)] +
              cR * lam[(int64_t)r.y * ELEM + v * NODES + face_node(fR, k)];
    surface_flux_rev(uL, uR, dir, ops, ic, lc, gf, gl, gr);
    for (int c = 0; c < 4; ++c) {
      gsurf[(int64_t)r.x * ELEM + fL * 16 + 4 * c + k] = gl[c];
      gsurf[(int64_t)r.y * ELEM + fR * 16 + 4 * c + k] = gr[c];
    }
    return;
  }
  const int lm = threadIdx.x >> 3;
  const int64_t idx = (int64_t)(blockIdx.x - if_blocks) * FREV_MORT + lm;
  const int half = (threadIdx.x >> 2) & 1, k = threadIdx.x & 3;
  const bool valid = idx < n_mort;
  int4 r = valid ? morts[idx] : make_int4(0, 0, 0, 0);
  const int dir = r.w & 1, large_side = (r.w >> 1) & 1;
  const int large_face = large_side == 0 ? 2 * dir + 1 : 2 * dir;
  const int small_face = large_side == 0 ? 2 * dir : 2 * dir + 1;
  const int small = half ? r.z : r.y;
  if (valid && half == 0) {
    const double cl = method[r.x] >= min_member ? lift_coef(large_face, two_over_len, level[r.x], iw) : 0.0;
    for (int v = 0; v < 4; ++v) s_gphi[lm][v][k] = cl * lam[(int64_t)r.x * ELEM + v * NODES + face_node(large_face, k)];
  }
  __syncthreads();
  if (valid) {
    double ui[4] = {0.0, 0.0, 0.0, 0.0}, us[4], gi[4], gs[4];
    for (int l = 0; l < NN; ++l) {
      const double w = half ? ops.p_hi[k][l] : ops.p_lo[k][l];
      double ul[4];
      load(r.x, face_node(large_face, l), ul);
      for (int v = 0; v < 4; ++v) ui[v] = fma(w, ul[v], ui[v]);
    }
    load(small, face_node(small_face, k), us);
    const double cs = lift_coef(small_face, two_over_len, level[small], iw);
    double gf[4];
    for (int v = 0; v < 4; ++v) {
      double g = cs * lam[(int64_t)small * ELEM + v * NODES + face_node(small_face, k)];
      for (int m = 0; m < NN; ++m) g = fma(half ? ops.r_hi[m][k] : ops.r_lo[m][k], s_gphi[lm][v][m], g);
      gf[v] = g;
    }
    if (large_side == 0)
      surface_flux_rev(ui, us, dir, ops, ic, lc, gf, gi, gs);
    else
      surface_flux_rev(us, ui, dir, ops, ic, lc, gf, gs, gi);
    for (int c = 0; c < 4; ++c) {
      gsurf[(int64_t)small * ELEM + small_face * 16 + 4 * c + k] = gs[c];
      s_gui[lm][half][c][k] = gi[c];
    }
  }
  __syncthreads();
  if (valid) {
    for (int cc = 0; cc < 2; ++cc) {
      const int c = 2 * half + cc;
      double g = 0.0;
      for (int l = 0; l < NN; ++l) {
        g = fma(ops.p_lo[l][k], s_gui[lm][0][c][l], g);
        g = fma(ops.p_hi[l][k], s_gui[lm][1][c][l], g);
      }
      gsurf[(int64_t)r.x * ELEM + large_face * 16 + 4 * c + k] = g;
    }
  }
}

// Element kernel over the active prefix of the sorted list (the volume adjoint
// by the reverse sweep above); g receives the volume part only.  Each group of
// 16 threads (one per node) strides over the active elements, so that a grid
// sized to the resident capacity keeps every SM busy to the end.  The face
// adjoints (gsurf) are gathered afterwards by face_gather.
constexpr int VJP_ELEMS = 4;

template <int YS>
__global__ void __launch_bounds__(64) k_vjp_volume(Ops ops, int64_t n_act, const int32_t* __restrict__ elems,
                                                    const int32_t* __restrict__ level,
                                                    const int32_t* __restrict__ method, double two_over_len,
                                                    StageArgs sa, const double* __restrict__ lam,
                                                    const double* __restrict__ logt, double* __restrict__ g) {
  __shared__ NodeQ<double> s_q[VJP_ELEMS][NODES];
  __shared__ double s_mu[VJP_ELEMS][4][NODES];       // -(2/h) lam at the nodes
  __shared__ double s_g[VJP_ELEMS][48][2 * NQ];       // per pair: adjoints of its two node records
  __shared__ double s_log[2 * LOG_TABLE_SIZE];
  const int le = threadIdx.x >> 4, t = threadIdx.x & 15, i = t & 3, j = t >> 2;
  const unsigned gmask = 0xFFFFu << (threadIdx.x & 16);   // the 16 lanes of this group
  for (int q = threadIdx.x; q < 2 * LOG_TABLE_SIZE; q += 64) s_log[q] = logt[q];
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * VJP_ELEMS;
  for (int64_t slot = (int64_t)blockIdx.x * VJP_ELEMS + le; slot < n_act; slot += stride) {
    const int64_t e = elems[slot];
    double y[4];
    stage_y<YS>(sa, method, e, t, y);
    const double scale = -ldexp(two_over_len, level[e]);
    __syncwarp(gmask);   // the previous element's shared records are consumed
    for (int v = 0; v < 4; ++v) s_mu[le][v][t] = scale * lam[e * ELEM + v * NODES + t];
    const NodeQ<double> myq = node_q(y, ops.gm1, s_log, s_log + LOG_TABLE_SIZE);
    s_q[le][t] = myq;
    __syncwarp(gmask);
    for (int kk = 0; kk < 3; ++kk) {
      const int p = t + 16 * kk;
      const int dir = p >= 24;
      const int q = dir ? p - 24 : p;
      const int line = q / 6, qq = q - 6 * line;
      const int a = (qq >= 3) + (qq >= 5);
      const int b = qq + 1 - (a * (5 - a)) / 2;
      const int na = dir ? a * 4 + line : line * 4 + a;
      const int nb = dir ? b * 4 + line : line * 4 + b;
      double gf[4], gA[NQ], gB[NQ];
      for (int v = 0; v < 4; ++v) gf[v] = ops.dsplit[a][b] * s_mu[le][v][na] + ops.dsplit[b][a] * s_mu[le][v][nb];
      for (int m = 0; m < NQ; ++m) gA[m] = gB[m] = 0.0;
      ec_flux_rev(s_q[le][na], s_q[le][nb], dir, ops.inv_gm1, gf, gA, gB);
      for (int m = 0; m < NQ; ++m) {
        s_g[le][p][m] = gA[m];
        s_g[le][p][NQ + m] = gB[m];
      }
    }
    __syncwarp(gmask);
    double gq[NQ];
    for (int m = 0; m < NQ; ++m) gq[m] = 0.0;
    for (int mm = 0; mm < 4; ++mm) {
      if (mm != i) {
        const int p = j * 6 + pair_slot(min(i, mm), max(i, mm));
        const int side = i < mm ? 0 : NQ;
        for (int m = 0; m < NQ; ++m) gq[m] += s_g[le][p][side + m];
      }
      if (mm != j) {
        const int p = 24 + i * 6 + pair_slot(min(j, mm), max(j, mm));
        const int side = j < mm ? 0 : NQ;
        for (int m = 0; m < NQ; ++m) gq[m] += s_g[le][p][side + m];
      }
    }
    double out[4];
    node_q_rev(y, myq, ops.gm1, gq, out);
    for (int c = 0; c < 4; ++c) g[e * ELEM + c * NODES + t] = out[c];
  }
}

// adjoint of the traces of element e at node t (= 4 j + i), variable c: the
// sum over the element faces through that node of the face records in gsurf
__device__ __forceinline__ double face_gather(const double* __restrict__ gs, int c, int t) {
  const int i = t & 3, j = t >> 2;
  double o = 0.0;
  if (i == 0) o += gs[0 * 16 + 4 * c + j];
  if (i == 3) o += gs[1 * 16 + 4 * c + j];
  if (j == 0) o += gs[2 * 16 + 4 * c + i];
  if (j == 3) o += gs[3 * 16 + 4 * c + i];
  return o;
}

// g = (volume part if the element is active, else 0) + its face adjoints:
// the complete J(Y)^T lam of one partitioned RHS evaluation
__global__ void k_vjp_gather(int64_t n, const int32_t* __restrict__ method, int min_member,
                             const double* __restrict__ gsurf, double* __restrict__ g) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * ELEM; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = q / ELEM;
    const int r = (int)(q - e * ELEM);
    const double vol = method[e] >= min_member ? g[q] : 0.0;
    g[q] = vol + face_gather(gsurf + e * ELEM, r >> 4, r & 15);
  }
}

// adjoint of the stage combination, with gq = J(Y_i)^T lam_i formed as in
// k_vjp_gather: lamU += gq; lamK1 += dt alpha gq; lamKp (+)= dt beta gq
// (lamKp may alias lamK1; assign_p: lamKp receives its first contribution, no prior zeroing)
// face_gather that also clears the entries it read (each face entry belongs to one node), so that
// the face adjoints start from zero at the next stage without a separate clearing pass
__device__ __forceinline__ double face_gather_clear(double* __restrict__ gs, int c, int t) {
  const int i = t & 3, j = t >> 2;
  double o = 0.0;
  if (i == 0) { o += gs[0 * 16 + 4 * c + j]; gs[0 * 16 + 4 * c + j] = 0.0; }
  if (i == 3) { o += gs[1 * 16 + 4 * c + j]; gs[1 * 16 + 4 * c + j] = 0.0; }
  if (j == 0) { o += gs[2 * 16 + 4 * c + i]; gs[2 * 16 + 4 * c + i] = 0.0; }
  if (j == 3) { o += gs[3 * 16 + 4 * c + i]; gs[3 * 16 + 4 * c + i] = 0.0; }
  return o;
}

// Over the elements elems[0 .. n) of the stage's halo (the active elements and their face
// neighbours: every element whose volume or face adjoint can be nonzero), add the gathered
// adjoint gq to lamU and the stage combination's shares to lamK1 and lamKp (assigned or added);
// the face adjoints read are cleared.  Elements outside the halo receive nothing at this stage,
// and their lamKp entries are read later only where the element is active, which it is not at
// any earlier stage.
__global__ void k_adj_accum(int64_t n, const int32_t* __restrict__ elems, const int32_t* __restrict__ method,
                            int min_member, const StageCoef* __restrict__ coef, double dt,
                            const double* __restrict__ g, double* __restrict__ gsurf, double* __restrict__ lamU,
                            double* __restrict__ lamK1, double* lamKp, int assign_p) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * ELEM; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t slot = q / ELEM;
    const int r = (int)(q - slot * ELEM);
    const int64_t e = elems[slot];
    const int m = method[e];
    const double gq = (m >= min_member ? g[e * ELEM + r] : 0.0) + face_gather_clear(gsurf + e * ELEM, r >> 4, r & 15);
    const int64_t qe = e * ELEM + r;
    lamU[qe] += gq;
    if (coef) {
      const StageCoef c = coef[m];
      if (lamKp == lamK1) {
        lamK1[qe] += dt * (c.alpha + c.beta) * gq;
      } else {
        lamK1[qe] += dt * c.alpha * gq;
        lamKp[qe] = assign_p ? dt * c.beta * gq : lamKp[qe] + dt * c.beta * gq;
      }
    }
  }
}

// final-update adjoint seed: lamU = lam; lamKs = dt bs lam; lamKp += dt bp lam; lamK1 += dt b1 lam
__global__ void k_adj_seed(int64_t n, double dt, double b1, double bp, double bs, const double* __restrict__ lam,
                           double* __restrict__ lamU, double* __restrict__ lamK1, double* __restrict__ lamKp,
                           double* __restrict__ lamKs) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * ELEM; q += (int64_t)gridDim.x * blockDim.x) {
    const double l = lam[q];
    lamU[q] = l;
    lamKs[q] = dt * bs * l;
    lamK1[q] = dt * b1 * l;
    if (lamKp) lamKp[q] = dt * bp * l;
  }
}

}  // namespace ad

static unsigned ew_blocks(int64_t n) {
  const int64_t b = (n * ELEM + 255) / 256, cap = (int64_t)device_sm_count() * 32;
  return (unsigned)(b > cap ? cap : (b < 1 ? 1 : b));
}

cudaError_t launch_adj_accum(cudaStream_t st, int64_t n, const int32_t* elems, const int32_t* method, int min_member,
                             const StageCoef* coef, double dt, const double* g, double* gsurf, double* lamU,
                             double* lamK1, double* lamKp, int assign_p) {
  if (n <= 0) return cudaSuccess;
  ad::k_adj_accum<<<ew_blocks(n), 256, 0, st>>>(n, elems, method, min_member, coef, dt, g, gsurf, lamU, lamK1, lamKp,
                                                assign_p);
  return cudaGetLastError();
}

cudaError_t launch_adj_seed(cudaStream_t st, int64_t n, double dt, double b1, double bp, double bs, const double* lam,
                            double* lamU, double* lamK1, double* lamKp, double* lamKs) {
  ad::k_adj_seed<<<ew_blocks(n), 256, 0, st>>>(n, dt, b1, bp, bs, lam, lamU, lamK1, lamKp, lamKs);
  return cudaGetLastError();
}

cudaError_t launch_jvp(cudaStream_t st, const Ops& ops, int64_t n_if, const int4* ifs, int64_t n_mort,
                       const int4* morts, int64_t n_el, const int32_t* elems, const int32_t* level,
                       double two_over_len, const double* Y, const double* V, const double* logt, double* surf,
                       double* surf_d, double* K, double* Kd) {
  const int64_t bi = (n_if + 31) / 32, bm = (n_mort + 15) / 16;
  if (bi + bm > 0)
    ad::k_jvp_faces<<<(unsigned)(bi + bm), 128, 0, st>>>(ops, n_if, ifs, n_mort, morts, bi, Y, V, logt, surf, surf_d);
  if (n_el > 0)
    ad::k_jvp_volume<<<(unsigned)((n_el + 7) / 8), 128, 0, st>>>(ops, n_el, elems, level, two_over_len, Y, V, surf,
                                                                 surf_d, logt, K, Kd);
  return cudaGetLastError();
}

cudaError_t launch_vjp_faces(cudaStream_t st, YSource ysrc, const Ops& ops, int64_t n_if, const int4* ifs,
                             int64_t n_mort, const int4* morts, int64_t n_all, const int32_t* level,
                             const int32_t* method, int min_member, double two_over_len, const StageArgs& sa,
                             const double* lam, const double* logt, double* gsurf, bool clear) {
  if (clear) {
    cudaError_t e = cudaMemsetAsync(gsurf, 0, (size_t)n_all * ELEM * sizeof(double), st);
    if (e != cudaSuccess) return e;
  }
  const int64_t bi = (n_if + ad::FREV_IF - 1) / ad::FREV_IF, bm = (n_mort + ad::FREV_MORT - 1) / ad::FREV_MORT;
  if (bi + bm == 0) return cudaSuccess;
  if (ysrc == Y_GIVEN)
    ad::k_vjp_faces_rev<Y_GIVEN><<<(unsigned)(bi + bm), ad::FREV_THREADS, 0, st>>>(
        ops, n_if, ifs, n_mort, morts, bi, level, method, min_member, two_over_len, sa, lam, logt, gsurf);
  else
    ad::k_vjp_faces_rev<Y_COMBINE><<<(unsigned)(bi + bm), ad::FREV_THREADS, 0, st>>>(
        ops, n_if, ifs, n_mort, morts, bi, level, method, min_member, two_over_len, sa, lam, logt, gsurf);
  return cudaGetLastError();
}

// blocks of the volume VJP: at most what is resident at once (the kernel strides); the capacity is
// computed once per device (a repeated computation by racing threads gives the same value)
template <int YS>
static unsigned vjp_volume_blocks(int64_t n_act) {
  constexpr int MAX_DEVICES = 64;
  static int cached[MAX_DEVICES] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  int resident = (dev >= 0 && dev < MAX_DEVICES) ? cached[dev] : 0;
  if (resident == 0) {
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ad::k_vjp_volume<YS>, 64, 0);
    resident = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    if (dev >= 0 && dev < MAX_DEVICES) cached[dev] = resident;
  }
  const int64_t need = (n_act + ad::VJP_ELEMS - 1) / ad::VJP_ELEMS;
  return (unsigned)(need < resident ? need : resident);
}

cudaError_t launch_vjp_volume(cudaStream_t st, YSource ysrc, const Ops& ops, int64_t n_act, const int32_t* elems,
                              const int32_t* level, const int32_t* method, double two_over_len,
                              const StageArgs& sa, const double* lam, const double* logt, double* g) {
  if (n_act <= 0) return cudaSuccess;
  if (ysrc == Y_GIVEN)
    ad::k_vjp_volume<Y_GIVEN><<<vjp_volume_blocks<Y_GIVEN>(n_act), 64, 0, st>>>(ops, n_act, elems, level, method,
                                                                              two_over_len, sa, lam, logt, g);
  else
    ad::k_vjp_volume<Y_COMBINE><<<vjp_volume_blocks<Y_COMBINE>(n_act), 64, 0, st>>>(ops, n_act, elems, level, method,
                                                                                  two_over_len, sa, lam, logt, g);
  return cudaGetLastError();
}

cudaError_t launch_vjp_gather(cudaStream_t st, int64_t n, const int32_t* method, int min_member, const double* gsurf,
                              double* g) {
  if (n <= 0) return cudaSuccess;
  ad::k_vjp_gather<<<ew_blocks(n), 256, 0, st>>>(n, method, min_member, gsurf, g);
  return cudaGetLastError();
}

}  // namespace perk
