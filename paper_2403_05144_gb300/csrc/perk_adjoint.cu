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
// Adjoint fields of a node's quantities.  The half velocities v/2 of the node records enter the
// flux through the arithmetic means; their adjoints are folded into those of v1 and v2 (a
// contribution g to v/2 is one of g/2 to v), so that a pair passes seven values per side on to
// its nodes, and five where both logarithmic means take their series (no logarithm is read).
//   0 rho, 1 beta = rho/p, 2 v1, 3 v2, 4 p/2, 5 ln rho, 6 ln beta
enum { F_RHO = 0, F_BETA, F_V1, F_V2, F_HP, F_LNRHO, F_LNBETA, NF };
constexpr int NF_SER = F_LNRHO;   // fields of a pair whose means both take their series
// Adjoint accumulators start at -0.0, not +0.0: -0.0 + x is x exactly for every x, so the
// compiler drops the first addition into each of them (+0.0 + x differs from x for x = -0.0
// and must be kept).

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

// The part of the reverse sweep shared by both branches of the means: given the adjoint g of the
// flux f#(A, B) in direction dir and the forward values rho_ln, 1/{{beta}}_ln (ibeta), accumulate
// the adjoints of the velocities and of p/2 into gA, gB and return those of rho_ln and ibeta.
__device__ __forceinline__ void ec_flux_rev_common(const NodeQ<double>& A, const NodeQ<double>& B, int dir,
                                                   double inv_gm1, const double g[4], double rho_ln, double ibeta,
                                                   double* gA, double* gB, double& g_rho_ln, double& g_ibeta) {
  const double v1m = A.hv1 + B.hv1, v2m = A.hv2 + B.hv2;
  const double vnA = dir ? A.v2 : A.v1, vnB = dir ? B.v2 : B.v1;
  const double vnm = dir ? v2m : v1m;
  const double frho = rho_ln * vnm;
  const double kin = fma(A.hv1, B.v1, A.hv2 * B.v2);
  const double T = fma(ibeta, inv_gm1, kin);
  // f = (frho, frho v1m + [dir = 0] pm, frho v2m + [dir = 1] pm, frho T + (A.hp vnB + B.hp vnA))
  const double g_frho = fma(g[3], T, fma(g[2], v2m, fma(g[1], v1m, g[0])));
  const double g_pm = dir ? g[2] : g[1];
  const double g_T = g[3] * frho;                  // = adjoint of kin
  g_ibeta = g_T * inv_gm1;
  g_rho_ln = g_frho * vnm;
  gA[F_HP] += fma(g[3], vnB, g_pm);
  gB[F_HP] += fma(g[3], vnA, g_pm);
  // half the adjoints of the means v1m, v2m (each mean is (vA + vB)/2)
  const double hfrho = 0.5 * frho, hrho_ln = 0.5 * rho_ln;
  double h1 = g[1] * hfrho, h2 = g[2] * hfrho;
  if (dir)
    h2 = fma(g_frho, hrho_ln, h2);
  else
    h1 = fma(g_frho, hrho_ln, h1);
  // kin = (A.v1 B.v1 + A.v2 B.v2) / 2
  gA[F_V1] += fma(g_T, B.hv1, h1);
  gB[F_V1] += fma(g_T, A.hv1, h1);
  gA[F_V2] += fma(g_T, B.hv2, h2);
  gB[F_V2] += fma(g_T, A.hv2, h2);
  // the normal velocities of the pressure term
  if (dir) {
    gA[F_V2] += g[3] * B.hp;
    gB[F_V2] += g[3] * A.hp;
  } else {
    gA[F_V1] += g[3] * B.hp;
    gB[F_V1] += g[3] * A.hp;
  }
}

// Series branch of a logarithmic mean, m = s M(u), u = (d/s)^2 (d = b - a, s = a + b; M = H for
// {{rho}}_ln, and 1/{{beta}}_ln = M(u)/s with M = 2A): the adjoints of s and d from that of m,
// from the derivative of the closed form (dm/dd = 2 (d/s) M'(u) for H; for 2A the 1/s factor adds
// -m/s to dm/ds).  Differentiating the closed form rather than the shared reciprocal of the
// forward evaluation changes the result only by rounding.
__device__ __forceinline__ void ser_rho_rev(double g, double H, double Hd, double ur, double fr, double& g_s,
                                            double& g_d) {
  g_s = g * fma(-2.0 * ur, Hd, H);          // d(s H)/ds = H - 2 u H'
  g_d = g * ((fr + fr) * Hd);               // d(s H)/dd = 2 f H'
}
__device__ __forceinline__ void ser_beta_rev(double g, double A2, double A2d, double ub, double fb, double isb,
                                             double& g_s, double& g_d) {
  const double w = g * (isb * isb);
  g_s = -w * fma(ub + ub, A2d, A2);         // d(2A/s)/ds = -(2A + 2 u (2A)') / s^2
  g_d = w * ((fb + fb) * A2d);              // d(2A/s)/dd = 2 f (2A)' / s^2
}

// Given the adjoint g of the flux f#(A, B) in direction dir, accumulate the adjoints of A's and
// B's node quantities (NF fields) into gA, gB: the forward intermediates are recomputed, branch
// decisions as in the forward flux.
__device__ __forceinline__ void ec_flux_rev(const NodeQ<double>& A, const NodeQ<double>& B, int dir, double inv_gm1,
                                            const double g[4], double gA[NF], double gB[NF]) {
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
  double g_rho_ln, g_ibeta;
  ec_flux_rev_common(A, B, dir, inv_gm1, g, rho_ln, ibeta, gA, gB, g_rho_ln, g_ibeta);
  // {{rho}}_ln: series s H(u), else d / (ln b - ln a)
  double g_sr, g_dr;
  if (ser_r) {
    ser_rho_rev(g_rho_ln, Hr, series_H_d(ur), ur, fr, g_sr, g_dr);
  } else {
    g_sr = -0.0;
    g_dr = g_rho_ln * qr;
    const double g_den = -g_rho_ln * fr * qr;       // d(d / D)/dD = -(d/D) / D
    gB[F_LNRHO] += g_den;
    gA[F_LNRHO] -= g_den;
  }
  // 1/{{beta}}_ln: series 2A(u) / s, else (ln b - ln a) / d
  double g_sb, g_db;
  if (ser_b) {
    ser_beta_rev(g_ibeta, A2, series_2A_d(ub), ub, fb, qb, g_sb, g_db);
  } else {
    g_sb = -0.0;
    g_db = -g_ibeta * ibeta * qb;                    // d(L / d)/dd = -(L/d) / d
    gB[F_LNBETA] += g_ibeta * qb;
    gA[F_LNBETA] -= g_ibeta * qb;
  }
  gA[F_RHO] += g_sr - g_dr;
  gB[F_RHO] += g_sr + g_dr;
  gA[F_BETA] += g_sb - g_db;
  gB[F_BETA] += g_sb + g_db;
}

// The same for a pair of an element whose node pairs all take the series of both means (known
// from the element's extremes, see series_only): five fields, no logarithm read.
__device__ __forceinline__ void ec_flux_rev_ser(const NodeQ<double>& A, const NodeQ<double>& B, int dir,
                                                double inv_gm1, const double g[4], double gA[NF_SER],
                                                double gB[NF_SER]) {
  const double dr = B.rho - A.rho, sr = A.rho + B.rho;
  const double db = B.beta - A.beta, sb = A.beta + B.beta;
  const double r = rcp_val(sr * sb);
  const double isr = sb * r, isb = sr * r;
  const double fr = dr * isr, ur = fr * fr;
  const double Hr = series_H(ur);
  const double fb = db * isb, ub = fb * fb;
  const double A2 = series_2A(ub);
  double g_rho_ln, g_ibeta;
  ec_flux_rev_common(A, B, dir, inv_gm1, g, sr * Hr, isb * A2, gA, gB, g_rho_ln, g_ibeta);
  double g_sr, g_dr, g_sb, g_db;
  ser_rho_rev(g_rho_ln, Hr, series_H_d(ur), ur, fr, g_sr, g_dr);
  ser_beta_rev(g_ibeta, A2, series_2A_d(ub), ub, fb, isb, g_sb, g_db);
  gA[F_RHO] += g_sr - g_dr;
  gB[F_RHO] += g_sr + g_dr;
  gA[F_BETA] += g_sb - g_db;
  gB[F_BETA] += g_sb + g_db;
}

// Node quantities as node_q computes them, without the logarithms (set to 0), plus 1/rho and
// p/rho = 1/beta for the reverse sweep (from the same reciprocal: rho p = (gamma-1)(rho E - |m|^2/2),
// r = 1/(rho^2 p), 1/rho = rho p r, p/rho = rho p (1/rho)^2).
__device__ __forceinline__ NodeQ<double> node_q_rec(const double u[4], double gm1, double& ir, double& ib) {
  NodeQ<double> q;
  const double rp = gm1 * fma(u[0], u[3], -0.5 * fma(u[1], u[1], u[2] * u[2]));
  const double r = rcp_val(u[0] * rp);
  ir = rp * r;
  q.rho = u[0];
  q.v1 = u[1] * ir;
  q.v2 = u[2] * ir;
  q.hp = 0.5 * (rp * ir);
  q.beta = (u[0] * u[0]) * (u[0] * r);
  q.hv1 = 0.5 * q.v1;
  q.hv2 = 0.5 * q.v2;
  q.lnrho = 0.0;
  q.lnbeta = 0.0;
  ib = (rp * ir) * ir;
  return q;
}

// adjoint of the node quantities with respect to the conserved state u (gq: NF fields, or
// NF_SER when LOGS is false and the logarithms were not read); ir = 1/rho, ib = 1/beta
template <bool LOGS>
__device__ __forceinline__ void node_q_rev(const NodeQ<double>& q, double gm1, const double* gq, double ir, double ib,
                                           double gu[4]) {
  const double beta = q.beta;
  const double ip = beta * ir;                 // 1/p = (rho/p)/rho
  double g_rho = gq[F_RHO];
  double g_beta = gq[F_BETA];
  if (LOGS) {
    g_rho = fma(gq[F_LNRHO], ir, g_rho);
    g_beta = fma(gq[F_LNBETA], ib, g_beta);
  }
  const double g_v1 = gq[F_V1], g_v2 = gq[F_V2];
  double g_p = 0.5 * gq[F_HP];
  g_rho = fma(g_beta, ip, g_rho);              // beta = rho / p
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
  double rho = -0.0, mn = -0.0, mt = -0.0, E = -0.0, ir = -0.0, v = -0.0, p = -0.0, c = -0.0;
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
    const double h = 0.5 * ops.gamma * rcp_val(s.c);
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
    double gSL = -0.0, gSR = -0.0, GL[4], GR[4];
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
    double gS = -0.0;
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
  double irA, ibA, irB, ibB;
  NodeQ<double> A = node_q_rec(uL, ops.gm1, irA, ibA), B = node_q_rec(uR, ops.gm1, irB, ibB);
  A.lnrho = log_val(A.rho, ic, lc);
  A.lnbeta = log_val(A.beta, ic, lc);
  B.lnrho = log_val(B.rho, ic, lc);
  B.lnbeta = log_val(B.beta, ic, lc);
  double gA[NF], gB[NF];
  for (int m = 0; m < NF; ++m) gA[m] = gB[m] = -0.0;
  ec_flux_rev(A, B, dir, ops.inv_gm1, gf, gA, gB);
  node_q_rev<true>(A, ops.gm1, gA, irA, ibA, guL);
  node_q_rev<true>(B, ops.gm1, gB, irB, ibB, guR);
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
// face items of one warp: 4 threads per interface (8 interfaces), 8 per mortar (4 mortars)
constexpr int FREV_IF = 32 / 4, FREV_MORT = 32 / 8;

// one warp's face item: FREV_IF interfaces (4 lanes each) or FREV_MORT mortars (8 lanes each)
struct FaceRevShared {
  double gphi[FREV_MORT][4][NN];
  double gui[FREV_MORT][2][4][NN];
};

// face item fb of a warp: interfaces fb*FREV_IF.. (fb < if_items), else mortars
template <int YS>
__device__ __forceinline__ void faces_rev_warp(const Ops& ops, int64_t fb, int64_t n_if, const int4* __restrict__ ifs,
                                               int64_t n_mort, const int4* __restrict__ morts, int64_t if_items,
                                                const int32_t* __restrict__ level,
                                                const int32_t* __restrict__ method, int min_member,
                                                double two_over_len, const StageArgs& sa,
                                                const double* __restrict__ lam, const double* __restrict__ logt,
                                                double* __restrict__ gsurf, FaceRevShared& sh) {
  auto& s_gphi = sh.gphi;
  auto& s_gui = sh.gui;
  const double* ic = logt;
  const double* lc = logt + LOG_TABLE_SIZE;
  const double iw = ops.inv_w0;
  auto load = [&](int64_t e, int node, double u[4]) { stage_y<YS>(sa, method, e, node, u); };
  const int lane = threadIdx.x & 31;
  if (fb < if_items) {
    const int64_t idx = fb * FREV_IF + (lane >> 2);
    const int k = lane & 3;
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
  const int lm = lane >> 3;
  const int64_t idx = (fb - if_items) * FREV_MORT + lm;
  const int half = (lane >> 2) & 1, k = lane & 3;
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
  __syncwarp();
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
  __syncwarp();
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

// Volume adjoint of one element per group of 16 threads (one per node); g receives the volume
// part only, the face adjoints (gsurf) are gathered afterwards.  Where every node pair of the
// element takes the series of both logarithmic means (judged from the element's extremes, as in
// the forward kernel), the pairs take the five-field sweep and no node logarithm is computed.
constexpr int VJP_ELEMS = 2;   // elements of a warp's volume item

// the pairs of one element (three per thread) and the adjoint of this thread's node
// (mu: -(2/h) lam at this thread's node; the pairs read their nodes' values by shuffles)
template <bool SER>
__device__ __forceinline__ void vjp_element(const Ops& ops, const NodeQ<double>* __restrict__ sq,
                                            const double mu[4], double (*__restrict__ sg)[2 * NF], unsigned gmask,
                                            int t, const NodeQ<double>& myq, double ir, double ib, double out[4]) {
  constexpr int K = SER ? NF_SER : NF;
  const int i = t & 3, j = t >> 2;
#pragma unroll
  for (int kk = 0; kk < 3; ++kk) {
    const int p = t + 16 * kk;
    const int dir = p >= 24;
    const int q = dir ? p - 24 : p;
    const int line = q / 6, qq = q - 6 * line;
    const int a = (qq >= 3) + (qq >= 5);
    const int b = qq + 1 - (a * (5 - a)) / 2;
    const int na = dir ? a * 4 + line : line * 4 + a;
    const int nb = dir ? b * 4 + line : line * 4 + b;
    double gf[4], gA[K], gB[K];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const double ma = __shfl_sync(gmask, mu[v], na, 16), mb = __shfl_sync(gmask, mu[v], nb, 16);
      gf[v] = ops.dsplit[a][b] * ma + ops.dsplit[b][a] * mb;
    }
#pragma unroll
    for (int m = 0; m < K; ++m) gA[m] = gB[m] = -0.0;
    if constexpr (SER)
      ec_flux_rev_ser(sq[na], sq[nb], dir, ops.inv_gm1, gf, gA, gB);
    else
      ec_flux_rev(sq[na], sq[nb], dir, ops.inv_gm1, gf, gA, gB);
#pragma unroll
    for (int m = 0; m < K; ++m) {
      sg[p][m] = gA[m];
      sg[p][K + m] = gB[m];
    }
  }
  __syncwarp(gmask);
  double gq[K];
#pragma unroll
  for (int m = 0; m < K; ++m) gq[m] = -0.0;
#pragma unroll
  for (int mm = 0; mm < 4; ++mm) {
    if (mm != i) {
      const int p = j * 6 + pair_slot(min(i, mm), max(i, mm));
      const int side = i < mm ? 0 : K;
#pragma unroll
      for (int m = 0; m < K; ++m) gq[m] += sg[p][side + m];
    }
    if (mm != j) {
      const int p = 24 + i * 6 + pair_slot(min(j, mm), max(j, mm));
      const int side = j < mm ? 0 : K;
#pragma unroll
      for (int m = 0; m < K; ++m) gq[m] += sg[p][side + m];
    }
  }
  node_q_rev<!SER>(myq, ops.gm1, gq, ir, ib, out);
}

struct VolRevShared {
  NodeQ<double> q[VJP_ELEMS][NODES];
  double g[VJP_ELEMS][48][2 * NF];      // per pair: adjoints of its two node records
};

// the volume adjoint of element elems[slot] by the 16-thread group le (node t); g receives it
template <int YS>
__device__ __forceinline__ void volume_rev_elem(const Ops& ops, int64_t slot, const int32_t* __restrict__ elems,
                                                const int32_t* __restrict__ level,
                                                const int32_t* __restrict__ method, double two_over_len,
                                                const StageArgs& sa, const double* __restrict__ lam,
                                                const double* __restrict__ logt, double* __restrict__ g,
                                                VolRevShared& sh, int le, int t, unsigned gmask) {
  const int64_t e = elems[slot];
  double y[4];
  stage_y<YS>(sa, method, e, t, y);
  const double scale = -ldexp(two_over_len, level[e]);
  double mu[4];
  for (int v = 0; v < 4; ++v) mu[v] = scale * lam[e * ELEM + v * NODES + t];
  double ir, ib;
  NodeQ<double> myq = node_q_rec(y, ops.gm1, ir, ib);
  unsigned long long rmin = dbits(myq.rho), rmax = rmin, bmin = dbits(myq.beta), bmax = bmin;
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {   // the element's 16 lanes
    rmin = min(rmin, __shfl_xor_sync(gmask, rmin, o, 16));
    rmax = max(rmax, __shfl_xor_sync(gmask, rmax, o, 16));
    bmin = min(bmin, __shfl_xor_sync(gmask, bmin, o, 16));
    bmax = max(bmax, __shfl_xor_sync(gmask, bmax, o, 16));
  }
  const bool ser = series_only(rmin, rmax, bmin, bmax);
  if (!ser) {
    myq.lnrho = log_val(myq.rho, logt, logt + LOG_TABLE_SIZE);
    myq.lnbeta = log_val(myq.beta, logt, logt + LOG_TABLE_SIZE);
  }
  __syncwarp(gmask);   // the previous element's shared records are consumed
  sh.q[le][t] = myq;
  __syncwarp(gmask);
  double out[4];
  if (ser)
    vjp_element<true>(ops, sh.q[le], mu, sh.g[le], gmask, t, myq, ir, ib, out);
  else
    vjp_element<false>(ops, sh.q[le], mu, sh.g[le], gmask, t, myq, ir, ib, out);
  for (int c = 0; c < 4; ++c) g[e * ELEM + c * NODES + t] = out[c];
}

// One launch per reverse stage: the volume items (VJP_ELEMS active elements) and the face items
// (FREV_IF interfaces or FREV_MORT mortars) of the stage, one warp each, dealt to the warps of a
// resident grid from the stage's counter *ticket (zero at launch): volume items first, so that the
// shorter face items fill the end.  The two kinds write disjoint outputs (g, gsurf) and depend on
// nothing the launch writes, so the order of the items does not change the results.
union RevWarpShared {
  VolRevShared v;
  FaceRevShared f;
};
constexpr int VJP_STAGE_THREADS = 64;

template <int YS>
__global__ void __launch_bounds__(VJP_STAGE_THREADS, 8)
    k_vjp_stage(Ops ops, int64_t n_act, const int32_t* __restrict__ elems, int64_t n_if,
                const int4* __restrict__ ifs, int64_t n_mort, const int4* __restrict__ morts, int64_t if_items,
                int64_t face_items, const int32_t* __restrict__ level, const int32_t* __restrict__ method,
                int min_member, double two_over_len, StageArgs sa, const double* __restrict__ lam,
                const double* __restrict__ logt, double* __restrict__ g, double* __restrict__ gsurf,
                unsigned long long* ticket) {
  __shared__ RevWarpShared sh[VJP_STAGE_THREADS / 32];
  const int lane = threadIdx.x & 31, le = lane >> 4, t = lane & 15;
  RevWarpShared& ws = sh[threadIdx.x >> 5];
  const unsigned gmask = 0xFFFFu << (lane & 16);
  const unsigned long long vol_items = (unsigned long long)((n_act + VJP_ELEMS - 1) / VJP_ELEMS);
  const unsigned long long items = vol_items + (unsigned long long)face_items;
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(ticket, 1ull);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= items) break;
    if (it < vol_items) {
      const int64_t slot = (int64_t)it * VJP_ELEMS + le;
      if (slot < n_act)
        volume_rev_elem<YS>(ops, slot, elems, level, method, two_over_len, sa, lam, logt, g, ws.v, le, t, gmask);
    } else {
      faces_rev_warp<YS>(ops, (int64_t)(it - vol_items), n_if, ifs, n_mort, morts, if_items, level, method,
                         min_member, two_over_len, sa, lam, logt, gsurf, ws.f);
    }
    __syncwarp();   // the item's shared records are consumed before the next item writes them
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
// Over the elements elems[0 .. n) of the stage's halo (the active elements and their face
// neighbours: every element whose volume or face adjoint can be nonzero), add the gathered
// adjoint gq to lamU and the stage combination's shares to lamK1 and lamKp (assigned or added);
// the face adjoints read are cleared, so that they start from zero at the next stage.  Elements
// outside the halo receive nothing at this stage, and their lamKp entries are read later only
// where the element is active, which it is not at any earlier stage.
// One thread per element value (node t = 4 j + i, variable c).  Every load is issued before any
// store (the volume part is loaded for every element and discarded where the element is
// inactive): with the stores of the cleared face records between them the loads would
// otherwise wait on one another, and the kernel, which mostly misses in L2 here, would run at
// a small fraction of the memory bandwidth.
__global__ void k_adj_accum(int64_t n, const int32_t* __restrict__ elems, const int32_t* __restrict__ method,
                            int min_member, const StageCoef* __restrict__ coef, double dt,
                            const double* __restrict__ g, double* __restrict__ gsurf, double* __restrict__ lamU,
                            double* lamK1, double* lamKp, int assign_p) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * ELEM) return;
  const int64_t slot = q / ELEM;
  const int r = (int)(q - slot * ELEM), c = r >> 4, t = r & 15, i = t & 3, j = t >> 2;
  const int64_t e = elems[slot];
  const int64_t qe = e * ELEM + r;
  double* gs = gsurf + e * ELEM;
  // the element faces through this node: -x / +x (i = 0 / 3) and -y / +y (j = 0 / 3)
  const int fa = i == 0 ? 4 * c + j : (i == 3 ? 16 + 4 * c + j : -1);
  const int fb = j == 0 ? 32 + 4 * c + i : (j == 3 ? 48 + 4 * c + i : -1);
  const bool alias = lamKp == lamK1;
  const int m = method[e];
  const double gv = g[qe];
  const double sa = fa >= 0 ? gs[fa] : 0.0;
  const double sb = fb >= 0 ? gs[fb] : 0.0;
  const double u = lamU[qe];
  const double k1 = coef ? lamK1[qe] : 0.0;
  const double kp = (coef && !alias && !assign_p) ? lamKp[qe] : 0.0;
  const double gq = (m >= min_member ? gv : 0.0) + (sa + sb);
  if (fa >= 0) gs[fa] = 0.0;
  if (fb >= 0) gs[fb] = 0.0;
  lamU[qe] = u + gq;
  if (coef) {
    const StageCoef cf = coef[m];
    if (alias) {
      lamK1[qe] = k1 + dt * (cf.alpha + cf.beta) * gq;
    } else {
      lamK1[qe] = k1 + dt * cf.alpha * gq;
      lamKp[qe] = assign_p ? dt * cf.beta * gq : kp + dt * cf.beta * gq;
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
  // one thread per element value: at most 2^31 - 1 blocks, i.e. 8.5e9 elements
  ad::k_adj_accum<<<(unsigned)((n * ELEM + 255) / 256), 256, 0, st>>>(n, elems, method, min_member, coef, dt, g, gsurf, lamU, lamK1, lamKp,
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

// blocks of the persistent reverse stage kernel: at most what is resident at once (it deals
// items); the capacity is computed once per device and stage-state source (a repeated
// computation by racing threads gives the same value)
template <class Kernel>
static unsigned resident_blocks(Kernel kernel, int slot, int64_t need) {
  constexpr int MAX_DEVICES = 64;
  static int cached[2][MAX_DEVICES] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  int resident = (dev >= 0 && dev < MAX_DEVICES) ? cached[slot][dev] : 0;
  if (resident == 0) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, ad::VJP_STAGE_THREADS, 0);
    resident = device_sm_count() * (per_sm > 0 ? per_sm : 1);
    if (dev >= 0 && dev < MAX_DEVICES) cached[slot][dev] = resident;
  }
  return (unsigned)(need < resident ? (need > 0 ? need : 1) : resident);
}

cudaError_t launch_vjp_stage(cudaStream_t st, YSource ysrc, const Ops& ops, int64_t n_act, const int32_t* elems,
                             int64_t n_if, const int4* ifs, int64_t n_mort, const int4* morts, const int32_t* level,
                             const int32_t* method, int min_member, double two_over_len, const StageArgs& sa,
                             const double* lam, const double* logt, double* g, double* gsurf,
                             unsigned long long* ticket) {
  // items of one warp each: the blocks needed for them, capped at the resident capacity
  const int64_t bi = (n_if + ad::FREV_IF - 1) / ad::FREV_IF, bm = (n_mort + ad::FREV_MORT - 1) / ad::FREV_MORT;
  const int64_t items = (n_act + ad::VJP_ELEMS - 1) / ad::VJP_ELEMS + bi + bm;
  if (items <= 0) return cudaSuccess;
  constexpr int WARPS = ad::VJP_STAGE_THREADS / 32;
  const int64_t blocks = (items + WARPS - 1) / WARPS;
  if (ysrc == Y_GIVEN)
    ad::k_vjp_stage<Y_GIVEN><<<resident_blocks(ad::k_vjp_stage<Y_GIVEN>, Y_GIVEN, blocks), ad::VJP_STAGE_THREADS, 0,
                               st>>>(
        ops, n_act, elems, n_if, ifs, n_mort, morts, bi, bi + bm, level, method, min_member, two_over_len, sa, lam,
        logt, g, gsurf, ticket);
  else
    ad::k_vjp_stage<Y_COMBINE><<<resident_blocks(ad::k_vjp_stage<Y_COMBINE>, Y_COMBINE, blocks),
                                 ad::VJP_STAGE_THREADS, 0, st>>>(
        ops, n_act, elems, n_if, ifs, n_mort, morts, bi, bi + bm, level, method, min_member, two_over_len, sa, lam,
        logt, g, gsurf, ticket);
  return cudaGetLastError();
}

cudaError_t launch_vjp_gather(cudaStream_t st, int64_t n, const int32_t* method, int min_member, const double* gsurf,
                              double* g) {
  if (n <= 0) return cudaSuccess;
  ad::k_vjp_gather<<<ew_blocks(n), 256, 0, st>>>(n, method, min_member, gsurf, g);
  return cudaGetLastError();
}

}  // namespace perk
