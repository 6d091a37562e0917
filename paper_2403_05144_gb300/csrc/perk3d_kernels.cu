// sm_103a kernels of the 3D P-ERK / DGSEM step (octree, hexahedral elements).
//
// One P-ERK stage (Eq. PartitionedRKSystem) is two launches over the active
// prefixes of the level-sorted lists, as in 2D:
//   k3_faces   numerical fluxes of the active interfaces (one thread per face
//              node) and mortars (one thread per small-face node; the large
//              trace interpolated to the four small faces, the four small-face
//              fluxes projected back by the exact L2 projection, both as tensor
//              products of the 1D operators);
//   k3_volume  flux-differencing volume integral over the three axes, surface
//              lifting on the six faces and the Jacobian, stage state formed on
//              the fly, one thread per node.
// k3_commit applies the guarded final update; k3_dt reduces the CFL step size.
// Templates on the nodes per direction NN = N + 1 (3 or 4).  FP64 throughout.

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "perk3d_device.cuh"
#include "perk3d_internal.h"
#include "perk_devmath.cuh"

namespace perk3 {

using perk::LOG_TABLE;
using perk::dbits;
using perk::series_only;
using perk::near_pair;
using perk::log_tab;
using perk::rcp_nr;
using perk::series_2A;
using perk::series_H;
using perk::Y_COMBINE;
using perk::Y_GIVEN;

// ---------------------------------------------------------------------------
// Two-point flux from node quantities (half values fold the 1/2 of the arithmetic means);
// padded to 96 bytes for 16-byte shared-memory loads.
struct __align__(16) NodeQ3 {
  double rho, lnrho, beta, lnbeta, v1, v2, v3, hv1, hv2, hv3, hp, pad;
};

// node quantities without the two logarithms (set to 0; see series_only)
__device__ __forceinline__ NodeQ3 node_q3_nolog(const double u[5], double gm1) {
  NodeQ3 q;
  // rho p = (gamma - 1)(rho E - |m|^2 / 2); one reciprocal gives 1/rho and rho/p
  const double rp = gm1 * fma(u[0], u[4], -0.5 * fma(u[1], u[1], fma(u[2], u[2], u[3] * u[3])));
  const double r = rcp_nr(u[0] * rp);   // 1 / (rho^2 p)
  const double ir = rp * r;             // 1 / rho
  q.rho = u[0];
  q.v1 = u[1] * ir;
  q.v2 = u[2] * ir;
  q.v3 = u[3] * ir;
  q.hp = 0.5 * (rp * ir);
  q.beta = (u[0] * u[0]) * (u[0] * r);  // rho / p
  q.hv1 = 0.5 * q.v1;
  q.hv2 = 0.5 * q.v2;
  q.hv3 = 0.5 * q.v3;
  q.lnrho = 0.0;
  q.lnbeta = 0.0;
  q.pad = 0.0;
  return q;
}

__device__ __forceinline__ NodeQ3 node_q3(const double u[5], double gm1, const double* inv_c, const double* ln_c) {
  NodeQ3 q = node_q3_nolog(u, gm1);
  q.lnrho = log_tab(q.rho, inv_c, ln_c);
  q.lnbeta = log_tab(q.beta, inv_c, ln_c);
  return q;
}

// Ranocha's entropy-conservative two-point flux along axis dir: f_rho = {{rho}}_ln {{v_n}},
// f_m = f_rho {{v}} + {{p}} n, f_E = f_rho (1/((gamma-1) {{rho/p}}_ln) + v_A . v_B / 2)
// + (p_A v_n,B + p_B v_n,A) / 2; one reciprocal serves both logarithmic means, and near-equal
// arguments take the artanh series of the mean.
__device__ __forceinline__ void ec_flux_q3(const NodeQ3& A, const NodeQ3& B, int dir, double inv_gm1, double f[5]) {
  const double dr = B.rho - A.rho, sr = A.rho + B.rho;
  const double db = B.beta - A.beta, sb = A.beta + B.beta;
  const bool ser_r = near_pair(A.rho, B.rho);
  const bool ser_b = near_pair(A.beta, B.beta);
  const double den_r = ser_r ? sr : B.lnrho - A.lnrho;
  const double den_b = ser_b ? sb : db;
  const double r = rcp_nr(den_r * den_b);
  const double qr = den_b * r;   // 1 / den_r
  const double qb = den_r * r;   // 1 / den_b
  const double fr = dr * qr;
  const double rho_ln = ser_r ? sr * series_H(fr * fr) : fr;
  double ibeta;
  if (ser_b) {
    const double fb = db * qb;
    ibeta = qb * series_2A(fb * fb);
  } else {
    ibeta = (B.lnbeta - A.lnbeta) * qb;
  }
  const double v1m = A.hv1 + B.hv1, v2m = A.hv2 + B.hv2, v3m = A.hv3 + B.hv3;
  const double pm = A.hp + B.hp;
  const double vnA = dir == 0 ? A.v1 : dir == 1 ? A.v2 : A.v3;
  const double vnB = dir == 0 ? B.v1 : dir == 1 ? B.v2 : B.v3;
  const double vnm = dir == 0 ? v1m : dir == 1 ? v2m : v3m;
  const double frho = rho_ln * vnm;
  f[0] = frho;
  f[1] = fma(frho, v1m, dir == 0 ? pm : 0.0);
  f[2] = fma(frho, v2m, dir == 1 ? pm : 0.0);
  f[3] = fma(frho, v3m, dir == 2 ? pm : 0.0);
  const double kin = fma(A.hv1, B.v1, fma(A.hv2, B.v2, A.hv3 * B.v3));
  f[4] = fma(frho, fma(ibeta, inv_gm1, kin), fma(A.hp, vnB, B.hp * vnA));
}

// ---------------------------------------------------------------------------
// Surface fluxes in the face frame (rho, m_n, m_t1, m_t2, E), tangential axes t1 < t2.
struct FS3 {
  double rho, mn, mt1, mt2, E, ir, v, p, c;
};

__device__ __forceinline__ void face_state3(const double u[5], double ir, int d, const Ops3& o, FS3& s) {
  s.rho = u[0];
  s.ir = ir;
  s.mn = d == 0 ? u[1] : d == 1 ? u[2] : u[3];
  s.mt1 = d == 0 ? u[2] : u[1];
  s.mt2 = d == 2 ? u[2] : u[3];
  s.E = u[4];
  s.v = s.mn * ir;
  s.p = o.gm1 * fma(-0.5 * ir, fma(s.mn, s.mn, fma(s.mt1, s.mt1, s.mt2 * s.mt2)), s.E);
  s.c = sqrt(o.gamma * s.p * ir);
}

__device__ __forceinline__ void face_pair3(const double uL[5], const double uR[5], int d, const Ops3& o, FS3& L,
                                           FS3& R) {
  const double r2 = rcp_nr(uL[0] * uR[0]);
  face_state3(uL, uR[0] * r2, d, o, L);
  face_state3(uR, uL[0] * r2, d, o, R);
}

__device__ __forceinline__ void flux_rot3(const FS3& s, double F[5]) {
  F[0] = s.mn;
  F[1] = fma(s.mn, s.v, s.p);
  F[2] = s.mt1 * s.v;
  F[3] = s.mt2 * s.v;
  F[4] = (s.E + s.p) * s.v;
}

__device__ __forceinline__ void rotate_back3(const double F[5], int d, double f[5]) {
  f[0] = F[0];
  f[1] = d == 0 ? F[1] : F[2];
  f[2] = d == 1 ? F[1] : d == 0 ? F[2] : F[3];
  f[3] = d == 2 ? F[1] : F[3];
  f[4] = F[4];
}

__device__ __forceinline__ void hll_mid3(const FS3& L, const FS3& R, double SL, double SR, double F[5]) {
  if (SL >= 0.0) {
    flux_rot3(L, F);
  } else if (SR <= 0.0) {
    flux_rot3(R, F);
  } else {
    double FL[5], FR[5];
    flux_rot3(L, FL);
    flux_rot3(R, FR);
    const double inv = rcp_nr(SR - SL);
    const double SLSR = SL * SR;
    const double dU[5] = {R.rho - L.rho, R.mn - L.mn, R.mt1 - L.mt1, R.mt2 - L.mt2, R.E - L.E};
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] = fma(SLSR, dU[v], SR * FL[v] - SL * FR[v]) * inv;
  }
}

// HLL with Davis' speeds S_L = min(v_L - c_L, v_R - c_R), S_R = max(v_L + c_L, v_R + c_R)
__device__ void flux3_hll(const double uL[5], const double uR[5], int d, const Ops3& o, double f[5]) {
  FS3 L, R;
  face_pair3(uL, uR, d, o, L, R);
  double F[5];
  hll_mid3(L, R, fmin(L.v - L.c, R.v - R.c), fmax(L.v + L.c, R.v + R.c), F);
  rotate_back3(F, d, f);
}

// HLLE: Einfeldt's bounds from the Roe averages (weights sqrt(rho)) of the three velocity
// components and of the enthalpy, c~^2 = (gamma - 1)(H~ - |v~|^2 / 2)
__device__ void flux3_hlle(const double uL[5], const double uR[5], int d, const Ops3& o, double f[5]) {
  FS3 L, R;
  face_pair3(uL, uR, d, o, L, R);
  // Roe weights sqrt(rho_L) / (sqrt(rho_L) + sqrt(rho_R)) = 1 / (1 + q), q = sqrt(rho_R / rho_L)
  const double qw = sqrt(R.rho * L.ir);
  const double wl = rcp_nr(1.0 + qw), wr = qw * wl;
  const double vn = fma(wl, L.v, wr * R.v);
  const double vt1 = fma(wl, L.mt1 * L.ir, wr * (R.mt1 * R.ir));
  const double vt2 = fma(wl, L.mt2 * L.ir, wr * (R.mt2 * R.ir));
  const double H = fma(wl, (L.E + L.p) * L.ir, wr * ((R.E + R.p) * R.ir));
  const double c = sqrt(o.gm1 * fma(-0.5, fma(vn, vn, fma(vt1, vt1, vt2 * vt2)), H));
  double F[5];
  hll_mid3(L, R, fmin(L.v - L.c, vn - c), fmax(R.v + R.c, vn + c), F);
  rotate_back3(F, d, f);
}

// HLLC (Toro, Spruce, Speares 1994) with Davis' speeds and the standard contact speed
__device__ void flux3_hllc(const double uL[5], const double uR[5], int d, const Ops3& o, double f[5]) {
  FS3 L, R;
  face_pair3(uL, uR, d, o, L, R);
  const double SL = fmin(L.v - L.c, R.v - R.c), SR = fmax(L.v + L.c, R.v + R.c);
  double F[5];
  if (SL >= 0.0) {
    flux_rot3(L, F);
  } else if (SR <= 0.0) {
    flux_rot3(R, F);
  } else {
    const double mL = L.rho * (SL - L.v), mR = R.rho * (SR - R.v);
    const double Ss = (R.p - L.p + mL * L.v - mR * R.v) * rcp_nr(mL - mR);
    const bool left = Ss >= 0.0;
    const FS3& K = left ? L : R;
    const double S = left ? SL : SR;
    const double m = left ? mL : mR;
    flux_rot3(K, F);
    const double q = rcp_nr((S - Ss) * m);
    const double fac = m * m * q;                  // rho (S - v) / (S - S*)
    const double p_over_m = K.p * (S - Ss) * q;    // p / (rho (S - v))
    const double Us[5] = {fac, fac * Ss, fac * (K.mt1 * K.ir), fac * (K.mt2 * K.ir),
                          fac * fma(Ss - K.v, Ss + p_over_m, K.E * K.ir)};
    const double Uk[5] = {K.rho, K.mn, K.mt1, K.mt2, K.E};
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] = fma(S, Us[v] - Uk[v], F[v]);
  }
  rotate_back3(F, d, f);
}

__device__ __forceinline__ void surface_flux3(const double uL[5], const double uR[5], int d, const Ops3& o,
                                              const double* __restrict__ logt, double f[5]) {
  if (o.surface_flux == PERK_SURFACE_HLLE) {
    flux3_hlle(uL, uR, d, o, f);
  } else if (o.surface_flux == PERK_SURFACE_HLLC) {
    flux3_hllc(uL, uR, d, o, f);
  } else if (o.surface_flux == PERK_SURFACE_EC) {
    const NodeQ3 A = node_q3(uL, o.gm1, logt, logt + LOG_TABLE);
    const NodeQ3 B = node_q3(uR, o.gm1, logt, logt + LOG_TABLE);
    ec_flux_q3(A, B, d, o.inv_gm1, f);
  } else {
    flux3_hll(uL, uR, d, o, f);
  }
}

// ---------------------------------------------------------------------------
// Faces: blocks [0, if_blocks) take IFB interfaces each (one thread per face node); the rest
// take MB mortars each (one thread per node of each of the four small faces).
constexpr int F3_THREADS = 128;

template <int NN>
struct FaceCfg {
  static constexpr int FN = NN * NN;
  static constexpr int IFB = F3_THREADS / FN;         // 14 (N = 2) or 8 (N = 3)
  static constexpr int MB = F3_THREADS / (4 * FN);    // 3 (N = 2) or 2 (N = 3)
};

template <int NN, int YS>
__global__ void __launch_bounds__(F3_THREADS) k3_faces(Ops3 ops, int64_t n_if, const int4* __restrict__ ifs,
                                                        int64_t n_mort, const int4* __restrict__ morts,
                                                        const int4* __restrict__ msmall, int64_t if_blocks,
                                                        const int32_t* __restrict__ method, StageArgs sa,
                                                        const double* __restrict__ logt, double* __restrict__ surf) {
  constexpr int FN = G<NN>::FN;
  constexpr int SURF = G<NN>::SURF;
  constexpr int IFB = FaceCfg<NN>::IFB;
  constexpr int MB = FaceCfg<NN>::MB;
  __shared__ double s_ul[MB][5][FN];       // large-face trace
  __shared__ double s_f[MB][4][5][FN];     // small-face fluxes by quadrant
  if (blockIdx.x < if_blocks) {
    const int li = threadIdx.x / FN, q = threadIdx.x - li * FN;
    const int64_t idx = (int64_t)blockIdx.x * IFB + li;
    if (li >= IFB || idx >= n_if) return;
    const int4 r = ifs[idx];
    const int d = r.z;
    double uL[5], uR[5], f[5];
    stage_state3<NN, YS>(sa, r.x, r.w, face_node3<NN>(2 * d + 1, q), uL);
    stage_state3<NN, YS>(sa, r.y, r.w, face_node3<NN>(2 * d, q), uR);
    surface_flux3(uL, uR, d, ops, logt, f);
    double* sL = surf + (int64_t)r.x * SURF + (2 * d + 1) * 5 * FN + q;
    double* sR = surf + (int64_t)r.y * SURF + (2 * d) * 5 * FN + q;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      sL[v * FN] = f[v];
      sR[v * FN] = f[v];
    }
    return;
  }
  // mortars
  const int lm = threadIdx.x / (4 * FN);
  const int rem = threadIdx.x - lm * 4 * FN;
  const int quad = rem / FN, q = rem - quad * FN;
  const int64_t idx = (int64_t)(blockIdx.x - if_blocks) * MB + lm;
  const bool valid = lm < MB && idx < n_mort;
  int4 r = make_int4(0, 0, 0, 0);
  if (valid) r = morts[idx];
  const int d = r.w & 3, large_side = (r.w >> 2) & 1, m_fine = r.w >> MORT_FLAG_BITS;
  const int large_face = large_side == 0 ? 2 * d + 1 : 2 * d;
  const int small_face = large_side == 0 ? 2 * d : 2 * d + 1;
  const int t1 = q % NN, t2 = q / NN;
  const int q1 = quad & 1, q2 = quad >> 1;
  if (valid && quad == 0) {
    double ul[5];
    stage_state3<NN, YS>(sa, r.x, method[r.x], face_node3<NN>(large_face, q), ul);
#pragma unroll
    for (int v = 0; v < 5; ++v) s_ul[lm][v][q] = ul[v];
  }
  __syncthreads();
  if (valid) {
    // the large trace at this small node: sum_l2 P_q2[t2][l2] sum_l1 P_q1[t1][l1] u_L(l1, l2)
    // (operator entries by value selects: no pointer into the kernel's parameter space)
    double w1[NN];
#pragma unroll
    for (int l1 = 0; l1 < NN; ++l1) w1[l1] = q1 ? ops.p_hi[t1][l1] : ops.p_lo[t1][l1];
    double ui[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int l2 = 0; l2 < NN; ++l2) {
      const double w2 = q2 ? ops.p_hi[t2][l2] : ops.p_lo[t2][l2];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        double row = 0.0;
#pragma unroll
        for (int l1 = 0; l1 < NN; ++l1) row = fma(w1[l1], s_ul[lm][v][l2 * NN + l1], row);
        ui[v] = fma(w2, row, ui[v]);
      }
    }
    const int4 sm = msmall[r.z];
    const int small = quad == 0 ? sm.x : quad == 1 ? sm.y : quad == 2 ? sm.z : sm.w;
    double us[5], f[5];
    stage_state3<NN, YS>(sa, small, m_fine, face_node3<NN>(small_face, q), us);
    if (large_side == 0)
      surface_flux3(ui, us, d, ops, logt, f);
    else
      surface_flux3(us, ui, d, ops, logt, f);
    double* s = surf + (int64_t)small * SURF + small_face * 5 * FN + q;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      s[v * FN] = f[v];
      s_f[lm][quad][v][q] = f[v];
    }
  }
  __syncthreads();
  if (valid) {
    // large-face flux at node (t1, t2): sum over quadrants of the tensor-product projection;
    // this thread produces variable `quad`, and variable 4 when quad == 0
    for (int vv = 0; vv < (quad == 0 ? 2 : 1); ++vv) {
      const int v = vv ? 4 : quad;
      double acc = 0.0;
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) {
#pragma unroll
        for (int l2 = 0; l2 < NN; ++l2) {
          double row = 0.0;
#pragma unroll
          for (int l1 = 0; l1 < NN; ++l1)
            row = fma((qq & 1) ? ops.r_hi[t1][l1] : ops.r_lo[t1][l1], s_f[lm][qq][v][l2 * NN + l1], row);
          acc = fma((qq >> 1) ? ops.r_hi[t2][l2] : ops.r_lo[t2][l2], row, acc);
        }
      }
      surf[(int64_t)r.x * SURF + large_face * 5 * FN + v * FN + q] = acc;
    }
  }
}

// ---------------------------------------------------------------------------
// Volume: one thread per node, VE elements per 128-thread block.
constexpr int V3_THREADS = 128;

template <int NN>
struct VolCfg {
  static constexpr int VE = V3_THREADS / G<NN>::NODES;   // 4 (N = 2) or 2 (N = 3)
};

template <int NN>
__device__ __forceinline__ int pslot3(int a, int b) {   // a < b
  return a * (2 * NN - a - 1) / 2 + (b - a - 1);
}

template <int NN, int YS, bool CHECK>
__global__ void __launch_bounds__(V3_THREADS, 6) k3_volume(Ops3 ops, int64_t n, const int32_t* __restrict__ elems,
                                                         const int32_t* __restrict__ level,
                                                         const int32_t* __restrict__ method, double two_over_len,
                                                         StageArgs sa, const double* __restrict__ surf,
                                                         double* __restrict__ K, UpdateArgs ua,
                                                         const double* __restrict__ logt) {
  constexpr int FN = G<NN>::FN, NODES = G<NN>::NODES, ELEM = G<NN>::ELEM, SURF = G<NN>::SURF;
  constexpr int NPL = G<NN>::NPL, NP = G<NN>::NP;
  constexpr int VE = VolCfg<NN>::VE;
  __shared__ NodeQ3 s_q[VE][NODES];
  __shared__ double s_flux[VE][5][NP];
  __shared__ double s_log[2 * LOG_TABLE];
  __shared__ unsigned long long s_ext[VE][4];   // bit-pattern extremes: min rho, max rho, min rho/p, max rho/p
  const int t = threadIdx.x;
  const int le = t / NODES, node = t - le * NODES;
  const bool inblk = le < VE;
  const int64_t slot = (int64_t)blockIdx.x * VE + le;
  const bool valid = inblk && slot < n;
  const int64_t e = valid ? elems[slot] : 0;
  const int m = valid ? method[e] : 0;
  const int i = node % NN, j = (node / NN) % NN, k = node / FN;

  // global loads first: the stage state and the fluxes of the faces through this node
  double y[5];
  if (valid) {
    stage_state3<NN, YS>(sa, e, m, node, y);
  } else {
    y[0] = 1.0; y[1] = 0.0; y[2] = 0.0; y[3] = 0.0; y[4] = 2.5;
  }
  double fx[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, fy[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, fz[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (valid) {
    const double* sf = surf + e * SURF;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      if (i == 0) fx[v] = __ldg(sf + 0 * 5 * FN + v * FN + k * NN + j);
      if (i == NN - 1) fx[v] = __ldg(sf + 1 * 5 * FN + v * FN + k * NN + j);
      if (j == 0) fy[v] = __ldg(sf + 2 * 5 * FN + v * FN + k * NN + i);
      if (j == NN - 1) fy[v] = __ldg(sf + 3 * 5 * FN + v * FN + k * NN + i);
      if (k == 0) fz[v] = __ldg(sf + 4 * 5 * FN + v * FN + j * NN + i);
      if (k == NN - 1) fz[v] = __ldg(sf + 5 * 5 * FN + v * FN + j * NN + i);
    }
  }
  for (int q = t; q < 2 * LOG_TABLE; q += V3_THREADS) s_log[q] = logt[q];
  if (t < 4 * VE) s_ext[t >> 2][t & 3] = (t & 1) ? 0ull : ~0ull;
  __syncthreads();
  // node logarithms only in elements where some pair leaves the series range of the means
  NodeQ3 q = node_q3_nolog(y, ops.gm1);
  if (inblk) {
    atomicMin(&s_ext[le][0], dbits(q.rho));
    atomicMax(&s_ext[le][1], dbits(q.rho));
    atomicMin(&s_ext[le][2], dbits(q.beta));
    atomicMax(&s_ext[le][3], dbits(q.beta));
  }
  __syncthreads();
  if (inblk) {
    if (!series_only(s_ext[le][0], s_ext[le][1], s_ext[le][2], s_ext[le][3])) {
      q.lnrho = log_tab(q.rho, s_log, s_log + LOG_TABLE);
      q.lnbeta = log_tab(q.beta, s_log, s_log + LOG_TABLE);
    }
    s_q[le][node] = q;
  }
  __syncthreads();

  // the symmetric pairs of the block's elements: pair pp = (dir, line, slot)
  for (int p = t; p < VE * NP; p += V3_THREADS) {
    const int lp = p / NP, pp = p - lp * NP;
    const int dir = pp / (FN * NPL);
    const int rem = pp - dir * FN * NPL;
    const int line = rem / NPL;
    int s = rem - line * NPL, a = 0;
#pragma unroll
    for (int aa = 0; aa < NN - 1; ++aa) {
      const int len = NN - 1 - a;
      if (s >= len) {
        s -= len;
        ++a;
      }
    }
    const int b = a + 1 + s;
    int na, nb;
    if (dir == 0) {          // line = k NN + j
      na = line * NN + a;
      nb = line * NN + b;
    } else if (dir == 1) {   // line = k NN + i
      const int kk = line / NN, ii = line - kk * NN;
      na = (kk * NN + a) * NN + ii;
      nb = (kk * NN + b) * NN + ii;
    } else {                 // line = j NN + i
      na = a * FN + line;
      nb = b * FN + line;
    }
    double f[5];
    ec_flux_q3(s_q[lp][na], s_q[lp][nb], dir, ops.inv_gm1, f);
#pragma unroll
    for (int v = 0; v < 5; ++v) s_flux[lp][v][pp] = f[v];
  }
  __syncthreads();
  if (!valid) return;

  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int mm = 0; mm < NN; ++mm) {
    if (mm != i) {
      const double w = ops.dsplit[i][mm];
      const int p = (k * NN + j) * NPL + pslot3<NN>(min(i, mm), max(i, mm));
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v] = fma(w, s_flux[le][v][p], acc[v]);
    }
    if (mm != j) {
      const double w = ops.dsplit[j][mm];
      const int p = FN * NPL + (k * NN + i) * NPL + pslot3<NN>(min(j, mm), max(j, mm));
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v] = fma(w, s_flux[le][v][p], acc[v]);
    }
    if (mm != k) {
      const double w = ops.dsplit[k][mm];
      const int p = 2 * FN * NPL + (j * NN + i) * NPL + pslot3<NN>(min(k, mm), max(k, mm));
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v] = fma(w, s_flux[le][v][p], acc[v]);
    }
  }
  // surface lifting on the six faces (w_0 = w_N)
  const double iw = ops.inv_w0;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    if (i == 0) acc[v] = fma(-iw, fx[v], acc[v]);
    if (i == NN - 1) acc[v] = fma(iw, fx[v], acc[v]);
    if (j == 0) acc[v] = fma(-iw, fy[v], acc[v]);
    if (j == NN - 1) acc[v] = fma(iw, fy[v], acc[v]);
    if (k == 0) acc[v] = fma(-iw, fz[v], acc[v]);
    if (k == NN - 1) acc[v] = fma(iw, fz[v], acc[v]);
  }
  const double scale = -ldexp(two_over_len, level[e]);   // -(2/h)
  double kv[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    kv[v] = scale * acc[v];
    K[e * ELEM + v * NODES + node] = kv[v];
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

// ---------------------------------------------------------------------------
__global__ void k3_commit(int64_t nd, UpdateArgs ua, const double* __restrict__ Ks, const double* dtp,
                          double* __restrict__ U) {
  if (*ua.flag != 0) return;
  const double dt = dtp[0];
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nd; q += (int64_t)gridDim.x * blockDim.x) {
    double inc = ua.bs * Ks[q];
    if (ua.b1 != 0.0) inc = fma(ua.b1, ua.K1[q], inc);
    if (ua.bp != 0.0) inc = fma(ua.bp, ua.Kp[q], inc);
    U[q] = fma(dt, inc, U[q]);
  }
}

constexpr int DT3_THREADS = 256;

// min over nodes of h_e / ((N+1) lambda), lambda = |v1| + |v2| + |v3| + 3c; positive doubles order
// like their bit patterns, so the block minimum goes to *out by an integer atomicMin.  A node
// without an admissible state (rho <= 0, p <= 0, NaN or Inf) contributes the pattern 0 (+0.0),
// which the host reports as such.
template <int NN>
__global__ void __launch_bounds__(DT3_THREADS) k3_dt(int64_t n_nodes, const double* __restrict__ U,
                                                      const int32_t* __restrict__ level, double length,
                                                      double gamma, unsigned long long* out) {
  constexpr int NODES = G<NN>::NODES, ELEM = G<NN>::ELEM;
  __shared__ double s_min[DT3_THREADS / 32];
  double best = INFINITY;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_nodes; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = q / NODES;
    const int node = (int)(q - e * NODES);
    const double* u = U + e * ELEM + node;
    const double rho = u[0], ir = 1.0 / rho;
    const double v1 = u[NODES] * ir, v2 = u[2 * NODES] * ir, v3 = u[3 * NODES] * ir;
    const double p = (gamma - 1.0) * (u[4 * NODES] - 0.5 * rho * (v1 * v1 + v2 * v2 + v3 * v3));
    const double lam = fabs(v1) + fabs(v2) + fabs(v3) + 3.0 * sqrt(gamma * p * ir);
    const double h = ldexp(length, -level[e]);
    const double r = h / (NN * lam);
    best = (rho > 0.0 && p > 0.0 && r > 0.0 && r < INFINITY) ? fmin(best, r) : 0.0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) s_min[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = s_min[0];
    for (int w = 1; w < DT3_THREADS / 32; ++w) b = fmin(b, s_min[w]);
    if (b < INFINITY) atomicMin(out, (unsigned long long)__double_as_longlong(b));
  }
}

__global__ void k3_set(double* p, double v) { *p = v; }

// ---------------------------------------------------------------------------
// AMR: enstrophy indicator and solution transfer.

// eta[e] = max over the element's nodes of rho |curl v|^2 / 2; one thread per node, VE elements
// per 128-thread block; derivatives (2/h) D along each axis from the velocities in shared memory
template <int NN>
__global__ void __launch_bounds__(V3_THREADS) k3_enstrophy(Ops3 ops, int64_t n, const double* __restrict__ U,
                                                            const int32_t* __restrict__ level, double two_over_len,
                                                            double* __restrict__ eta) {
  constexpr int FN = G<NN>::FN, NODES = G<NN>::NODES, ELEM = G<NN>::ELEM;
  constexpr int VE = VolCfg<NN>::VE;
  __shared__ double s_v[VE][3][NODES];
  __shared__ unsigned long long s_max[VE];
  const int t = threadIdx.x;
  const int le = t / NODES, node = t - le * NODES;
  const int64_t e = (int64_t)blockIdx.x * VE + le;
  const bool valid = le < VE && e < n;
  const int i = node % NN, j = (node / NN) % NN, k = node / FN;
  double rho = 1.0;
  if (valid) {
    const double* u = U + e * ELEM + node;
    rho = u[0];
    const double ir = 1.0 / rho;
#pragma unroll
    for (int d = 0; d < 3; ++d) s_v[le][d][node] = u[(1 + d) * NODES] * ir;
  }
  if (t < VE) s_max[t] = 0ull;
  __syncthreads();
  if (valid) {
    // g[d][a] = d v_d / d x_a in reference units
    double g[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double gx = 0.0, gy = 0.0, gz = 0.0;
#pragma unroll
      for (int m = 0; m < NN; ++m) {
        gx = fma(ops.dmat[i][m], s_v[le][d][(k * NN + j) * NN + m], gx);
        gy = fma(ops.dmat[j][m], s_v[le][d][(k * NN + m) * NN + i], gy);
        gz = fma(ops.dmat[k][m], s_v[le][d][(m * NN + j) * NN + i], gz);
      }
      g[d][0] = gx;
      g[d][1] = gy;
      g[d][2] = gz;
    }
    const double s = ldexp(two_over_len, level[e]);   // 2 / h
    const double wx = s * (g[2][1] - g[1][2]);
    const double wy = s * (g[0][2] - g[2][0]);
    const double wz = s * (g[1][0] - g[0][1]);
    const double ens = 0.5 * rho * (wx * wx + wy * wy + wz * wz);
    // non-negative doubles order like their bit patterns (a NaN sorts above every number)
    atomicMax(&s_max[le], (unsigned long long)__double_as_longlong(ens));
  }
  __syncthreads();
  if (valid && node == 0) eta[e] = __longlong_as_double((long long)s_max[le]);
}

// One thread per node of a new element: copy, interpolation of the parent polynomial to a child
// (the 1D half-interval interpolation matrices along each axis), or the L2 projection of the eight
// children onto the parent (the 1D half-interval projections along each axis, summed).
template <int NN>
__global__ void __launch_bounds__(V3_THREADS) k3_transfer(Ops3 ops, int64_t n, const int32_t* __restrict__ map,
                                                           const double* __restrict__ Uold, double* __restrict__ Unew) {
  constexpr int FN = G<NN>::FN, NODES = G<NN>::NODES, ELEM = G<NN>::ELEM;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * NODES) return;
  const int64_t e = q / NODES;
  const int node = (int)(q - e * NODES);
  const int i = node % NN, j = (node / NN) % NN, k = node / FN;
  const int32_t* r = map + 9 * e;
  const int kind = r[0] & 3;
  double* out = Unew + e * ELEM + node;
  if (kind == 0) {
    const double* src = Uold + (int64_t)r[1] * ELEM + node;
#pragma unroll
    for (int v = 0; v < 5; ++v) out[v * NODES] = src[v * NODES];
    return;
  }
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const int nsrc = kind == 1 ? 1 : 8;
  for (int c = 0; c < nsrc; ++c) {
    // kind 1: the child position (cx, cy, cz) of this cell in its parent; kind 2: child c
    const int cx = kind == 1 ? (r[0] >> 2) & 1 : c & 1;
    const int cy = kind == 1 ? (r[0] >> 3) & 1 : (c >> 1) & 1;
    const int cz = kind == 1 ? (r[0] >> 4) & 1 : (c >> 2) & 1;
    const double* src = Uold + (int64_t)r[1 + c] * ELEM;
    double wx[NN], wy[NN], wz[NN];
#pragma unroll
    for (int m = 0; m < NN; ++m) {
      if (kind == 1) {
        wx[m] = cx ? ops.p_hi[i][m] : ops.p_lo[i][m];
        wy[m] = cy ? ops.p_hi[j][m] : ops.p_lo[j][m];
        wz[m] = cz ? ops.p_hi[k][m] : ops.p_lo[k][m];
      } else {
        wx[m] = cx ? ops.r_hi[i][m] : ops.r_lo[i][m];
        wy[m] = cy ? ops.r_hi[j][m] : ops.r_lo[j][m];
        wz[m] = cz ? ops.r_hi[k][m] : ops.r_lo[k][m];
      }
    }
#pragma unroll
    for (int c3 = 0; c3 < NN; ++c3)
#pragma unroll
      for (int b = 0; b < NN; ++b) {
        const double wzy = wz[c3] * wy[b];
#pragma unroll
        for (int a = 0; a < NN; ++a) {
          const double w = wzy * wx[a];
          const int m = (c3 * NN + b) * NN + a;
#pragma unroll
          for (int v = 0; v < 5; ++v) acc[v] = fma(w, __ldg(src + v * NODES + m), acc[v]);
        }
      }
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) out[v * NODES] = acc[v];
}

// ---------------------------------------------------------------------------
template <int NN>
static cudaError_t faces3(cudaStream_t st, YSource ys, const Ops3& ops, int64_t n_if, const int4* ifs, int64_t n_mort,
                          const int4* morts, const int4* msmall, const int32_t* method, const StageArgs& sa,
                          const double* logt, double* surf) {
  const int64_t ifb = (n_if + FaceCfg<NN>::IFB - 1) / FaceCfg<NN>::IFB;
  const int64_t mb = (n_mort + FaceCfg<NN>::MB - 1) / FaceCfg<NN>::MB;
  if (ifb + mb == 0) return cudaSuccess;
  const dim3 grid((unsigned)(ifb + mb));
  if (ys == Y_GIVEN)
    k3_faces<NN, Y_GIVEN><<<grid, F3_THREADS, 0, st>>>(ops, n_if, ifs, n_mort, morts, msmall, ifb, method, sa, logt,
                                                        surf);
  else
    k3_faces<NN, Y_COMBINE><<<grid, F3_THREADS, 0, st>>>(ops, n_if, ifs, n_mort, morts, msmall, ifb, method, sa,
                                                          logt, surf);
  return cudaGetLastError();
}

cudaError_t launch_faces3(cudaStream_t st, YSource ys, const Ops3& ops, int64_t n_if, const int4* ifs, int64_t n_mort,
                          const int4* morts, const int4* msmall, const int32_t* method, const StageArgs& sa,
                          const double* log_table, double* surf) {
  if (ops.nn == 3) return faces3<3>(st, ys, ops, n_if, ifs, n_mort, morts, msmall, method, sa, log_table, surf);
  if (ops.nn == 4) return faces3<4>(st, ys, ops, n_if, ifs, n_mort, morts, msmall, method, sa, log_table, surf);
  return cudaErrorInvalidValue;
}

template <int NN>
static cudaError_t volume3(cudaStream_t st, YSource ys, const Ops3& ops, int64_t n, const int32_t* elems,
                           const int32_t* level, const int32_t* method, double two_over_len, const StageArgs& sa,
                           const double* surf, double* K, const UpdateArgs* check, const double* logt) {
  if (n <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((n + VolCfg<NN>::VE - 1) / VolCfg<NN>::VE));
  const UpdateArgs ua = check ? *check : UpdateArgs{};
  if (ys == Y_GIVEN) {
    if (check)
      k3_volume<NN, Y_GIVEN, true><<<grid, V3_THREADS, 0, st>>>(ops, n, elems, level, method, two_over_len, sa, surf,
                                                                 K, ua, logt);
    else
      k3_volume<NN, Y_GIVEN, false><<<grid, V3_THREADS, 0, st>>>(ops, n, elems, level, method, two_over_len, sa,
                                                                  surf, K, ua, logt);
  } else {
    if (check)
      k3_volume<NN, Y_COMBINE, true><<<grid, V3_THREADS, 0, st>>>(ops, n, elems, level, method, two_over_len, sa,
                                                                   surf, K, ua, logt);
    else
      k3_volume<NN, Y_COMBINE, false><<<grid, V3_THREADS, 0, st>>>(ops, n, elems, level, method, two_over_len, sa,
                                                                    surf, K, ua, logt);
  }
  return cudaGetLastError();
}

cudaError_t launch_volume3(cudaStream_t st, YSource ys, const Ops3& ops, int64_t n, const int32_t* elems,
                           const int32_t* level, const int32_t* method, double two_over_len, const StageArgs& sa,
                           const double* surf, double* K, const UpdateArgs* check, const double* log_table) {
  if (ops.nn == 3)
    return volume3<3>(st, ys, ops, n, elems, level, method, two_over_len, sa, surf, K, check, log_table);
  if (ops.nn == 4)
    return volume3<4>(st, ys, ops, n, elems, level, method, two_over_len, sa, surf, K, check, log_table);
  return cudaErrorInvalidValue;
}

cudaError_t launch_commit3(cudaStream_t st, int64_t n_doubles, const UpdateArgs& ua, const double* Ks,
                           const double* dt, double* U) {
  if (n_doubles <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((n_doubles + 255) / 256, (int64_t)perk::device_sm_count() * 16);
  k3_commit<<<(unsigned)blocks, 256, 0, st>>>(n_doubles, ua, Ks, dt, U);
  return cudaGetLastError();
}

cudaError_t launch_enstrophy3(cudaStream_t st, const Ops3& ops, int64_t n_elem, const double* U,
                              const int32_t* level, double two_over_len, double* eta) {
  if (n_elem <= 0) return cudaSuccess;
  if (ops.nn == 3)
    k3_enstrophy<3><<<(unsigned)((n_elem + VolCfg<3>::VE - 1) / VolCfg<3>::VE), V3_THREADS, 0, st>>>(
        ops, n_elem, U, level, two_over_len, eta);
  else if (ops.nn == 4)
    k3_enstrophy<4><<<(unsigned)((n_elem + VolCfg<4>::VE - 1) / VolCfg<4>::VE), V3_THREADS, 0, st>>>(
        ops, n_elem, U, level, two_over_len, eta);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_transfer3(cudaStream_t st, const Ops3& ops, int64_t n_new, const int32_t* map, const double* Uold,
                             double* Unew) {
  if (n_new <= 0) return cudaSuccess;
  const int64_t threads = n_new * nodes3(ops.nn);
  const unsigned blocks = (unsigned)((threads + V3_THREADS - 1) / V3_THREADS);
  if (ops.nn == 3)
    k3_transfer<3><<<blocks, V3_THREADS, 0, st>>>(ops, n_new, map, Uold, Unew);
  else if (ops.nn == 4)
    k3_transfer<4><<<blocks, V3_THREADS, 0, st>>>(ops, n_new, map, Uold, Unew);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_dt3(cudaStream_t st, int nn, int64_t n_elem, const double* U, const int32_t* level, double length,
                       double gamma, double* out) {
  k3_set<<<1, 1, 0, st>>>(out, INFINITY);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || n_elem <= 0) return e;
  const int64_t n_nodes = n_elem * nodes3(nn);
  const unsigned blocks = (unsigned)std::min<int64_t>((n_nodes + DT3_THREADS - 1) / DT3_THREADS, (int64_t)perk::device_sm_count() * 8);
  unsigned long long* o = reinterpret_cast<unsigned long long*>(out);
  if (nn == 3)
    k3_dt<3><<<blocks, DT3_THREADS, 0, st>>>(n_nodes, U, level, length, gamma, o);
  else if (nn == 4)
    k3_dt<4><<<blocks, DT3_THREADS, 0, st>>>(n_nodes, U, level, length, gamma, o);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace perk3
