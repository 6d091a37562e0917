// sm_103a kernels of the P-ERK / DGSEM hot path.
//
// One P-ERK stage (Eq. PartitionedRKSystem; Sec. 3.1) works on the active
// prefixes of the level-sorted lists:
//   k_faces   numerical fluxes of the active interfaces and mortars (Sec. 6.2),
//             stage states formed on the fly at the face nodes;
//   k_volume  flux-differencing volume integral + surface lifting + Jacobian
//             of the active elements, stage state formed on the fly;
//   k_stage   both in one launch (Euler, plain volume term): face items first,
//             volume items waiting per element for their four faces.
// The step ends with k_commit (guarded final update).  k_partition rebuilds
// the level partition; k_dt_* reduce the CFL step size (Eq. CFL_DG).
//
// All arithmetic is FP64.  The FP64 pipe of GB300 is the binding resource of
// the volume kernel, so it evaluates every symmetric node pair once (48 pairs
// per element instead of 96 one-sided evaluations), takes the logarithms of
// density and rho/p once per node (table-driven), and forms both logarithmic
// means of a pair from one Newton-Raphson reciprocal.

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>

#include "perk.h"
#include "perk_internal.h"
#include "perk_devmath.cuh"

namespace perk {

// ---------------------------------------------------------------------------
// Logarithmic mean from per-node logarithms (used by the EC surface flux; the
// volume kernel uses the cheaper forms further below).
//
// With d = b - a, s = a + b, f = d/s and u = f^2:  ln(b/a) = 2 artanh(f)
// = 2 f A(u), A(u) = sum_k u^k / (2k+1).  Hence
//   {{x}}_ln = d / ln(b/a) = (s/2) G(u),  G = 1/A,
//   1/{{x}}_ln = (2/s) A(u).
// For u < 1e-2 the truncated series (k <= 7; remainder < 6e-18 relative) is
// used; otherwise the quotient of the difference and the difference of the
// precomputed logarithms, whose relative error there is below ~1e-15 |ln x|.
// G's coefficients follow from A G = 1 term by term (exact rationals).
__device__ __forceinline__ double series_A(double u) {
  double r = 1.0 / 15.0;
  r = fma(r, u, 1.0 / 13.0);
  r = fma(r, u, 1.0 / 11.0);
  r = fma(r, u, 1.0 / 9.0);
  r = fma(r, u, 1.0 / 7.0);
  r = fma(r, u, 1.0 / 5.0);
  r = fma(r, u, 1.0 / 3.0);
  return fma(r, u, 1.0);
}
__device__ __forceinline__ double series_G(double u) {
  double r = -25865068.0 / 1915538625.0;
  r = fma(r, u, -10719068.0 / 638512875.0);
  r = fma(r, u, -10196.0 / 467775.0);
  r = fma(r, u, -428.0 / 14175.0);
  r = fma(r, u, -44.0 / 945.0);
  r = fma(r, u, -4.0 / 45.0);
  r = fma(r, u, -1.0 / 3.0);
  return fma(r, u, 1.0);
}
__device__ __forceinline__ double ln_mean(double a, double b, double lna, double lnb) {
  const double d = b - a, s = a + b;
  if (d * d < 1e-2 * (s * s)) {
    const double is = 1.0 / s;
    const double f = d * is;
    return 0.5 * s * series_G(f * f);
  }
  return d / (lnb - lna);
}
__device__ __forceinline__ double inv_ln_mean(double a, double b, double lna, double lnb) {
  const double d = b - a, s = a + b;
  if (d * d < 1e-2 * (s * s)) {
    const double is = 1.0 / s;
    const double f = d * is;
    return 2.0 * is * series_A(f * f);
  }
  return (lnb - lna) / d;
}

// ---------------------------------------------------------------------------
// FP64 building blocks of the volume kernel (rcp_nr, log_tab, series_H,
// series_2A) live in perk_devmath.cuh, shared with the 3D kernels.

// Node quantities of the two-point flux (half values fold the 1/2 of the means),
// padded to 80 bytes so that shared-memory reads can use 16-byte loads.
struct __align__(16) NodeQ {
  double rho, lnrho, beta, lnbeta, v1, v2, hv1, hv2, hp, pad;
};

// node quantities without the two logarithms (set to 0; see series_only)
__device__ __forceinline__ NodeQ node_q_nolog(const double u[4], double gm1) {
  NodeQ q;
  // rho p = (gamma - 1) (rho E - |m|^2 / 2) needs no division; one reciprocal gives 1/rho and 1/p
  const double rp = gm1 * fma(u[0], u[3], -0.5 * fma(u[1], u[1], u[2] * u[2]));
  const double r = rcp_nr(u[0] * rp);        // 1 / (rho^2 p)
  const double ir = rp * r;                  // 1 / rho
  q.rho = u[0];
  q.v1 = u[1] * ir;
  q.v2 = u[2] * ir;
  q.hp = 0.5 * (rp * ir);                    // p / 2
  q.beta = (u[0] * u[0]) * (u[0] * r);       // rho / p
  q.hv1 = 0.5 * q.v1;
  q.hv2 = 0.5 * q.v2;
  q.lnrho = 0.0;
  q.lnbeta = 0.0;
  q.pad = 0.0;
  return q;
}

__device__ __forceinline__ NodeQ node_q(const double u[4], double gm1, const double* inv_c, const double* ln_c) {
  NodeQ q = node_q_nolog(u, gm1);
  q.lnrho = log_tab(q.rho, inv_c, ln_c);
  q.lnbeta = log_tab(q.beta, inv_c, ln_c);
  return q;
}

// Ranocha's two-point flux from NodeQ: one reciprocal serves both logarithmic means.
__device__ __forceinline__ void ec_flux_q(const NodeQ& A, const NodeQ& B, int dir, double inv_gm1, double f[4]) {
  const double dr = B.rho - A.rho, sr = A.rho + B.rho;
  const double db = B.beta - A.beta, sb = A.beta + B.beta;
  const bool ser_r = near_pair(A.rho, B.rho);
  const bool ser_b = near_pair(A.beta, B.beta);
  const double den_r = ser_r ? sr : B.lnrho - A.lnrho;
  const double den_b = ser_b ? sb : db;
  const double r = rcp_nr(den_r * den_b);
  const double qr = den_b * r;               // 1 / den_r
  const double qb = den_r * r;               // 1 / den_b
  const double fr = dr * qr;
  double rho_ln, ibeta;
  if (ser_r)
    rho_ln = sr * series_H(fr * fr);
  else
    rho_ln = fr;
  if (ser_b) {
    const double fb = db * qb;
    ibeta = qb * series_2A(fb * fb);
  } else {
    ibeta = (B.lnbeta - A.lnbeta) * qb;
  }
  const double v1m = A.hv1 + B.hv1;
  const double v2m = A.hv2 + B.hv2;
  const double pm = A.hp + B.hp;
  const double vnA = dir ? A.v2 : A.v1;
  const double vnB = dir ? B.v2 : B.v1;
  const double frho = rho_ln * (dir ? v2m : v1m);
  f[0] = frho;
  f[1] = fma(frho, v1m, dir ? 0.0 : pm);
  f[2] = fma(frho, v2m, dir ? pm : 0.0);
  const double kin = fma(A.hv1, B.v1, A.hv2 * B.v2);
  f[3] = fma(frho, fma(ibeta, inv_gm1, kin), fma(A.hp, vnB, B.hp * vnA));
}

// Ranocha's entropy-conservative, kinetic-energy-preserving two-point flux in
// direction dir (0 = x, 1 = y), from node primitives and their logarithms.
struct Prim {
  double rho, v1, v2, p, lnrho, beta, lnbeta;  // beta = rho / p
};

__device__ __forceinline__ void ec_flux(const Prim& A, const Prim& B, int dir, double inv_gm1, double f[4]) {
  const double rho_ln = ln_mean(A.rho, B.rho, A.lnrho, B.lnrho);
  const double ibeta_ln = inv_ln_mean(A.beta, B.beta, A.lnbeta, B.lnbeta);
  const double v1m = 0.5 * (A.v1 + B.v1);
  const double v2m = 0.5 * (A.v2 + B.v2);
  const double pm = 0.5 * (A.p + B.p);
  const double vnA = dir ? A.v2 : A.v1;
  const double vnB = dir ? B.v2 : B.v1;
  const double frho = rho_ln * (dir ? v2m : v1m);
  f[0] = frho;
  f[1] = fma(frho, v1m, dir ? 0.0 : pm);
  f[2] = fma(frho, v2m, dir ? pm : 0.0);
  const double kin = 0.5 * fma(A.v1, B.v1, A.v2 * B.v2);
  f[3] = fma(frho, fma(ibeta_ln, inv_gm1, kin), 0.5 * fma(A.p, vnB, B.p * vnA));
}

__device__ __forceinline__ Prim prim_from_cons(const double u[4], double gm1) {
  Prim P;
  const double ir = 1.0 / u[0];
  P.rho = u[0];
  P.v1 = u[1] * ir;
  P.v2 = u[2] * ir;
  P.p = gm1 * (u[3] - 0.5 * (u[1] * P.v1 + u[2] * P.v2));
  P.beta = u[0] / P.p;
  P.lnrho = log(P.rho);
  P.lnbeta = log(P.beta);
  return P;
}

// ---------------------------------------------------------------------------
// Surface fluxes f*(uL, uR) in direction dir.
__device__ __forceinline__ void phys_flux(const double u[4], double vn, double p, int dir, double f[4]) {
  f[0] = u[0] * vn;
  f[1] = fma(u[1], vn, dir ? 0.0 : p);
  f[2] = fma(u[2], vn, dir ? p : 0.0);
  f[3] = (u[3] + p) * vn;
}

// Surface fluxes in the face's frame: the state is rotated to (rho, m_n, m_t, E)
// with selects (no dynamically indexed arrays), the flux computed there and
// rotated back.  Reciprocals are Newton-Raphson ones; one reciprocal of
// rho_L rho_R gives both 1/rho.
struct FaceState {
  double rho, mn, mt, E, ir, v, p, c;
};

__device__ __forceinline__ void face_pair(const double uL[4], const double uR[4], int dir, const Ops& ops,
                                          FaceState& L, FaceState& R) {
  const double r2 = rcp_nr(uL[0] * uR[0]);
  L.rho = uL[0];
  R.rho = uR[0];
  L.ir = uR[0] * r2;
  R.ir = uL[0] * r2;
  L.mn = dir ? uL[2] : uL[1];
  L.mt = dir ? uL[1] : uL[2];
  R.mn = dir ? uR[2] : uR[1];
  R.mt = dir ? uR[1] : uR[2];
  L.E = uL[3];
  R.E = uR[3];
  L.v = L.mn * L.ir;
  R.v = R.mn * R.ir;
  L.p = ops.gm1 * fma(-0.5 * L.ir, fma(L.mn, L.mn, L.mt * L.mt), L.E);
  R.p = ops.gm1 * fma(-0.5 * R.ir, fma(R.mn, R.mn, R.mt * R.mt), R.E);
  L.c = sqrt(ops.gamma * L.p * L.ir);
  R.c = sqrt(ops.gamma * R.p * R.ir);
}

__device__ __forceinline__ void face_flux_rot(const FaceState& s, double F[4]) {
  F[0] = s.mn;
  F[1] = fma(s.mn, s.v, s.p);
  F[2] = s.mt * s.v;
  F[3] = (s.E + s.p) * s.v;
}

__device__ __forceinline__ void rotate_back(const double F[4], int dir, double f[4]) {
  f[0] = F[0];
  f[1] = dir ? F[2] : F[1];
  f[2] = dir ? F[1] : F[2];
  f[3] = F[3];
}

// HLL with Davis wave-speed estimates S_L = min(vL - cL, vR - cR), S_R = max(vL + cL, vR + cR).
__device__ void flux_hll(const double uL[4], const double uR[4], int dir, const Ops& ops, double f[4]) {
  FaceState L, R;
  face_pair(uL, uR, dir, ops, L, R);
  const double SL = fmin(L.v - L.c, R.v - R.c), SR = fmax(L.v + L.c, R.v + R.c);
  double F[4];
  if (SL >= 0.0) {
    face_flux_rot(L, F);
  } else if (SR <= 0.0) {
    face_flux_rot(R, F);
  } else {
    double FL[4], FR[4];
    face_flux_rot(L, FL);
    face_flux_rot(R, FR);
    const double inv = rcp_nr(SR - SL);
    const double SLSR = SL * SR;
    const double dU[4] = {R.rho - L.rho, R.mn - L.mn, R.mt - L.mt, R.E - L.E};
#pragma unroll
    for (int v = 0; v < 4; ++v) F[v] = fma(SLSR, dU[v], SR * FL[v] - SL * FR[v]) * inv;
  }
  rotate_back(F, dir, f);
}

// HLLE: the HLL flux with Einfeldt's bounds S_L = min(v_L - c_L, v~ - c~), S_R = max(v_R + c_R,
// v~ + c~), from the Roe averages (weights sqrt(rho)) of both velocity components and of the
// enthalpy (E + p)/rho, c~^2 = (gamma - 1)(H~ - |v~|^2 / 2).
__device__ void flux_hlle(const double uL[4], const double uR[4], int dir, const Ops& ops, double f[4]) {
  FaceState L, R;
  face_pair(uL, uR, dir, ops, L, R);
  const double sl = sqrt(L.rho), sr = sqrt(R.rho);
  const double iws = rcp_nr(sl + sr);
  const double wl = sl * iws, wr = sr * iws;
  const double vn = fma(wl, L.v, wr * R.v);
  const double vt = fma(wl, L.mt * L.ir, wr * (R.mt * R.ir));
  const double H = fma(wl, (L.E + L.p) * L.ir, wr * ((R.E + R.p) * R.ir));
  const double c = sqrt(ops.gm1 * fma(-0.5, fma(vn, vn, vt * vt), H));
  const double SL = fmin(L.v - L.c, vn - c), SR = fmax(R.v + R.c, vn + c);
  double F[4];
  if (SL >= 0.0) {
    face_flux_rot(L, F);
  } else if (SR <= 0.0) {
    face_flux_rot(R, F);
  } else {
    double FL[4], FR[4];
    face_flux_rot(L, FL);
    face_flux_rot(R, FR);
    const double inv = rcp_nr(SR - SL);
    const double SLSR = SL * SR;
    const double dU[4] = {R.rho - L.rho, R.mn - L.mn, R.mt - L.mt, R.E - L.E};
#pragma unroll
    for (int v = 0; v < 4; ++v) F[v] = fma(SLSR, dU[v], SR * FL[v] - SL * FR[v]) * inv;
  }
  rotate_back(F, dir, f);
}

// HLLC (Toro, Spruce, Speares 1994) with the same speeds and the standard contact speed.
__device__ void flux_hllc(const double uL[4], const double uR[4], int dir, const Ops& ops, double f[4]) {
  FaceState L, R;
  face_pair(uL, uR, dir, ops, L, R);
  const double SL = fmin(L.v - L.c, R.v - R.c), SR = fmax(L.v + L.c, R.v + R.c);
  double F[4];
  if (SL >= 0.0) {
    face_flux_rot(L, F);
  } else if (SR <= 0.0) {
    face_flux_rot(R, F);
  } else {
    const double mL = L.rho * (SL - L.v), mR = R.rho * (SR - R.v);
    const double Ss = (R.p - L.p + mL * L.v - mR * R.v) * rcp_nr(mL - mR);
    const bool left = Ss >= 0.0;
    const FaceState& K = left ? L : R;
    const double S = left ? SL : SR;
    const double m = left ? mL : mR;
    face_flux_rot(K, F);
    // one reciprocal for fac = m / (S - S*) and p / m
    const double q = rcp_nr((S - Ss) * m);
    const double fac = m * m * q;
    const double p_over_m = K.p * (S - Ss) * q;
    const double Us[4] = {fac, fac * Ss, fac * (K.mt * K.ir), fac * fma(Ss - K.v, Ss + p_over_m, K.E * K.ir)};
    const double Uk[4] = {K.rho, K.mn, K.mt, K.E};
#pragma unroll
    for (int v = 0; v < 4; ++v) F[v] = fma(S, Us[v] - Uk[v], F[v]);
  }
  rotate_back(F, dir, f);
}

__device__ void flux_ec_surface(const double uL[4], const double uR[4], int dir, const Ops& ops, double f[4]) {
  const Prim A = prim_from_cons(uL, ops.gm1), B = prim_from_cons(uR, ops.gm1);
  ec_flux(A, B, dir, ops.inv_gm1, f);
}

__device__ __forceinline__ void surface_flux(const double uL[4], const double uR[4], int dir, const Ops& ops,
                                             double f[4]) {
  if (ops.surface_flux == PERK_SURFACE_HLLC)
    flux_hllc(uL, uR, dir, ops, f);
  else if (ops.surface_flux == PERK_SURFACE_EC)
    flux_ec_surface(uL, uR, dir, ops, f);
  else if (ops.surface_flux == PERK_SURFACE_HLLE)
    flux_hlle(uL, uR, dir, ops, f);
  else
    flux_hll(uL, uR, dir, ops, f);
}

// Stamps of the fused kernels: the stage of the step that last wrote a face's numerical flux
// (k_stage, k_step) or completed an element's stage vector (k_step).
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

constexpr int STAMP_WAIT_LIMIT = 1 << 23;   // polls (about 32 ns apart) before a wait gives up

// waits until the stamp at p reaches v (relaxed polls, then one fence: the values were written
// before the stamp was released; stamps only grow); false if the wait gives up
__device__ __forceinline__ bool wait_stamp(const unsigned long long* p, unsigned long long v) {
  unsigned ns = 32;
  for (int it = 0; it < STAMP_WAIT_LIMIT; ++it) {
    if (ld_relaxed(p) >= v) {
      __threadfence();
      return true;
    }
    __nanosleep(ns);
    ns = ns < 512 ? 2 * ns : 512;   // back off: few polls from many waiting warps
  }
  return false;
}

// ---------------------------------------------------------------------------
// Stage state at one node of element e.
__device__ __forceinline__ int face_node(int face, int k) {
  // faces: 0 = -x (i = 0), 1 = +x (i = N), 2 = -y (j = 0), 3 = +y (j = N); node index = j * 4 + i
  return face == 0 ? 4 * k : face == 1 ? 4 * k + 3 : face == 2 ? k : 12 + k;
}

// Y_LIVE (one launch per step): as Y_COMBINE, but K_1 and K_{i-1} are written by the same launch:
// the element's progress stamp is awaited first, and they are read through L2 (not the read-only
// path, which may hold values from before the launch wrote them).
constexpr int Y_LIVE = 2;

template <int YS>
__device__ __forceinline__ double ld_stage_vec(const double* p) {
  if (YS == Y_LIVE) return __ldcg(p);
  return __ldg(p);
}

template <int YS>
__device__ __forceinline__ void stage_state(const StageArgs& sa, int64_t e, int m, int node, double y[4]) {
  const int64_t base = e * ELEM + node;
  if (YS == Y_GIVEN) {
#pragma unroll
    for (int v = 0; v < 4; ++v) y[v] = __ldg(sa.Y + base + v * NODES);
  } else {
    const StageCoef c = sa.coef[m];
    const double dt = sa.dt[sa.member ? sa.member[e] : 0];
    const bool use_a = __double_as_longlong(c.alpha) != 0;   // integer tests, off the FP64 pipe
    const bool use_b = __double_as_longlong(c.beta) != 0;
    if (YS == Y_LIVE && sa.prog && (use_a || use_b)) {
      // K_{i-1} is complete once stage i-1 of the element is, K_1 once stage 0 is
      if (!wait_stamp(sa.prog + e, sa.prog_base + (use_b ? sa.stage : 1))) atomicOr(sa.err, 2);
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) y[v] = __ldg(sa.U + base + v * NODES);
    if (use_a) {
      const double da = dt * c.alpha;
#pragma unroll
      for (int v = 0; v < 4; ++v) y[v] = fma(da, ld_stage_vec<YS>(sa.K1 + base + v * NODES), y[v]);
    }
    if (use_b) {
      const double db = dt * c.beta;
      const double* Kp = coupled_stage(sa, c);
#pragma unroll
      for (int v = 0; v < 4; ++v) y[v] = fma(db, ld_stage_vec<YS>(Kp + base + v * NODES), y[v]);
    }
  }
}

// ---------------------------------------------------------------------------
// Faces: 4 threads per interface (one per face node), 8 per mortar (half, node).
constexpr int FACE_THREADS = 32;
constexpr int IF_PER_BLOCK = FACE_THREADS / 4;
constexpr int MORT_PER_BLOCK = FACE_THREADS / 8;

// 8 interfaces (4 threads each, one per face node) starting at `first`.  STAMP: after the
// fluxes are written, each interface's two element faces are stamped with `stamp` (release), so
// that a volume item of the same launch may read them.
template <int YS, bool STAMP>
__device__ __forceinline__ void face_item_interfaces(const Ops& ops, int64_t n_if, const int4* __restrict__ ifs,
                                                     int64_t first, const StageArgs& sa, double* __restrict__ surf,
                                                     unsigned long long* stamps, unsigned long long stamp) {
  const int64_t idx = first + (threadIdx.x >> 2);
  const int k = threadIdx.x & 3;
  const bool valid = idx < n_if;
  int4 r = make_int4(0, 0, 0, 0);
  if (valid) {
    r = ifs[idx];
    const int dir = r.z;
    double uL[4], uR[4], f[4];
    stage_state<YS>(sa, r.x, r.w, face_node(2 * dir + 1, k), uL);
    stage_state<YS>(sa, r.y, r.w, face_node(2 * dir, k), uR);
    surface_flux(uL, uR, dir, ops, f);
    double* sL = surf + (int64_t)r.x * ELEM + (2 * dir + 1) * 16 + k;
    double* sR = surf + (int64_t)r.y * ELEM + (2 * dir) * 16 + k;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      sL[4 * v] = f[v];
      sR[4 * v] = f[v];
    }
  }
  if (STAMP) {
    __threadfence();
    __syncwarp();
    if (valid && k == 0) {
      st_release(stamps + 4 * (int64_t)r.x + 2 * r.z + 1, stamp);
      st_release(stamps + 4 * (int64_t)r.y + 2 * r.z, stamp);
    }
  }
}

// 4 mortars (8 threads each: half, node) starting at `first`: the large trace interpolated to
// each half, the flux at the small side's nodes, its L2 projection back onto the large face.
template <int YS, bool STAMP>
__device__ __forceinline__ void face_item_mortars(const Ops& ops, int64_t n_mort, const int4* __restrict__ morts,
                                                  int64_t first, const int32_t* __restrict__ method,
                                                  const StageArgs& sa, double* __restrict__ surf,
                                                  double (*s_half)[2][4][NN], unsigned long long* stamps,
                                                  unsigned long long stamp) {
  const int lm = threadIdx.x >> 3;
  const int64_t idx = first + lm;
  const int half = (threadIdx.x >> 2) & 1;
  const int k = threadIdx.x & 3;
  const bool valid = idx < n_mort;
  int4 r = make_int4(0, 0, 0, 0);
  if (valid) r = morts[idx];
  const int dir = r.w & 1, large_side = (r.w >> 1) & 1, m_fine = r.w >> 2;
  const int large_face = large_side == 0 ? 2 * dir + 1 : 2 * dir;
  const int small_face = large_side == 0 ? 2 * dir : 2 * dir + 1;
  const int small = half ? r.z : r.y;
  if (valid) {
    // trace of the large element interpolated to node k of this half
    double ul[4][4];
    const int m_large = method[r.x];
#pragma unroll
    for (int l = 0; l < NN; ++l) stage_state<YS>(sa, r.x, m_large, face_node(large_face, l), ul[l]);
    double ui[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int l = 0; l < NN; ++l) {
      const double w = half ? ops.p_hi[k][l] : ops.p_lo[k][l];
#pragma unroll
      for (int v = 0; v < 4; ++v) ui[v] = fma(w, ul[l][v], ui[v]);
    }
    double us[4], f[4];
    stage_state<YS>(sa, small, m_fine, face_node(small_face, k), us);
    if (large_side == 0)
      surface_flux(ui, us, dir, ops, f);
    else
      surface_flux(us, ui, dir, ops, f);
    double* s = surf + (int64_t)small * ELEM + small_face * 16 + k;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      s[4 * v] = f[v];
      s_half[lm][half][v][k] = f[v];
    }
  }
  __syncwarp();
  if (valid) {
    // projection onto the large face: thread (half, k) produces vars 2*half, 2*half+1 at node k
#pragma unroll
    for (int vv = 0; vv < 2; ++vv) {
      const int v = 2 * half + vv;
      double acc = 0.0;
#pragma unroll
      for (int l = 0; l < NN; ++l) {
        acc = fma(ops.r_lo[k][l], s_half[lm][0][v][l], acc);
        acc = fma(ops.r_hi[k][l], s_half[lm][1][v][l], acc);
      }
      surf[(int64_t)r.x * ELEM + large_face * 16 + 4 * v + k] = acc;
    }
  }
  if (STAMP) {
    __threadfence();
    __syncwarp();
    if (valid && k == 0) {
      st_release(stamps + 4 * (int64_t)small + small_face, stamp);
      if (half == 0) st_release(stamps + 4 * (int64_t)r.x + large_face, stamp);
    }
  }
}

template <int YS>
__global__ void __launch_bounds__(FACE_THREADS) k_faces(Ops ops, int64_t n_if, const int4* __restrict__ ifs,
                                                         int64_t n_mort, const int4* __restrict__ morts,
                                                         int64_t if_blocks, const int32_t* __restrict__ method,
                                                         StageArgs sa, double* __restrict__ surf) {
  __shared__ double s_half[MORT_PER_BLOCK][2][4][NN];  // [mortar][half][var][node]
  if (blockIdx.x < if_blocks)
    face_item_interfaces<YS, false>(ops, n_if, ifs, (int64_t)blockIdx.x * IF_PER_BLOCK, sa, surf, nullptr, 0);
  else
    face_item_mortars<YS, false>(ops, n_mort, morts, (int64_t)(blockIdx.x - if_blocks) * MORT_PER_BLOCK, method, sa,
                                 surf, s_half, nullptr, 0);
}

// ---------------------------------------------------------------------------
// Volume integral (flux differencing) + surface lifting + Jacobian.
// 16 threads per element (one per node), VOL_ELEMS = 2, 4 or 8 elements per block (chosen per
// context by perk_autotune_volume; 2 by default: small blocks spread the element-stages evenly
// over the SMs when a stage has only a few thousand active elements).
constexpr int NPAIR = 48;  // 2 directions x 4 lines x 6 pairs

__device__ __forceinline__ int pair_slot(int a, int b) {  // a < b, slots 0..5
  return (a * (7 - a)) / 2 + b - a - 1;
}

// Where a volume item of the fused stage kernel finds its element's face fluxes: the stamps of
// the face items of the same launch (its faces are done once all four carry `stamp`).
struct FaceWait {
  const unsigned long long* stamps;
  unsigned long long stamp;
  int* err;                    // bit 1 raised if a wait gives up
  unsigned long long* prog;    // one launch per step: the elements' progress stamps (else nullptr)
};
// Shared memory of a volume item (VOL_ELEMS elements, 16 threads each); with shock capturing
// also the stage state and the indicator variable.
template <int VOL_ELEMS, bool SHOCK>
struct VolumeShared {
  NodeQ prim[VOL_ELEMS][NODES];
  double flux[VOL_ELEMS][4][NPAIR];
  double u[VOL_ELEMS][4][NODES];
  double eps[VOL_ELEMS][NODES];
};
template <int VOL_ELEMS>
struct VolumeShared<VOL_ELEMS, false> {
  NodeQ prim[VOL_ELEMS][NODES];
  double flux[VOL_ELEMS][4][NPAIR];
  double (*u)[4][NODES];    // unused without shock capturing
  double (*eps)[NODES];
};

// Volume term of VOL_ELEMS active elements (list slots slot0 ..), their surface lifting and
// Jacobian; the log table is in s_log.  FUSED: the face fluxes come from face items of the same
// launch, read once the element's four faces carry the launch's stamp.
template <int YS, bool CHECK, int VOL_ELEMS, bool SHOCK, bool FUSED>
__device__ __forceinline__ void volume_item(const Ops& ops, int64_t n, int64_t slot0, const int32_t* __restrict__ elems,
                                            const int32_t* __restrict__ level, const int32_t* __restrict__ method,
                                            double two_over_len, const StageArgs& sa,
                                            const double* __restrict__ surf, double* __restrict__ K,
                                            const UpdateArgs& ua, const double* __restrict__ log_table,
                                            double* s_log, VolumeShared<VOL_ELEMS, SHOCK>& sh,
                                            const FaceWait& fw) {
  auto& s_prim = sh.prim;
  auto& s_flux = sh.flux;
  auto& s_u = sh.u;
  auto& s_eps = sh.eps;
  const int le = threadIdx.x >> 4;
  const int t = threadIdx.x & 15;
  const int i = t & 3, j = t >> 2;
  const int64_t slot = slot0 + le;
  const bool valid = slot < n;
  const int64_t e = valid ? elems[slot] : 0;
  const int m = valid ? method[e] : 0;

  // every global load of the launch is issued here, before the first barrier: the grid is
  // usually a single wave, so a load issued later would stall all warps at the same time
  double y[4];
  if (valid) {
    stage_state<YS>(sa, e, m, t, y);
  } else {
    y[0] = 1.0; y[1] = 0.0; y[2] = 0.0; y[3] = 2.5;
  }
  // numerical fluxes of the faces through this node (x face at i = 0 or 3, y face at j = 0 or 3)
  double fsx[4] = {0.0, 0.0, 0.0, 0.0}, fsy[4] = {0.0, 0.0, 0.0, 0.0};
  if (!FUSED && valid) {
    const double* sf = surf + e * ELEM;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      if (i == 0) fsx[v] = __ldg(sf + 0 * 16 + 4 * v + j);
      if (i == 3) fsx[v] = __ldg(sf + 1 * 16 + 4 * v + j);
      if (j == 0) fsy[v] = __ldg(sf + 2 * 16 + 4 * v + i);
      if (j == 3) fsy[v] = __ldg(sf + 3 * 16 + 4 * v + i);
    }
  }
  for (int q = threadIdx.x; q < 2 * LOG_TABLE; q += VOL_ELEMS * NODES) s_log[q] = log_table[q];
  __syncthreads();
  {
    // node logarithms only where some pair of the element leaves the series range of the means
    NodeQ q = node_q_nolog(y, ops.gm1);
    unsigned long long rmin = dbits(q.rho), rmax = rmin, bmin = dbits(q.beta), bmax = bmin;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {   // the element's 16 lanes
      rmin = min(rmin, __shfl_xor_sync(0xffffffffu, rmin, o, 16));
      rmax = max(rmax, __shfl_xor_sync(0xffffffffu, rmax, o, 16));
      bmin = min(bmin, __shfl_xor_sync(0xffffffffu, bmin, o, 16));
      bmax = max(bmax, __shfl_xor_sync(0xffffffffu, bmax, o, 16));
    }
    if (!series_only(rmin, rmax, bmin, bmax)) {
      q.lnrho = log_tab(q.rho, s_log, s_log + LOG_TABLE);
      q.lnbeta = log_tab(q.beta, s_log, s_log + LOG_TABLE);
    }
    s_prim[le][t] = q;
  }
  __syncwarp();

  // the three pairs of this thread: slots t, t + 16, t + 32 of 48
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
    double f[4];
    ec_flux_q(s_prim[le][na], s_prim[le][nb], dir, ops.inv_gm1, f);
#pragma unroll
    for (int v = 0; v < 4; ++v) s_flux[le][v][p] = f[v];
  }
  __syncwarp();

  double dx[4], dy[4];
#pragma unroll
  for (int mm = 0; mm < 4; ++mm) {
    dx[mm] = ops.dsplit[i][mm];
    dy[mm] = ops.dsplit[j][mm];
  }
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int mm = 0; mm < 4; ++mm) {
    if (mm != i) {
      const int p = j * 6 + pair_slot(min(i, mm), max(i, mm));
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[v] = fma(dx[mm], s_flux[le][v][p], acc[v]);
    }
    if (mm != j) {
      const int p = 24 + i * 6 + pair_slot(min(j, mm), max(j, mm));
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[v] = fma(dy[mm], s_flux[le][v][p], acc[v]);
    }
  }

  if (SHOCK) {
    // subcell shock capturing: the element's blending factor from the modes of its indicator
    // variable, then (1 - alpha) (flux differencing) + alpha (subcell finite volumes)
    const unsigned gmask = 0xFFFFu << (threadIdx.x & 16);   // the 16 lanes of this element
    s_eps[le][t] = ops.shock == PERK_SHOCK_DENSITY ? y[0] : y[0] * (2.0 * s_prim[le][t].hp);
#pragma unroll
    for (int v = 0; v < 4; ++v) s_u[le][v][t] = y[v];
    __syncwarp(gmask);   // also: every lane of the element has consumed the pair fluxes
    double md = 0.0;     // mode (a, b) = (i, j) in the orthonormal Legendre basis
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      double r = 0.0;
#pragma unroll
      for (int ii = 0; ii < 4; ++ii) r = fma(ops.vinv[i][ii], s_eps[le][jj * 4 + ii], r);
      md = fma(ops.vinv[j][jj], r, md);
    }
    const double m2 = md * md;
    const int shell = max(i, j);
    double top = shell == 3 ? m2 : 0.0, mid = shell == 2 ? m2 : 0.0, low = shell <= 1 ? m2 : 0.0;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      top += __shfl_xor_sync(0xffffffffu, top, o, 16);
      mid += __shfl_xor_sync(0xffffffffu, mid, o, 16);
      low += __shfl_xor_sync(0xffffffffu, low, o, 16);
    }
    const double energy = fmax(top / (top + mid + low), mid / (mid + low));
    double alpha = 1.0 / (1.0 + exp(-ops.sc_s_over_T * (energy - ops.sc_T)));
    alpha = alpha < 1e-3 ? 0.0 : fmin(alpha, ops.alpha_max);
    if (alpha > 0.0) {   // the same for the element's 16 lanes
      // the 24 subcell fluxes: q < 12 along x (row q / 3, between nodes q % 3 and q % 3 + 1),
      // q >= 12 along y (column (q - 12) / 3); stored over the consumed pair fluxes
      for (int qq = t; qq < 24; qq += 16) {
        const int dq = qq >= 12, r = dq ? qq - 12 : qq, line = r / 3, k = r - 3 * line;
        const int na = dq ? k * 4 + line : line * 4 + k;
        const int nb = dq ? (k + 1) * 4 + line : line * 4 + k + 1;
        double ua[4], ub[4], f[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          ua[v] = s_u[le][v][na];
          ub[v] = s_u[le][v][nb];
        }
        surface_flux(ua, ub, dq, ops, f);
#pragma unroll
        for (int v = 0; v < 4; ++v) s_flux[le][v][qq] = f[v];
      }
      __syncwarp(gmask);
      // finite-volume term at this node, (F_{i+1/2} - F_{i-1/2}) / w_i in x plus the same in y, with
      // zero at the element ends: there the physical flux of the strong form's surface term cancels,
      // as it does against the diagonal of the flux-differencing term
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const double fxr = i < 3 ? s_flux[le][v][j * 3 + i] : 0.0;
        const double fxl = i > 0 ? s_flux[le][v][j * 3 + i - 1] : 0.0;
        const double fyr = j < 3 ? s_flux[le][v][12 + i * 3 + j] : 0.0;
        const double fyl = j > 0 ? s_flux[le][v][12 + i * 3 + j - 1] : 0.0;
        const double fv = (fxr - fxl) * ops.inv_w[i] + (fyr - fyl) * ops.inv_w[j];
        acc[v] = fma(alpha, fv - acc[v], acc[v]);
      }
    }
  }
  if (!valid) return;

  if (FUSED) {
    // the element's four faces, written by face items of the same launch that were all dispensed
    // before this item: lane t < 4 of the element watches face t, then the element's lanes meet
    if (t < 4 && !wait_stamp(fw.stamps + 4 * e + t, fw.stamp)) atomicOr(fw.err, 2);
    __syncwarp(0xFFFFu << (threadIdx.x & 16));
    const double* sf = surf + e * ELEM;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      if (i == 0) fsx[v] = __ldcg(sf + 0 * 16 + 4 * v + j);
      if (i == 3) fsx[v] = __ldcg(sf + 1 * 16 + 4 * v + j);
      if (j == 0) fsy[v] = __ldcg(sf + 2 * 16 + 4 * v + i);
      if (j == 3) fsy[v] = __ldcg(sf + 3 * 16 + 4 * v + i);
    }
  }

  // surface lifting with the numerical fluxes of the four faces (w_0 = w_N)
  const double iw = ops.inv_w0;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    if (i == 0) acc[v] = fma(-iw, fsx[v], acc[v]);
    if (i == 3) acc[v] = fma(iw, fsx[v], acc[v]);
    if (j == 0) acc[v] = fma(-iw, fsy[v], acc[v]);
    if (j == 3) acc[v] = fma(iw, fsy[v], acc[v]);
  }
  const double scale = -ldexp(two_over_len, level[e]);  // -(2/h)
  double kv[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    kv[v] = scale * acc[v];
    K[e * ELEM + v * NODES + t] = kv[v];
  }
  if (FUSED && fw.prog) {
    // one launch per step: this stage of the element is complete (its K values written first)
    __threadfence();
    __syncwarp(0xFFFFu << (threadIdx.x & 16));
    if (t == 0) st_release(fw.prog + e, fw.stamp);
  }
  if (CHECK) {
    // admissibility of the state this step would commit at this node (K_1 and K_{S-1} were written
    // earlier in the same launch where YS is Y_LIVE, and are complete: this element's stage
    // state waited for them)
    const double dt = sa.dt[sa.member ? sa.member[e] : 0];
    const int64_t base = e * ELEM + t;
    double un[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      double inc = ua.bs * kv[v];
      if (ua.b1 != 0.0) inc = fma(ua.b1, ld_stage_vec<YS>(ua.K1 + base + v * NODES), inc);
      if (ua.bp != 0.0) inc = fma(ua.bp, ld_stage_vec<YS>(ua.Kp + base + v * NODES), inc);
      un[v] = fma(dt, inc, __ldg(ua.U + base + v * NODES));
    }
    const double p = ops.gm1 * (un[3] - 0.5 * (un[1] * un[1] + un[2] * un[2]) / un[0]);
    const bool ok = isfinite(un[0]) && isfinite(un[1]) && isfinite(un[2]) && isfinite(un[3]) && un[0] > 0.0 &&
                    p > 0.0 && isfinite(p);
    if (!ok) *ua.flag = 1;
  }
}

template <int YS, bool CHECK, int VOL_ELEMS, bool SHOCK>
__global__ void __launch_bounds__(VOL_ELEMS * NODES) k_volume(Ops ops, int64_t n, const int32_t* __restrict__ elems,
                                                         const int32_t* __restrict__ level,
                                                         const int32_t* __restrict__ method, double two_over_len,
                                                         StageArgs sa, const double* __restrict__ surf,
                                                         double* __restrict__ K, UpdateArgs ua,
                                                         const double* __restrict__ log_table) {
  __shared__ VolumeShared<VOL_ELEMS, SHOCK> sh;
  __shared__ double s_log[2 * LOG_TABLE];
  volume_item<YS, CHECK, VOL_ELEMS, SHOCK, false>(ops, n, (int64_t)blockIdx.x * VOL_ELEMS, elems, level, method,
                                                  two_over_len, sa, surf, K, ua, log_table, s_log, sh, FaceWait{});
}

// ---------------------------------------------------------------------------
// One stage in one launch (Euler, the plain volume term): the face items (8 interfaces or 4
// mortars each) and the volume items (2 elements each) of the stage's active prefixes are one
// work list, one item per one-warp block.  A volume item computes its flux differencing, then
// waits for the stamps of its element's four faces (set by the face items with release
// semantics) before the surface lifting.  Face items never wait.  When every block of the launch
// can be resident at once (`resident`), block b takes item b of a list that spreads the face
// items evenly among the volume items, so each SM gets its share of both kinds of work; the
// blocks a volume item waits for are running.  Otherwise items are dealt faces first by an
// atomic counter: every face item has then been handed out, to a block already running, before
// any volume item, so the waits end either way.  The face work runs beside the volume work and
// the stage needs no second launch.  ctl[stage] counts the stage's dealt items and ctl[MAX_S] the
// steps; both are advanced by the step's final update (k_commit), so a stamp
// (steps * MAX_S + stage + 1) names one stage of one step.
struct StageSync {
  unsigned long long* ctl;      // [MAX_S] per-stage item counters, then [MAX_S] the step count
  unsigned long long* stamps;   // [n_elem][4 faces]
  int* err;                     // bit 1: a wait gave up (the step is then not committed)
  int stage;
};

constexpr int STAGE_VE = 2;   // elements per volume item

template <bool CHECK>
__global__ void __launch_bounds__(FACE_THREADS) k_stage(Ops ops, int64_t n_if, const int4* __restrict__ ifs,
                                                       int64_t n_mort, const int4* __restrict__ morts, int64_t n_el,
                                                       const int32_t* __restrict__ elems,
                                                       const int32_t* __restrict__ level,
                                                       const int32_t* __restrict__ method, double two_over_len,
                                                       StageArgs sa, double* __restrict__ surf,
                                                       double* __restrict__ K, UpdateArgs ua,
                                                       const double* __restrict__ log_table, StageSync sync,
                                                       bool resident) {
  static_assert(STAGE_VE * NODES == FACE_THREADS, "one warp per work item");
  __shared__ unsigned long long s_item, s_launch;
  __shared__ double s_log[2 * LOG_TABLE];
  __shared__ union {
    VolumeShared<STAGE_VE, false> vol;
    double half[MORT_PER_BLOCK][2][4][NN];
  } sh;
  const int64_t if_items = (n_if + IF_PER_BLOCK - 1) / IF_PER_BLOCK;
  const int64_t face_items = if_items + (n_mort + MORT_PER_BLOCK - 1) / MORT_PER_BLOCK;
  const int64_t items = face_items + (n_el + STAGE_VE - 1) / STAGE_VE;
  const int64_t face_items0 = face_items;
  if (threadIdx.x == 0) {
    if (resident) {
      // every block of the launch is resident at once: block b takes item b of a list in which
      // the face items are spread evenly over the volume items (F of T items are faces; block b is
      // a face block when floor((b + 1) F / T) > floor(b F / T)), so every SM gets its share of both
      const int64_t b = blockIdx.x, F = face_items0, T = (int64_t)gridDim.x;
      const int64_t f0 = b * F / T, f1 = (b + 1) * F / T;
      s_item = f1 > f0 ? (unsigned long long)f0 : (unsigned long long)(F + b - f1);
    } else {
      s_item = atomicAdd(sync.ctl + sync.stage, 1ull);
    }
    s_launch = *(volatile unsigned long long*)(sync.ctl + MAX_S);
  }
  __syncwarp();
  const int64_t item = (int64_t)s_item;
  const unsigned long long stamp = s_launch * MAX_S + sync.stage + 1;
  if (item < if_items) {
    face_item_interfaces<Y_COMBINE, true>(ops, n_if, ifs, item * IF_PER_BLOCK, sa, surf, sync.stamps, stamp);
  } else if (item < face_items) {
    face_item_mortars<Y_COMBINE, true>(ops, n_mort, morts, (item - if_items) * MORT_PER_BLOCK, method, sa, surf,
                                       sh.half, sync.stamps, stamp);
  } else if (item < items) {
    volume_item<Y_COMBINE, CHECK, STAGE_VE, false, true>(ops, n_el, (item - face_items) * STAGE_VE, elems, level,
                                                         method, two_over_len, sa, surf, K, ua, log_table, s_log,
                                                         sh.vol, FaceWait{sync.stamps, stamp, sync.err, nullptr});
  }
}

// One launch per step: every warp takes items in stage order from one counter (the next one
// fetched while the current one runs).  An item waits, with bounded waits, only for items dealt
// before it (a face item for the stage vectors of its elements, a volume item for those and for
// its four faces), so the warp holding the smallest unfinished item never waits and every
// wait ends.  The waits also order the reuse of the buffers: the two buffers that alternate for
// K_2, K_3, .. and the face fluxes are overwritten only by items that waited for every reader
// of the previous contents.
int64_t step_stage_items(int64_t n_if, int64_t n_mort, int64_t n_el) {
  return (n_if + IF_PER_BLOCK - 1) / IF_PER_BLOCK + (n_mort + MORT_PER_BLOCK - 1) / MORT_PER_BLOCK +
         (n_el + STAGE_VE - 1) / STAGE_VE;
}

__global__ void __launch_bounds__(FACE_THREADS) k_step(Ops ops, StepPlan plan, const int4* __restrict__ ifs,
                                                      const int4* __restrict__ morts,
                                                      const int32_t* __restrict__ elems,
                                                      const int32_t* __restrict__ level,
                                                      const int32_t* __restrict__ method, double two_over_len,
                                                      StageArgs sa, double* __restrict__ surf, UpdateArgs check,
                                                      const double* __restrict__ log_table, StageSync sync,
                                                      unsigned long long* prog) {
  static_assert(STAGE_VE * NODES == FACE_THREADS, "one warp per work item");
  __shared__ unsigned long long s_launch;
  __shared__ double s_log[2 * LOG_TABLE];
  __shared__ union {
    VolumeShared<STAGE_VE, false> vol;
    double half[MORT_PER_BLOCK][2][4][NN];
  } sh;
  const int lane = threadIdx.x;
  if (lane == 0) s_launch = *(volatile unsigned long long*)(sync.ctl + MAX_S);
  __syncwarp();
  const unsigned long long base = s_launch * MAX_S;
  const int64_t items = plan.first[plan.S];
  unsigned long long next = 0;
  if (lane == 0) next = atomicAdd(sync.ctl, 1ull);
  next = __shfl_sync(0xffffffffu, next, 0);
  for (;;) {
    const int64_t item = (int64_t)next;
    // a wait that gave up abandons the launch (the step is then not committed): no further item
    // waits its full bound
    int gave_up = 0;
    if (lane == 0) gave_up = *(volatile int*)sync.err & 2;
    if (item >= items || __shfl_sync(0xffffffffu, gave_up, 0)) break;
    if (lane == 0) next = atomicAdd(sync.ctl, 1ull);
    next = __shfl_sync(0xffffffffu, next, 0);
    int i = 0;
    while (item >= plan.first[i + 1]) ++i;
    const int64_t local = item - plan.first[i];
    StageArgs s = sa;
    s.Kp = plan.Kp[i];
    s.coef = sa.coef + (size_t)i * MAX_R;
    s.prog = nullptr;   // the item's waits are done here, one lane per element
    const unsigned long long stamp = base + i + 1;
    const int64_t if_items = (plan.n_if[i] + IF_PER_BLOCK - 1) / IF_PER_BLOCK;
    const int64_t face_items = if_items + (plan.n_mort[i] + MORT_PER_BLOCK - 1) / MORT_PER_BLOCK;
    {
      // the element whose stage vectors this lane waits for (-1: none), and its member
      int64_t we = -1;
      int wm = 0;
      if (local < if_items) {
        const int64_t idx = local * IF_PER_BLOCK + (lane >> 2);
        if (idx < plan.n_if[i] && (lane & 3) < 2) {
          const int4 r = ifs[idx];
          we = (lane & 3) == 0 ? r.x : r.y;
          wm = r.w;
        }
      } else if (local < face_items) {
        const int64_t idx = (local - if_items) * MORT_PER_BLOCK + (lane >> 3);
        const int sub = lane & 7;   // 0: the large element, 1, 2: the small ones
        if (idx < plan.n_mort[i] && sub < 3) {
          const int4 r = morts[idx];
          we = sub == 0 ? r.x : (sub == 1 ? r.y : r.z);
          wm = sub == 0 ? method[r.x] : r.w >> 2;
        }
      } else {
        const int64_t slot = (local - face_items) * STAGE_VE + (lane >> 4);
        if (slot < plan.n_el[i] && (lane & 15) == 0) {
          we = elems[slot];
          wm = method[we];
        }
      }
      if (we >= 0) {
        const StageCoef c = s.coef[wm];
        const bool use_a = __double_as_longlong(c.alpha) != 0, use_b = __double_as_longlong(c.beta) != 0;
        // K_{i-1} is complete once stage i-1 of the element is, K_1 once stage 0 is
        if ((use_a || use_b) && !wait_stamp(prog + we, base + (use_b ? i : 1))) atomicOr(sync.err, 2);
      }
      __syncwarp();
    }
    if (local < if_items) {
      face_item_interfaces<Y_LIVE, true>(ops, plan.n_if[i], ifs, local * IF_PER_BLOCK, s, surf, sync.stamps, stamp);
    } else if (local < face_items) {
      face_item_mortars<Y_LIVE, true>(ops, plan.n_mort[i], morts, (local - if_items) * MORT_PER_BLOCK, method, s,
                                      surf, sh.half, sync.stamps, stamp);
    } else {
      const FaceWait fw{sync.stamps, stamp, sync.err, prog};
      const int64_t slot0 = (local - face_items) * STAGE_VE;
      if (i == plan.S - 1)
        volume_item<Y_LIVE, true, STAGE_VE, false, true>(ops, plan.n_el[i], slot0, elems, level, method, two_over_len,
                                                         s, surf, plan.K[i], check, log_table, s_log, sh.vol, fw);
      else
        volume_item<Y_LIVE, false, STAGE_VE, false, true>(ops, plan.n_el[i], slot0, elems, level, method,
                                                          two_over_len, s, surf, plan.K[i], check, log_table, s_log,
                                                          sh.vol, fw);
    }
    __syncwarp();   // the item's shared records are consumed before the next item writes them
  }
}

// Guarded final update U += dt (b1 K1 + bp Kp + bs Ks), skipped entirely when
// the admissibility flag is raised.
__global__ void k_commit(int64_t n2, UpdateArgs ua, const double2* __restrict__ Ks, const double* dtp,
                         double2* __restrict__ U) {
  if (ua.stage_ctl && blockIdx.x == 0 && threadIdx.x == 0) {
    // the fused stage kernels of this step are done: their item counters restart, the step count advances
    for (int s = 0; s < MAX_S; ++s) ua.stage_ctl[s] = 0;
    ua.stage_ctl[MAX_S] += 1;
  }
  if (*ua.flag != 0) return;
  const double2* K1 = reinterpret_cast<const double2*>(ua.K1);
  const double2* Kp = reinterpret_cast<const double2*>(ua.Kp);
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n2; q += (int64_t)gridDim.x * blockDim.x) {
    const double dt = dtp[ua.member ? ua.member[q / (ELEM / 2)] : 0];
    const double2 ks = Ks[q];
    double2 inc = make_double2(ua.bs * ks.x, ua.bs * ks.y);
    if (ua.b1 != 0.0) {
      const double2 k1 = K1[q];
      inc.x = fma(ua.b1, k1.x, inc.x);
      inc.y = fma(ua.b1, k1.y, inc.y);
    }
    if (ua.bp != 0.0) {
      const double2 kp = Kp[q];
      inc.x = fma(ua.bp, kp.x, inc.x);
      inc.y = fma(ua.bp, kp.y, inc.y);
    }
    double2 u = U[q];
    u.x = fma(dt, inc.x, u.x);
    u.y = fma(dt, inc.y, u.y);
    U[q] = u;
  }
}

__global__ void k_set_scalar(double* p, double v) { *p = v; }

// ---------------------------------------------------------------------------
// Level partition: one block; stable counting sort of the element, interface
// and mortar lists by member, finest member first.
constexpr int PART_THREADS = 1024;

__device__ int block_scan_members(int key, int R, int* s_wtot /* [MAX_R][32] */, int* s_wscan, int* rank_out) {
  // returns, for this thread, its rank among threads of the same key (exclusive),
  // and writes the per-key chunk totals to s_wscan[r * 33 + 32]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  int my_rank = 0;
  for (int r = 0; r < R; ++r) {
    const unsigned bal = __ballot_sync(0xffffffffu, key == r);
    if (key == r) my_rank = __popc(bal & lt);
    if (lane == 0) s_wtot[r * 32 + warp] = __popc(bal);
  }
  __syncthreads();
  if (warp < R) {
    const int v = s_wtot[warp * 32 + lane];
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int n = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += n;
    }
    s_wscan[warp * 33 + lane] = incl - v;
    if (lane == 31) s_wscan[warp * 33 + 32] = incl;
  }
  __syncthreads();
  *rank_out = (key >= 0) ? s_wscan[key * 33 + warp] + my_rank : 0;
  return 0;
}

__global__ void __launch_bounds__(PART_THREADS) k_partition(int64_t n_elem, int64_t n_if, int64_t n_mort,
                                                              const int32_t* __restrict__ level,
                                                              const int4* __restrict__ if_raw,
                                                              const int4* __restrict__ mort_raw, int R, int S,
                                                              const int32_t* __restrict__ stage_minmem,
                                                              const int32_t* __restrict__ member, int n_members,
                                                              int32_t* member_lmax, int32_t* method,
                                                              int32_t* elem_sorted, int4* if_sorted,
                                                              int4* mort_sorted, int64_t* counts,
                                                              int32_t* level_minmax, int mort_flag_bits,
                                                              const int64_t* __restrict__ d_nfaces) {
  if (d_nfaces) {
    n_if = d_nfaces[0];
    n_mort = d_nfaces[1];
  }
  __shared__ int s_min, s_max;
  __shared__ int s_cnt[3][MAX_R];
  __shared__ int s_base[MAX_R];
  __shared__ int s_run[MAX_R];
  __shared__ int s_wtot[MAX_R * 32];
  __shared__ int s_wscan[MAX_R * 33];
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_min = 1 << 30;
    s_max = -1;
  }
  if (tid < 3 * MAX_R) s_cnt[tid / MAX_R][tid % MAX_R] = 0;
  __syncthreads();
  int lmin = 1 << 30, lmax = -1;
  for (int64_t e = tid; e < n_elem; e += PART_THREADS) {
    const int l = level[e];
    lmin = min(lmin, l);
    lmax = max(lmax, l);
  }
  atomicMin(&s_min, lmin);
  atomicMax(&s_max, lmax);
  // finest level present in every ensemble member (one member: the global maximum)
  for (int m = tid; m < n_members; m += PART_THREADS) member_lmax[m] = -1;
  __syncthreads();
  for (int64_t e = tid; e < n_elem; e += PART_THREADS) atomicMax(&member_lmax[member ? member[e] : 0], level[e]);
  __syncthreads();
  // P-ERK members and their counts
  for (int64_t e = tid; e < n_elem; e += PART_THREADS) {
    const int Lmax = member_lmax[member ? member[e] : 0];
    const int mth = max(0, (R - 1) - (Lmax - level[e]));
    method[e] = mth;
    atomicAdd(&s_cnt[0][mth], 1);
  }
  __syncthreads();
  for (int64_t q = tid; q < n_if; q += PART_THREADS) atomicAdd(&s_cnt[1][method[if_raw[q].x]], 1);
  for (int64_t q = tid; q < n_mort; q += PART_THREADS) atomicAdd(&s_cnt[2][method[mort_raw[q].y]], 1);
  __syncthreads();

  for (int list = 0; list < 3; ++list) {
    const int64_t n = list == 0 ? n_elem : list == 1 ? n_if : n_mort;
    if (tid == 0) {
      int b = 0;
      for (int r = R - 1; r >= 0; --r) {
        s_base[r] = b;
        b += s_cnt[list][r];
        s_run[r] = 0;
      }
    }
    __syncthreads();
    for (int64_t start = 0; start < n; start += PART_THREADS) {
      const int64_t q = start + tid;
      int key = -1;
      int4 rec = make_int4(0, 0, 0, 0);
      if (q < n) {
        if (list == 0) {
          key = method[q];
        } else if (list == 1) {
          rec = if_raw[q];
          key = method[rec.x];
          rec.w = key;
        } else {
          rec = mort_raw[q];
          key = method[rec.y];
          rec.w = (rec.w & ((1 << mort_flag_bits) - 1)) | (key << mort_flag_bits);
        }
      }
      int rank;
      block_scan_members(key, R, s_wtot, s_wscan, &rank);
      if (key >= 0) {
        const int pos = s_base[key] + s_run[key] + rank;
        if (list == 0)
          elem_sorted[pos] = (int32_t)q;
        else if (list == 1)
          if_sorted[pos] = rec;
        else
          mort_sorted[pos] = rec;
      }
      __syncthreads();
      if (tid < R) s_run[tid] += s_wscan[tid * 33 + 32];
      __syncthreads();
    }
  }
  // active counts per stage: member r is active at stage i (0-based) iff r >= stage_minmem[i]
  // (the members active at a stage are the finest ones, so each active set is a prefix).
  // Halo counts: members r >= stage_minmem[i] - 1.  Face neighbours differ by at most one level
  // (2:1 balance), so their members differ by at most one: the halo prefix holds every element
  // that shares a face with an active one, and every face of those elements.
  if (tid < S) {
    int64_t ce = 0, ci = 0, cm = 0, he = 0, hi = 0, hm = 0;
    for (int r = 0; r < R; ++r) {
      if (r >= stage_minmem[tid]) {
        ce += s_cnt[0][r];
        ci += s_cnt[1][r];
        cm += s_cnt[2][r];
      }
      if (r >= stage_minmem[tid] - 1) {
        he += s_cnt[0][r];
        hi += s_cnt[1][r];
        hm += s_cnt[2][r];
      }
    }
    counts[0 * MAX_S + tid] = ce;
    counts[1 * MAX_S + tid] = ci;
    counts[2 * MAX_S + tid] = cm;
    counts[3 * MAX_S + tid] = he;
    counts[4 * MAX_S + tid] = hi;
    counts[5 * MAX_S + tid] = hm;
  }
  if (tid == 0) {
    level_minmax[0] = s_min;
    level_minmax[1] = s_max;
  }
}

// ---------------------------------------------------------------------------
// CFL step size: min over elements of h_e / max_nodes(|v1| + |v2| + 2c).  A node without an
// admissible state (rho <= 0, p <= 0, NaN or Inf) poisons the minimum with NaN, so that the host
// reports it instead of a step size taken from the other nodes.
__device__ __forceinline__ double nan_min(double a, double b) { return (a != a || b != b) ? NAN : fmin(a, b); }

__global__ void __launch_bounds__(DT_THREADS) k_dt_partial(int64_t n_nodes, const double* __restrict__ U,
                                                            const int32_t* __restrict__ level, double length,
                                                            double gamma, double* block_min) {
  __shared__ double s[DT_THREADS / 32];
  double best = INFINITY;
  for (int64_t q = (int64_t)blockIdx.x * DT_THREADS + threadIdx.x; q < n_nodes; q += (int64_t)gridDim.x * DT_THREADS) {
    const int64_t e = q / NODES;
    const int t = (int)(q - e * NODES);
    const double* u = U + e * ELEM + t;
    const double rho = u[0], ir = 1.0 / rho;
    const double v1 = u[NODES] * ir, v2 = u[2 * NODES] * ir;
    const double p = (gamma - 1.0) * (u[3 * NODES] - 0.5 * rho * (v1 * v1 + v2 * v2));
    const double c = sqrt(gamma * p * ir);
    const double lam = fabs(v1) + fabs(v2) + 2.0 * c;
    const double h = ldexp(length, -level[e]);
    const double r = h / lam;
    best = (rho > 0.0 && p > 0.0 && r > 0.0 && r < INFINITY) ? nan_min(best, r) : NAN;
  }
  for (int o = 16; o > 0; o >>= 1) best = nan_min(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    best = threadIdx.x < DT_THREADS / 32 ? s[threadIdx.x] : INFINITY;
    for (int o = 16; o > 0; o >>= 1) best = nan_min(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (threadIdx.x == 0) block_min[blockIdx.x] = best;
  }
}

__global__ void k_dt_final(int n, const double* block_min, double* out) {
  double best = INFINITY;
  for (int q = threadIdx.x; q < n; q += 32) best = nan_min(best, block_min[q]);
  for (int o = 16; o > 0; o >>= 1) best = nan_min(best, __shfl_xor_sync(0xffffffffu, best, o));
  if (threadIdx.x == 0) *out = best;
}

// ---------------------------------------------------------------------------
// AMR: density-gradient indicator and solution transfer (16 threads per cell).
constexpr int AMR_THREADS = 128;
constexpr int AMR_ELEMS = AMR_THREADS / NODES;

// eta_e = h max_nodes |grad rho| / mean(rho) = 2 max_nodes |(D rho)_x, (D rho)_y| / mean(rho)
__global__ void __launch_bounds__(AMR_THREADS) k_indicator(int64_t n, const double* __restrict__ U, Ops ops,
                                                            double w0, double w1, int kind,
                                                            double* __restrict__ eta) {
  __shared__ double s_f[AMR_ELEMS][NODES];
  const int le = threadIdx.x >> 4, t = threadIdx.x & 15, i = t & 3, j = t >> 2;
  const int64_t e = (int64_t)blockIdx.x * AMR_ELEMS + le;
  const bool valid = e < n;
  const double rho = valid ? U[e * ELEM + t] : 1.0;
  if (kind == PERK_INDICATOR_LOHNER_VX) {
    // Loehner's estimator of v_x; round-to-nearest operations in a fixed order
    const double vx = valid ? U[e * ELEM + NODES + t] / rho : 0.0;
    s_f[le][t] = vx;
    __syncwarp();
    double r = 0.0;
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const int c = d ? j : i;                       // position of this node along the line
      if (c == 0 || c == 3) continue;
      const int step = d ? 4 : 1;
      const double um = s_f[le][t - step], u0 = vx, up = s_f[le][t + step];
      const double num = fabs(__dadd_rn(__dsub_rn(up, __dmul_rn(2.0, u0)), um));
      const double den = __dadd_rn(__dadd_rn(fabs(__dsub_rn(up, u0)), fabs(__dsub_rn(u0, um))),
                                   __dmul_rn(PERK_LOHNER_EPS,
                                             __dadd_rn(__dadd_rn(fabs(up), __dmul_rn(2.0, fabs(u0))), fabs(um))));
      if (den > 0.0) r = fmax(r, num / den);
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o, 16));
    if (valid && t == 0) eta[e] = r;
    return;
  }
  s_f[le][t] = rho;
  __syncwarp();
  double gx = 0.0, gy = 0.0;
#pragma unroll
  for (int m = 0; m < NN; ++m) {
    // the derivative matrix is dsplit/2 off the diagonal; its diagonal is -(row sum)
    const double dxm = 0.5 * ops.dsplit[i][m], dym = 0.5 * ops.dsplit[j][m];
    gx = fma(dxm, s_f[le][j * 4 + m] - s_f[le][j * 4 + i], gx);
    gy = fma(dym, s_f[le][m * 4 + i] - s_f[le][j * 4 + i], gy);
  }
  double g2 = fma(gx, gx, gy * gy);
  const double wi = (i == 0 || i == 3) ? w0 : w1, wj = (j == 0 || j == 3) ? w0 : w1;
  double wr = wi * wj * rho;
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    g2 = fmax(g2, __shfl_xor_sync(0xffffffffu, g2, o, 16));
    wr += __shfl_xor_sync(0xffffffffu, wr, o, 16);
  }
  if (valid && t == 0) eta[e] = 2.0 * sqrt(g2) / (0.25 * wr);
}

// kind 0: copy src[0]; kind 1: child (cx, cy) of parent src[0] by interpolation;
// kind 2: parent of the four children src[0..3] (order cx + 2 cy) by L2 projection.
__global__ void __launch_bounds__(AMR_THREADS) k_transfer(int64_t n, const int32_t* __restrict__ map,
                                                           const double* __restrict__ Uold, Ops ops,
                                                           double* __restrict__ Unew) {
  __shared__ double s_src[AMR_ELEMS][4][ELEM];
  const int le = threadIdx.x >> 4, t = threadIdx.x & 15, i = t & 3, j = t >> 2;
  const int64_t e = (int64_t)blockIdx.x * AMR_ELEMS + le;
  if (e >= n) return;   // whole half-warps drop out together; only __syncwarp below
  const int32_t* rec = map + 5 * e;
  const int kind = rec[0] & 3, cx = (rec[0] >> 2) & 1, cy = (rec[0] >> 3) & 1;
  const int nsrc = kind == 2 ? 4 : 1;
  for (int s = 0; s < nsrc; ++s)
    for (int q = t; q < ELEM; q += NODES) s_src[le][s][q] = Uold[(int64_t)rec[1 + s] * ELEM + q];
  __syncwarp(0xffffu << (threadIdx.x & 16));
  double out[4];
  if (kind == 0) {
#pragma unroll
    for (int v = 0; v < 4; ++v) out[v] = s_src[le][0][v * NODES + t];
  } else if (kind == 1) {
    const double(*Px)[NN] = cx ? ops.p_hi : ops.p_lo;
    const double(*Py)[NN] = cy ? ops.p_hi : ops.p_lo;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      double acc = 0.0;
      for (int b = 0; b < NN; ++b) {
        double row = 0.0;
        for (int a = 0; a < NN; ++a) row = fma(Px[i][a], s_src[le][0][v * NODES + b * 4 + a], row);
        acc = fma(Py[j][b], row, acc);
      }
      out[v] = acc;
    }
  } else {
#pragma unroll
    for (int v = 0; v < 4; ++v) out[v] = 0.0;
    for (int c = 0; c < 4; ++c) {
      const double(*Rx)[NN] = (c & 1) ? ops.r_hi : ops.r_lo;
      const double(*Ry)[NN] = (c & 2) ? ops.r_hi : ops.r_lo;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        for (int b = 0; b < NN; ++b) {
          double row = 0.0;
          for (int a = 0; a < NN; ++a) row = fma(Rx[i][a], s_src[le][c][v * NODES + b * 4 + a], row);
          out[v] = fma(Ry[j][b], row, out[v]);
        }
      }
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) Unew[e * ELEM + v * NODES + t] = out[v];
}

// ---------------------------------------------------------------------------
// launchers
cudaError_t launch_indicator(cudaStream_t st, int64_t n, const double* U, const Ops& ops, double w0, double w1,
                             int kind, double* eta) {
  if (n == 0) return cudaSuccess;
  k_indicator<<<(unsigned)((n + AMR_ELEMS - 1) / AMR_ELEMS), AMR_THREADS, 0, st>>>(n, U, ops, w0, w1, kind, eta);
  return cudaGetLastError();
}

cudaError_t launch_transfer(cudaStream_t st, int64_t n, const int32_t* map, const double* Uold, const Ops& ops,
                            double* Unew) {
  if (n == 0) return cudaSuccess;
  k_transfer<<<(unsigned)((n + AMR_ELEMS - 1) / AMR_ELEMS), AMR_THREADS, 0, st>>>(n, map, Uold, ops, Unew);
  return cudaGetLastError();
}

cudaError_t launch_partition(cudaStream_t st, int64_t n_elem, int64_t n_if, int64_t n_mort, const int32_t* level,
                             const int4* if_raw, const int4* mort_raw, int R, int S, const int32_t* stage_minmem,
                             const int32_t* member, int n_members, int32_t* member_lmax, int32_t* method,
                             int32_t* elem_sorted, int4* if_sorted, int4* mort_sorted, int64_t* counts,
                             int32_t* level_minmax, int mort_flag_bits, const int64_t* d_nfaces) {
  if (mort_flag_bits < 1 || mort_flag_bits > 8) return cudaErrorInvalidValue;
  k_partition<<<1, PART_THREADS, 0, st>>>(n_elem, n_if, n_mort, level, if_raw, mort_raw, R, S, stage_minmem, member, n_members,
                                          member_lmax, method, elem_sorted, if_sorted, mort_sorted, counts,
                                          level_minmax, mort_flag_bits, d_nfaces);
  return cudaGetLastError();
}

// per-member minimum of h_e / lambda_e: positive doubles order like their bit patterns; a node
// without an admissible state (rho <= 0, p <= 0, NaN or Inf) contributes the pattern 0 (+0.0),
// which the host reports as such
__global__ void __launch_bounds__(DT_THREADS) k_dt_members(int64_t n_nodes, const double* __restrict__ U,
                                                            const int32_t* __restrict__ level,
                                                            const int32_t* __restrict__ member, double length,
                                                            double gamma, unsigned long long* out) {
  for (int64_t q = (int64_t)blockIdx.x * DT_THREADS + threadIdx.x; q < n_nodes; q += (int64_t)gridDim.x * DT_THREADS) {
    const int64_t e = q / NODES;
    const int t = (int)(q - e * NODES);
    const double* u = U + e * ELEM + t;
    const double rho = u[0], ir = 1.0 / rho;
    const double v1 = u[NODES] * ir, v2 = u[2 * NODES] * ir;
    const double p = (gamma - 1.0) * (u[3 * NODES] - 0.5 * rho * (v1 * v1 + v2 * v2));
    const double lam = fabs(v1) + fabs(v2) + 2.0 * sqrt(gamma * p * ir);
    const double r = ldexp(length, -level[e]) / lam;
    const bool ok = rho > 0.0 && p > 0.0 && r > 0.0 && r < INFINITY;
    atomicMin(out + member[e], ok ? (unsigned long long)__double_as_longlong(r) : 0ull);
  }
}

__global__ void k_fill(double* p, int n, double v) {
  for (int q = threadIdx.x; q < n; q += blockDim.x) p[q] = v;
}

cudaError_t launch_dt_members(cudaStream_t st, int64_t n_elem, const double* U, const int32_t* level,
                              const int32_t* member, int n_members, double length, double gamma, double* out) {
  k_fill<<<1, 256, 0, st>>>(out, n_members, INFINITY);
  const int64_t nodes = n_elem * NODES;
  const unsigned blocks = (unsigned)std::min<int64_t>((int64_t)device_sm_count() * 8, (nodes + DT_THREADS - 1) / DT_THREADS);
  if (blocks > 0)
    k_dt_members<<<blocks, DT_THREADS, 0, st>>>(nodes, U, level, member, length, gamma,
                                                reinterpret_cast<unsigned long long*>(out));
  return cudaGetLastError();
}

cudaError_t launch_faces(cudaStream_t st, YSource ysrc, const Ops& ops, int64_t n_if, const int4* ifs, int64_t n_mort,
                         const int4* morts, const int32_t* method, const StageArgs& sa, double* surf) {
  const int64_t bi = (n_if + IF_PER_BLOCK - 1) / IF_PER_BLOCK;
  const int64_t bm = (n_mort + MORT_PER_BLOCK - 1) / MORT_PER_BLOCK;
  if (bi + bm == 0) return cudaSuccess;
  if (ysrc == Y_GIVEN)
    k_faces<Y_GIVEN><<<(unsigned)(bi + bm), FACE_THREADS, 0, st>>>(ops, n_if, ifs, n_mort, morts, bi, method, sa, surf);
  else
    k_faces<Y_COMBINE><<<(unsigned)(bi + bm), FACE_THREADS, 0, st>>>(ops, n_if, ifs, n_mort, morts, bi, method, sa,
                                                                     surf);
  return cudaGetLastError();
}

// blocks of k_stage the current device holds at once (occupancy x SMs), cached per device
int stage_resident_blocks() {
  constexpr int kMaxDevices = 64;
  static std::atomic<int> cache[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
  int n = cache[dev].load(std::memory_order_relaxed);
  if (n > 0) return n;
  int per_sm = 0, per_sm2 = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stage<false>, FACE_THREADS, 0) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, k_stage<true>, FACE_THREADS, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  n = std::min(per_sm, per_sm2) * device_sm_count();
  cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

cudaError_t launch_stage(cudaStream_t st, int stage, const Ops& ops, int64_t n_if, const int4* ifs, int64_t n_mort,
                         const int4* morts, int64_t n_el, const int32_t* elems, const int32_t* level,
                         const int32_t* method, double two_over_len, const StageArgs& sa, double* surf, double* K,
                         const UpdateArgs* check, const double* log_table, unsigned long long* ctl,
                         unsigned long long* stamps, int* err) {
  if (stage < 0 || stage >= MAX_S) return cudaErrorInvalidValue;
  if (ops.shock != PERK_SHOCK_OFF) return cudaErrorInvalidValue;
  const int64_t items = (n_if + IF_PER_BLOCK - 1) / IF_PER_BLOCK + (n_mort + MORT_PER_BLOCK - 1) / MORT_PER_BLOCK +
                        (n_el + STAGE_VE - 1) / STAGE_VE;
  if (items == 0) return cudaSuccess;
  UpdateArgs ua{};
  if (check) ua = *check;
  const StageSync sync{ctl, stamps, err, stage};
  const bool resident = items <= stage_resident_blocks();
  if (check)
    k_stage<true><<<(unsigned)items, FACE_THREADS, 0, st>>>(ops, n_if, ifs, n_mort, morts, n_el, elems, level, method,
                                                             two_over_len, sa, surf, K, ua, log_table, sync, resident);
  else
    k_stage<false><<<(unsigned)items, FACE_THREADS, 0, st>>>(ops, n_if, ifs, n_mort, morts, n_el, elems, level,
                                                              method, two_over_len, sa, surf, K, ua, log_table, sync,
                                                              resident);
  return cudaGetLastError();
}

// blocks of k_step: the resident capacity (computed once per device)
static int step_resident_blocks() {
  constexpr int kMaxDevices = 64;
  static std::atomic<int> cache[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
  int n = cache[dev].load(std::memory_order_relaxed);
  if (n > 0) return n;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step, FACE_THREADS, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  n = per_sm * device_sm_count();
  cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

cudaError_t launch_step(cudaStream_t st, const Ops& ops, const StepPlan& plan, const int4* ifs, const int4* morts,
                        const int32_t* elems, const int32_t* level, const int32_t* method, double two_over_len,
                        const StageArgs& sa, double* surf, const UpdateArgs& check, const double* log_table,
                        unsigned long long* ctl, unsigned long long* stamps, unsigned long long* prog, int* err) {
  if (plan.S < 1 || plan.S > STEP_MAX_S || ops.shock != PERK_SHOCK_OFF) return cudaErrorInvalidValue;
  const int64_t items = plan.first[plan.S];
  if (items <= 0) return cudaSuccess;
  const int64_t cap = step_resident_blocks();
  if (cap <= 0) return cudaErrorInvalidConfiguration;
  const StageSync sync{ctl, stamps, err, 0};
  k_step<<<(unsigned)std::min<int64_t>(cap, items), FACE_THREADS, 0, st>>>(
      ops, plan, ifs, morts, elems, level, method, two_over_len, sa, surf, check, log_table, sync, prog);
  return cudaGetLastError();
}

template <int VE, bool SHOCK>
static void volume_grid(YSource ysrc, bool check, cudaStream_t st, const Ops& ops, int64_t n, const int32_t* elems,
                        const int32_t* level, const int32_t* method, double two_over_len, const StageArgs& sa,
                        const double* surf, double* K, const UpdateArgs& ua, const double* log_table) {
  const unsigned blocks = (unsigned)((n + VE - 1) / VE);
  if (ysrc == Y_GIVEN)
    k_volume<Y_GIVEN, false, VE, SHOCK><<<blocks, VE * NODES, 0, st>>>(ops, n, elems, level, method, two_over_len,
                                                                       sa, surf, K, ua, log_table);
  else if (check)
    k_volume<Y_COMBINE, true, VE, SHOCK><<<blocks, VE * NODES, 0, st>>>(ops, n, elems, level, method, two_over_len,
                                                                        sa, surf, K, ua, log_table);
  else
    k_volume<Y_COMBINE, false, VE, SHOCK><<<blocks, VE * NODES, 0, st>>>(ops, n, elems, level, method,
                                                                         two_over_len, sa, surf, K, ua, log_table);
}

template <int VE>
static void volume_grid_any(YSource ysrc, bool check, cudaStream_t st, const Ops& ops, int64_t n,
                            const int32_t* elems, const int32_t* level, const int32_t* method, double two_over_len,
                            const StageArgs& sa, const double* surf, double* K, const UpdateArgs& ua,
                            const double* log_table) {
  if (ops.shock != PERK_SHOCK_OFF)
    volume_grid<VE, true>(ysrc, check, st, ops, n, elems, level, method, two_over_len, sa, surf, K, ua, log_table);
  else
    volume_grid<VE, false>(ysrc, check, st, ops, n, elems, level, method, two_over_len, sa, surf, K, ua, log_table);
}

cudaError_t launch_volume(cudaStream_t st, YSource ysrc, const Ops& ops, int64_t n, const int32_t* elems,
                          const int32_t* level, const int32_t* method, double two_over_len, const StageArgs& sa,
                          const double* surf, double* K, const UpdateArgs* check, const double* log_table,
                          int elems_per_block) {
  if (n == 0) return cudaSuccess;
  UpdateArgs ua{};
  if (check) ua = *check;
  switch (elems_per_block) {
    case 2:
      volume_grid_any<2>(ysrc, check != nullptr, st, ops, n, elems, level, method, two_over_len, sa, surf, K, ua,
                     log_table);
      break;
    case 4:
      volume_grid_any<4>(ysrc, check != nullptr, st, ops, n, elems, level, method, two_over_len, sa, surf, K, ua,
                     log_table);
      break;
    case 8:
      volume_grid_any<8>(ysrc, check != nullptr, st, ops, n, elems, level, method, two_over_len, sa, surf, K, ua,
                     log_table);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int device_sm_count() {
  constexpr int kMaxDevices = 64;
  static std::atomic<int> cache[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 1;
  int n = cache[dev].load(std::memory_order_relaxed);
  if (n > 0) return n;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    return 1;
  }
  cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

// Diagnostics: the volume kernel's logarithm and reciprocal on n inputs.
__global__ void k_selftest_math(int64_t n, const double* __restrict__ x, double* __restrict__ out,
                                const double* __restrict__ log_table) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  out[2 * q] = log_tab(x[q], log_table, log_table + LOG_TABLE);
  out[2 * q + 1] = rcp_nr(x[q]);
}

cudaError_t launch_selftest_math(cudaStream_t st, int64_t n, const double* x, double* out, const double* log_table) {
  if (n <= 0) return cudaSuccess;
  k_selftest_math<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x, out, log_table);
  return cudaGetLastError();
}

cudaError_t launch_commit(cudaStream_t st, int64_t n_elem, const UpdateArgs& ua, const double* Ks, const double* dt,
                          double* U) {
  const int64_t n2 = n_elem * ELEM / 2;
  if (n2 == 0) return cudaSuccess;
  int64_t blocks = (n2 + 255) / 256;
  const int64_t cap = (int64_t)device_sm_count() * 16;
  if (blocks > cap) blocks = cap;
  k_commit<<<(unsigned)blocks, 256, 0, st>>>(n2, ua, reinterpret_cast<const double2*>(Ks), dt,
                                             reinterpret_cast<double2*>(U));
  return cudaGetLastError();
}

cudaError_t launch_set_scalar(cudaStream_t st, double* p, double v) {
  k_set_scalar<<<1, 1, 0, st>>>(p, v);
  return cudaGetLastError();
}

cudaError_t launch_dt(cudaStream_t st, int64_t n_elem, const double* U, const int32_t* level, double length,
                      double gamma, double* block_min, int n_blocks, double* out) {
  k_dt_partial<<<n_blocks, DT_THREADS, 0, st>>>(n_elem * NODES, U, level, length, gamma, block_min);
  k_dt_final<<<1, 32, 0, st>>>(n_blocks, block_min, out);
  return cudaGetLastError();
}

}  // namespace perk
