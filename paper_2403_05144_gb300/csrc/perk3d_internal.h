// Internal declarations shared by the 3D host runtime (perk3d_host.cpp) and the
// 3D kernels (perk3d_kernels.cu).  Not part of the ABI.
#pragma once

#include "perk3d.h"
#include "perk_internal.h"

namespace perk3 {

using perk::StageArgs;
using perk::StageCoef;
using perk::UpdateArgs;
using perk::YSource;

constexpr int NV3 = 5;     // conserved variables
constexpr int MAXNN = 4;   // nodes per direction of the largest built degree (N = 3)
constexpr int MORT_FLAG_BITS = 3;   // mortar record .w: dir (2 bits) | large_side << 2 | member << 3

inline int64_t nodes3(int nn) { return (int64_t)nn * nn * nn; }
inline int64_t elem3(int nn) { return NV3 * nodes3(nn); }      // doubles per element
inline int64_t surf3(int nn) { return 6 * NV3 * nn * nn; }      // doubles of face fluxes per element

// Reference-element operators of degree nn - 1 (entries beyond nn unused).
struct Ops3 {
  int nn;
  double dsplit[MAXNN][MAXNN];   // 2 D_ij off the diagonal, 0 on it
  double dmat[MAXNN][MAXNN];     // the derivative matrix D_ij = l_j'(x_i)
  double inv_w0;                 // 1 / w_0 = 1 / w_N
  double p_lo[MAXNN][MAXNN];     // large-face trace -> lower half (interpolation, along one axis)
  double p_hi[MAXNN][MAXNN];
  double r_lo[MAXNN][MAXNN];     // lower half -> large face (exact L2 projection, along one axis)
  double r_hi[MAXNN][MAXNN];
  double gamma, gm1, inv_gm1;
  int surface_flux;
};

// Interfaces and mortars of the active prefixes in one launch.  ifs: (left, right, dir, member);
// morts: (large, s0, table index, dir | large_side << 2 | member << 3); msmall[table index] =
// the four small cells by quadrant q1 + 2 q2.
cudaError_t launch_faces3(cudaStream_t st, YSource ys, const Ops3& ops, int64_t n_if, const int4* ifs, int64_t n_mort,
                          const int4* morts, const int4* msmall, const int32_t* method, const StageArgs& sa,
                          const double* log_table, double* surf);
// Volume integral + surface lifting + Jacobian of the first n entries of elems; check: the
// admissibility test of the state the step would commit (last stage).
cudaError_t launch_volume3(cudaStream_t st, YSource ys, const Ops3& ops, int64_t n, const int32_t* elems,
                           const int32_t* level, const int32_t* method, double two_over_len, const StageArgs& sa,
                           const double* surf, double* K, const UpdateArgs* check, const double* log_table);
// U += dt (b1 K1 + bp Kp + bs Ks) over n_doubles entries unless *ua.flag is raised.
cudaError_t launch_commit3(cudaStream_t st, int64_t n_doubles, const UpdateArgs& ua, const double* Ks,
                           const double* dt, double* U);
// out[0] = min_e h_e / ((N+1) lambda_e) as a double (out is reset to +inf first).
cudaError_t launch_dt3(cudaStream_t st, int nn, int64_t n_elem, const double* U, const int32_t* level, double length,
                       double gamma, double* out);

// eta[e] = max over nodes of rho |curl v|^2 / 2 (the enstrophy indicator)
cudaError_t launch_enstrophy3(cudaStream_t st, const Ops3& ops, int64_t n_elem, const double* U,
                              const int32_t* level, double two_over_len, double* eta);
// AMR transfer: map[9 * q] = kind | cx << 2 | cy << 3 | cz << 4 (kind 0 copy, 1 refine, 2 coarsen),
// then the source cells (copy/refine: one; coarsen: the eight children by cx + 2 cy + 4 cz)
cudaError_t launch_transfer3(cudaStream_t st, const Ops3& ops, int64_t n_new, const int32_t* map, const double* Uold,
                             double* Unew);

// BR1 viscous terms of one stage (perk3d_br1.cu): face averages of w and gradients on the halo
// prefixes, viscous flux and divergence on the active prefixes; K += viscous part; surf (the
// inviscid face-flux buffer, free once the volume kernel has run) holds the face averages,
// q[e][axis][variable][node] the viscous fluxes (15 n^3 doubles per element); check:
// admissibility on the last stage
cudaError_t launch_br1_3d(cudaStream_t st, YSource ys, const Ops3& ops, double mu, double kappa, int64_t n_if_halo,
                          int64_t n_mort_halo, int64_t n_if_act, int64_t n_mort_act, const int4* ifs,
                          const int4* morts, const int4* msmall, int64_t n_el_halo, int64_t n_el_act,
                          const int32_t* elems, const int32_t* level, const int32_t* method, double two_over_len,
                          const StageArgs& sa, double* surf, double* q, double* K, const UpdateArgs* check);

}  // namespace perk3
