// Device helpers shared by the 3D kernels (perk3d_kernels.cu, perk3d_br1.cu): element geometry
// constants, the face-node map and the stage state formed on the fly.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "perk3d_internal.h"

namespace perk3 {

template <int NN>
struct G {
  static constexpr int FN = NN * NN;            // nodes per face
  static constexpr int NODES = NN * NN * NN;    // nodes per element
  static constexpr int ELEM = NV3 * NODES;      // doubles per element
  static constexpr int SURF = 6 * NV3 * FN;     // face-data doubles per element: [face][var][face node]
  static constexpr int NPL = NN * (NN - 1) / 2; // symmetric pairs per grid line
  static constexpr int NP = 3 * FN * NPL;       // symmetric pairs per element
  static constexpr int F = 15 * NODES;          // BR1 viscous fluxes per element: [axis][var][node]
};

// Volume node of face node q (t1 = q % NN, t2 = q / NN along the face's tangential axes t1 < t2)
// on face f: 0/1 = -x/+x, 2/3 = -y/+y, 4/5 = -z/+z.  Volume node = (k NN + j) NN + i.
template <int NN>
__device__ __forceinline__ int face_node3(int f, int q) {
  const int t1 = q % NN, t2 = q / NN, b = (f & 1) ? NN - 1 : 0;
  const int d = f >> 1;
  return d == 0 ? (t2 * NN + t1) * NN + b : d == 1 ? (t2 * NN + b) * NN + t1 : (b * NN + t2) * NN + t1;
}

// the stage state at one node of element e (member m): given, or U + dt (alpha K_1 + beta K_{i-1})
template <int NN, int YS>
__device__ __forceinline__ void stage_state3(const StageArgs& sa, int64_t e, int m, int node, double y[5]) {
  const int64_t base = e * G<NN>::ELEM + node;
  constexpr int ND = G<NN>::NODES;
  if (YS == perk::Y_GIVEN) {
#pragma unroll
    for (int v = 0; v < 5; ++v) y[v] = __ldg(sa.Y + base + v * ND);
  } else {
    const StageCoef c = sa.coef[m];
    const double dt = sa.dt[0];
#pragma unroll
    for (int v = 0; v < 5; ++v) y[v] = __ldg(sa.U + base + v * ND);
    if (__double_as_longlong(c.alpha) != 0) {   // integer test, off the FP64 pipe
      const double da = dt * c.alpha;
#pragma unroll
      for (int v = 0; v < 5; ++v) y[v] = fma(da, __ldg(sa.K1 + base + v * ND), y[v]);
    }
    if (__double_as_longlong(c.beta) != 0) {
      const double db = dt * c.beta;
#pragma unroll
      for (int v = 0; v < 5; ++v) y[v] = fma(db, __ldg(sa.Kp + base + v * ND), y[v]);
    }
  }
}

}  // namespace perk3
