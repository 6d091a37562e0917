"""CPU oracle for the P-ERK / DGSEM hot path (test infrastructure only).

A plain, slow, float64 numpy implementation of what the CUDA library computes,
written from the paper (Doehring, Schlottke-Lakemper, Gassner, Torrilhon,
"Multirate Time-Integration based on Dynamic ODE Partitioning through
Adaptively Refined Meshes for Compressible Fluid Dynamics") and from the
textbook definitions it cites.  Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark may import it; the product path never does,
and it shares no code with the CUDA library.

Modules
  lgl       Legendre-Gauss-Lobatto nodes, weights, derivative and mortar operators
  euler     2D Euler fluxes: physical, entropy-conservative two-point, HLL, HLLC
  treemesh  geometric face matching on a periodic quadtree leaf list
  dgsem     full DGSEM right-hand side F(U) and the masked partitioned RHS
  perk      P-ERK2 coefficient construction and the dense partitioned-RK step
  godunov   1D upwind finite-volume model problem of the paper's Sec. 3.2
"""
