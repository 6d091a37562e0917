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
  euler     2D Euler fluxes: physical, entropy-conservative two-point, HLL, HLLC, HLLE
  treemesh  geometric face matching on a periodic quadtree leaf list
  dgsem     full DGSEM right-hand side F(U) and the masked partitioned RHS
  perk      P-ERK2 / P-ERK3 coefficient construction and the dense partitioned-RK step
  godunov   1D upwind finite-volume model problem of the paper's Sec. 3.2
  amr       quadtree AMR: indicators, balance, new leaves, exact transfer
  br1       BR1 viscous terms of the 2D Navier-Stokes equations
  shock     subcell shock capturing (blended volume term)
  spectrum  spectrum-optimised stability polynomials
  autodiff  torch transcription of the RHS and step for derivative checks
  euler3d, octree, dgsem3d, amr3d, br1_3d
            the same for the 3D octree case of the paper's Sec. 7.1.3 (Taylor-Green vortex)
"""
