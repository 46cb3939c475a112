"""FP64 CPU oracle for the Parareal / ALE-FSI hot path.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or
execute this package: it is used by `tests/`, by the smoke check in
`__graft_entry__.py` and by the CPU-baseline leg of `bench.py`. It shares no
code with the CUDA library; the only common inputs come from the seeded
workload module, which holds no arithmetic of the method.

Parity status (what pins each part lives in tests/test_oracle_*.py):
  * Q2 element, quadrature ............ pinned (partition of unity, exactness)
  * ALE kinematics F, J, F^{-1} ........ pinned (identity map, stretch, translation)
  * fluid residual ..................... pinned (plain NS at u = 0, Poiseuille,
                                          affine divergence-free field,
                                          manufactured-solution rates h^3 / h^2
                                          in the Navier-Stokes limit, also on a
                                          moved ALE mesh)
  * stabilisation weight ............... pinned (every row scales by its own
                                          power of the units under a change of
                                          units; a weight with h for h^2 or
                                          without rho_f breaks it)
  * mass terms ......................... pinned (each material's density, with
                                          rho_s != rho_f)
  * solid residual ..................... pinned (homogeneous StVK patch test,
                                          rigid motion)
  * Jacobian ........................... pinned (central finite differences)
  * theta time step .................... pinned (second-order rate)
  * Newton ............................. pinned (quadratic decay)
  * discrete adjoint (adjoint.py) ...... pinned (old-state Jacobian and the
                                          gradient against central differences)
  * Parareal ........................... pinned (Dahlquist closed form,
                                          k = N reproduces the serial run)
  * speedup model ...................... pinned (value printed in Sec. 4.1)
  * d-dimensional step (fsi_nd.py) ...... pinned: at d = 2 equal to fsi.py; at
                                          d = 3 extrusion to 2D rows, y-z exchange
                                          symmetry, helpers vs numpy, affine
                                          divergence-free field, rigid solid
                                          motion, Q1 kernel of the stabilisation,
                                          inflow mean, finite differences, Newton
  * full FSI trajectory ................ parity unpinned: the paper prints no
                                          numbers for these workloads, so GPU vs
                                          oracle agreement is self-consistency.
"""
