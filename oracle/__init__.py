"""Plain, slow CPU FP64 oracle for the parallel orbital-updating (ParO) method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA library (no kernels, headers, tables or helpers); the two meet only on
the seeded inputs produced by ``paper_1405_0260_gb300.workloads``.

Module ``oracle.paro`` follows Dai, Gong, Zhou, Zhu, "A parallel
orbital-updating approach for electronic structure calculations":
  * Q1 finite elements on a uniform hexahedral mesh with homogeneous Dirichlet
    data (Section 2.1 spaces, Section 2.2 weak form eq. (2.6)-(2.7), Appendix
    bilinear form a(u, v)).
  * Step 3 of Algorithms 1.1 / 3.1 / A.1: N independent source problems, solved
    here with Jacobi-preconditioned CG on the shifted SPD system.
  * Step 4: the Rayleigh-Ritz projection onto span{u_i^(n+1/2)}.
  * Step 5: the loop, stopped on max |Delta lambda|.
Module ``oracle.ks`` adds the Kohn-Sham pieces of Section 2.2 (density,
Hartree by a Poisson solve, Slater exchange) for the SCF workload.
Module ``oracle.adapt`` holds the adaptive loop of Section 2.1 on tensor-product
meshes: residual error indicators per cell (Estimate), Doerfler and maximum
marking, eqs. (2.2)-(2.3) (Mark), bisection of the marked cells' axis intervals
(Refine) and the nested transfer of the orbitals.

Parity status per function is listed in each module header.
"""
