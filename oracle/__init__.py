"""Plain FP64 CPU oracle for the TVD/PAQIF elastohydrodynamic-lubrication hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` use it.  It shares no code with
the CUDA library (no kernels, headers, tables or helpers) and never imports it.

Modules
-------
paqif_ref     banded (projected) solves: dense LU, projected Gauss-Seidel,
              brute-force active-set enumeration (Sec. 2.1-2.2, Sec. 3.2).
aqif_ref      the AQIF factorization L0 = W0 Z0, its two sweeps and the
              partitioned method's Steps 1-7 on dense matrices (Sec. 2.2.1-2.2.4).
kernels_ref   closed-form deformation kernels for piecewise-constant pressure
              (Sec. 3.3.1, line and point contact).
material_ref  Moes parameter conversion, Roelands viscosity, Dowson-Higginson
              density, the diffusive coefficient eps (Sec. 3.3, Appendix A).
line_ref      line-contact film thickness, TVD-limited Reynolds residual, its
              exact Jacobian, the band Jacobian of the limiter-based
              Newton-Raphson method, and an independent dense semismooth
              Newton solve of the discrete complementarity problem with force
              balance (Sec. 3.3.1-3.3.4).
point_ref     the same for point contact (Sec. 3.3, Example 5).
adjoint_ref   dense adjoint of the converged line-contact state.

cd_ref        the linear convection-diffusion workload of the line splittings:
              van Leer's kappa-scheme, the Ls0 / Ls1 x-line relaxation (Sec. 3.1, Sec. 6).

Every floating-point computation is float64.  Each function cites the passage
of the paper it restates.  Functions whose result is not pinned by anything
outside the oracle say "parity unpinned" in their docstring.
"""
