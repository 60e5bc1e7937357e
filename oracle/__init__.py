"""FP64 CPU oracle for the domain wall fermion multigrid hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package may import, call or
execute anything in this directory; only tests/, the smoke check in
__graft_entry__ and the CPU baseline leg of bench.py use it.

The oracle is a plain, slow, deliberately unoptimised restatement of the
operators and algorithms of Boyle & Yamaguchi, "Comparison of Domain Wall
Fermion Multigrid Methods" (arXiv:2103.05034), in numpy complex128.  It shares
no code with the CUDA path; the only common module is `synth` (seeded inputs).

Modules:
  dwf     Section 2, Eqs. (1)-(5): D_W, D_hop, D_DW, D_par, Gamma_5, H_DW;
          red-black Schur complement M_ee - M_eo M_oo^-1 M_oe (Section 5.1)
  krylov  CG on the normal equations, red-black CGNR (Section 5.1, Table 5),
          power method (Section 3.4)
  cheby   Chebyshev polynomials, smoother and filters (Sections 3.2, 3.4)
  coarse  blocking, chirality projection, little Dirac operator (Sections 3.1,
          3.4)
  mg      composite V(1,1) preconditioner (Section 3.3) and flexible GCR
  hybrid  the three-level hybrid multigrid (Algorithm F, Section 4): 4D D_W
          coarsening, the coarse domain wall operator, H_DW coarsening of
          the coarse space, fixed-iteration W-cycle
  force   pseudofermion action and its gauge-link derivative (HMC context,
          Section 6; derived from first principles)
"""
