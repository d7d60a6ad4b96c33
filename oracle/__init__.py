"""Plain, slow, CPU-only FP64 oracle for two-site ab initio DMRG.

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import this package. The
product library (paper_2103_09976_gb300) never imports it, and this package
never imports the product; the two share nothing but the seeded input
generators in synth/.

Modules:
  splitmix  counter-based SplitMix64 generator + Box-Muller normals
  fock      Fock-space operators, the ab initio Hamiltonian (Eq. qc-hamil), FCI
  blocks    quantum-number bases and block-sparse operators
  nc        U(1)xU(1) normal/complementary (NC) left-right decomposition
            (spin-orbital form of Eq. h-nc and Eq. op-def), site operators,
            blocking (Eq. blocked-ops) and transformation (Eq. op-trans)
  cn        complementary/normal (CN) partition (Eq. h-cn), CN blocking, the
            normal-to-complementary transformation and the mixed NC/CN
            scheme (Sec. III.A)
  sigma     H_eff . psi as a sum over NC terms of block-sparse O_L psi O_R^T
            products (Sec. II.D-E); synthetic middle-bond operator layout
  davidson  plain Davidson eigensolver (Appendix A, solving step)
  dmrg      plain two-site DMRG sweeps (Appendix A)

Every function is FP64. Parity status per function is listed in the module
headers; all functions here are pinned by tests in tests/test_oracle_*.py.
"""
