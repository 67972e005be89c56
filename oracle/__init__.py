"""CPU FP64 oracle for the BF + HSS-ULV approximate FIO inverse.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
benchmark's CPU-baseline leg may import it.  It shares no code with the CUDA
library and never consumes anything the CUDA path produced.

Modules:
  problem    grids, phase functions, dense K (Eq. 1.1-1.2)
  butterfly  BF factors from their definitions and their products (Section 2.2, Eq. 2.1)
  hss        HSS generators, telescoping (Eq. 2.7-2.8), black-box construction
             (Section 3), ULV factorization and solve (Section 2.4)
  philox     counter-based Gaussian test matrices (Philox4x32-10 + Box-Muller)
  solver     Algorithm 1 / Eq. 4.2: f^ = F~ K~^* u

Parity status: every function above is pinned by tests/test_oracle_*.py
(DFT closed form, dense K, adjoint identity, interpolation invariants,
Def. 2.2 vs Eq. 2.8, exact HSS recovery, dense solves, dense LU of K).
"""
