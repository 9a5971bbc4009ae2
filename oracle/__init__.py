"""CPU oracle for periodic spin-orbital CCSD (test infrastructure only).

A plain, slow, complex128 implementation of what the GPU library computes,
written from the paper's equations.  Only the tests, the package smoke check
and the CPU-baseline leg of the benchmark may import it; the library itself
never calls into it, and the two share no code.

Modules
  kmesh       momentum arithmetic on the k grid (Sec. 3.2.5)
  integrals   access to any <pq||rs> class through the symmetries (Sec. 3.3)
  ccsd_k      form A: the original T1/T2 equations and intermediates (Sec. 2)
  ccsd_k_rearranged  form B: the rearranged equations (Sec. 3.3.1-3.3.4)
  ccsd_k_block  form A at chosen momentum blocks, for grids where the full form A
              does not fit the host
  process_grid  the paper's N_k^2 distributed schedule on host ranks (Sec. 3.2,
              Table 1, Sec. 4.3-4.4), threads or gloo processes
  molecular   k-free spin-orbital CCSD on dense tensors (N_k = 1 / supercell)
  fci         two-electron full CI (exactness pin)
  driver      t0 = f(0), Jacobi update t + R/D, convergence test (Sec. 4.4),
              DIIS, correlation energy

Every hot-path function is pinned by a test that does not reuse it (MP2
closed form, two-electron FCI, molecular limit, supercell unfolding in two
bases, form A = form B, symmetry invariants); none is parity-unpinned.
"""
