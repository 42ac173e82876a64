"""FP64 CPU oracle for the hybrid DM-baryon interaction step of Hainje & Farrar.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code, tables or constants with the CUDA path
under ``paper_2603_24688_gb300/``; the only module both sides use is the seeded
input generator ``paper_2603_24688_gb300.workloads``, which holds none of the
method's arithmetic.

Every function here is a plain, slow restatement of the paper's equations in
float64 (numpy), written for checking by eye against the paper:

  kernel.py     cubic-spline kernel (Sec. 2.4) and the overlap integral g_ij
                (Eq. dm-update-prob, App. D)
  hyp1f1.py     confluent hypergeometric 1F1(a, b; -x) (Sec. 2.4, DLMF 13.2.39 and
                13.7.2)
  rates.py      momentum/energy transfer integrals A, B (Eqs. scrA, scrB) and
                their power-law closed forms (App. B); the Maxwellian-averaged
                total rate R; a 1D quadrature for general cross sections
  philox.py     Philox4x32-10 counter-based generator (Salmon et al., SC'11)
  pairs.py      DM-gas pair set {(i, j): d_ij < h_i + h_j} by brute force and by a
                plain cell list (Sec. 2.4, App. D)
  meanfield.py  gas acceleration and heating (Eqs. gas-dVdt, gas-dTdt)
  mc.py         DM Monte Carlo update (Eqs. dm-update-vels, dm-update-prob,
                scatter_chi, prob_criterion)
  expect.py     expected DM transfers and the pairwise conservation identities
                (App. C)
  step.py       one interaction step with kicks and FP64 conservation sums
  units.py      physical constants and the code-unit system (kpc, km/s, Msun)

Parity status of each function is stated in its module docstring.
"""
