"""CPU oracle for the CPRAND / CPRAND-MIX hot path (FP64, NumPy).

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check in __graft_entry__ and the CPU-baseline
leg of bench.py may import this package.  The CUDA library neither imports nor links it, and the
oracle takes nothing from the library: the two share only the seeded input generator (synth/).

Modules
  philox     Philox4x32-10 (Salmon et al., SC'11)
  streams    which Philox draw feeds which random quantity of the method
  cp         §2.1 tensor algebra, CP-ALS (Alg. 1), SKR (Alg. 2), CPRAND (Alg. 3), stopping rules
  mixing     DCT-II mixing, CPRAND-MIX in its real form (Alg. 5)
  mixing_fft unitary-DFT mixing, CPRAND-MIX in its complex form (Alg. 4, real LS of eq. (rcLS))
  coherence  leverage scores and coherence (§2.2, §3.2.2)

Parity unpinned: nothing.  Every function is pinned by a test in tests/test_oracle_*.py against
a value the paper prints, a closed form, a library routine or brute force.
"""
