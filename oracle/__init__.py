"""CPU oracle for the BTTB/BCCB sensitivity products (FP64, numpy).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously-correct
reference the CUDA path is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg (and its
``--impl reference`` arm) may import it.  It shares no code with the CUDA library
and never imports the product package; the only code both sides use is the seeded
input module ``synth``, which holds no arithmetic of the method.

Modules:
  prism     -- prism kernels (gravity g_z, magnetic total-field anomaly), Sec. 2.1
  operator  -- dense G, FFT products and direct row sums, Sec. 2.1, Sec. 2.5, App. A
  irls      -- IRLS focusing inversion with GKB / RSVD solvers, Sec. 2.2-2.4, Alg. 1-2

Every function cites the passage it follows; pins live in ``tests/test_oracle_*.py``.
"""
