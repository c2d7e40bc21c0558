"""Reference oracle for the noisy-circuit simulator hot path.

TEST INFRASTRUCTURE ONLY.  A plain, slow, complex128 CPU restatement of what
Bogdanov et al. (arXiv:1412.2293) compute, written so that each step can be
checked against the paper by eye.  It shares no code with the CUDA path: the
only module both sides import is ``paper_1412_2293_gb300.inputs`` (seeded
workload descriptors, no simulation arithmetic).  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline and reference legs of
``bench.py`` may import it; the product path never does.

Modules
  philox      Philox4x32-10 and the Gaussian draw xi ~ N(0,1) of Eq. 1
  gates       gate matrices (Eqs. 1, 2, 4, 5, 7, 8), Kraus sets (Eqs. 3, 6, 9)
              and the paper's closed forms (Eqs. 10, 11, 15)
  statevec    amplitude update of Sec. 2 (k-qubit, explicit index groups)
  density     exact density matrix (Sec. 3, Eq. 3) and its vectorised form
  fixed_rank  fixed-rank approximation (Sec. 3.2) with the tie rule
  circuits    runs gate-descriptor lists in each representation
  choi        Choi-Jamiolkowski relative states (Sec. 4, Eqs. 16-17)
  relaxation  T1/T2 relaxation channels, the phase-error channel (Eq. 19),
              the three-qubit phase code and Shor's code (Sec. 4.1-4.2,
              Eq. 18)

Pinning (what fixes each function independently of itself) is listed in each
module's docstring; the pins are the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py``.  The one function without an independent pin is
the fixed-rank truncation for 1 < r < full rank when eigenvalues tie at the
cutoff: parity unpinned beyond monotonicity and the limiting cases.
"""
