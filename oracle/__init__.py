"""FP64 CPU oracle for the LO-AFQMC local-energy path.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, deliberately
unoptimised restatement of the quantities the paper defines (Weber et al.,
"A Localized-Orbital Energy Evaluation for Auxiliary-Field Quantum Monte
Carlo", arXiv 2202.00832).  It exists to check the CUDA library; it shares no
code with it, and the library never imports it.  Only the test suite, the
smoke check of ``__graft_entry__`` and the ``cpu_baseline`` leg of
``bench.py`` may import or run anything here.

Modules
  energy   local energy of single-determinant trials: overlap, LU, log-det,
           Theta (eq. Q), Green's function (eq. GwQ), the generalized Wick
           sum (eq. 2e_general) and its Cholesky form (eq. 2e_HRchol_RCAS)
  lo       Foster-Boys localization (Sec. 4), blockwise pair SVD with the
           single threshold T_SVD (Sec. 3.1.1) and the LO energy
           (eqs. 2e_HR_RCAS_LO / 2e_HR_RCAS)
  mlp      the pair-screening network (8 -> 64 -> 64 -> 1) that the
           conclusions' pair-screening idea (Sec. 5) motivates

Parity status: every function is pinned by a ``-m "not gpu"`` test against a
closed form, an invariance, brute force or a textbook library routine, except
where its docstring says "parity unpinned".
"""
