"""CPU oracle for the TRPL+K eigensolver -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 restatement of the method of Wu, Xue and Stathopoulos,
"TRPL+K: Thick-Restart Preconditioned Lanczos+K Method for Large Symmetric
Eigenvalue Problems" (arXiv 1711.10128), written to be checked against the
paper by eye.  It exists to prove the CUDA path right; it is never part of
the product.  Only the test suite, the smoke check and the CPU-baseline leg of
the benchmark may import it.  It shares no code with the CUDA path; from the
product package it uses only the seeded input generators
(``paper_1711_10128_gb300.workloads``, which hold none of the method's
arithmetic), to build the full-size operators of ``reference_runs``.

Modules
-------
``trplk``  Algorithm 1 (with the generalized-pencil reading), its steps as
           separate functions, and the final FP64 residual check.
``dense``  a textbook cyclic Jacobi eigensolver for small symmetric matrices
           (the brute-force check for tiny problems).
``fsai``   factorised sparse approximate inverse preconditioners (classical
           and MLP-predicted) with the training loss and its gradient.
``reference_runs``  runs ``trplk.solve`` to convergence on the full-size
           operators and stores eigenvalues, residuals and cycle counts
           (``reference_runs.json``) for the full-size parity tests and the
           CPU baseline's extrapolation.

Parity status of each function is stated in its docstring; every function is
pinned by a ``-m "not gpu"`` test against closed forms, brute force or
invariants fixed by the paper and the mathematics.
"""
