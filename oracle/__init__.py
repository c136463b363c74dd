"""CPU FP64 oracle for the Zolo-csd hot path (test infrastructure only).

This package is the independent reference the CUDA path is checked against.
It shares no code with the product library and is imported only by the test
suite, by ``__graft_entry__.smoke()`` and by the CPU-baseline leg of
``bench.py``; nothing on the product path may import or call it.

Contents
--------
jacobi   ctypes front end of the plain-C one-sided Jacobi SVD and cyclic
         Jacobi eigensolver (jacobi.c).
csd      Algorithm 1 (with the rank-deficient variant, Algorithm 3) written
         out step by step with Jacobi sub-solvers in place of Zolo-pd/Zolo-eig.
zolo     Zolotarev rational functions (Section 5) from mpmath's Jacobi
         elliptic functions; expected Zolo-pd iterates U r_k(Sigma) V^*.
metrics  backward error, orthogonality, distance to partial isometries d(A).
"""
