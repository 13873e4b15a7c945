"""Plain, slow FP64 CPU oracle of randomized Krylov-Schur (rKS) with deflation.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call, link
or execute anything in this package: only the tests, the smoke check in
``__graft_entry__`` and the benchmark's CPU-baseline leg use it.  It shares no
code with the CUDA library (no kernels, headers, helpers or constants); the two
meet only through the seeded inputs of ``paper_2508_05400_gb300.inputs``.

Modules:
  sketch  - the sparse-sign embedding Omega from its hash specification.
  rks     - Algorithm 1 (rKS) and Algorithm 2 (extension) with the locking of
            Sec. 4.2-4.3, residual estimates of Sec. 4.1, whitening of Sec. 3.3.
  sketch_qr - the randomized QR factorisations of a block listed in Sec. 2
            (randomized Gram-Schmidt, sketch and whiten, randomized
            Cholesky QR).

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py``
(closed forms, brute force, invariants, published generator outputs); none is
"parity unpinned" except the eigenvalues of the non-symmetric Toeplitz matrix at
n = 2000, whose eigenvalue condition number (~1e261) makes them undefined in
floating point (only residuals are pinned there).
"""
