"""GB300-native randomized Krylov-Schur (rKS) eigensolver with deflation.

``paper_2508_05400_gb300.rks`` is the Python binding of the C-ABI library
``librks.so`` (CUDA kernels for sm_103a); ``paper_2508_05400_gb300.inputs``
holds the seeded synthetic operators and start vectors.  Importing this package
loads nothing: the library is loaded on first use of the binding.
"""
