"""Plain FP64 CPU oracle for the blocked fixed-precision farPCA loop.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) may import, link or execute anything in this package; only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` use it.  It shares no code with the CUDA path: the Philox
generator, the test-matrix kinds and the farPCA steps are written here a second
time, from the paper (arxiv 2506.03859) and from the Philox definition
(Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11).

Modules
  philox       Philox4x32-10, vectorised over numpy arrays.
  omega        the test matrices Omega of Def. 2.1-2.4 (and the Gaussian one),
               drawn from Philox counters.
  farpca       the QB-form farPCA loop (randQB_EI form, Sec. 2.1), the parity
               target of the CUDA path.
  farpca_paper the same loop written as Alg. 1 / Alg. 2 print it (Y, W, Z, T,
               eigSVD), used to cross-check ``farpca``.
  svd          the SVD the method returns (Alg. 1's last steps, QB form) and
               the post-processing truncation of Sec. 5.3.

Every function is pinned by a ``-m "not gpu"`` test; see the pins listed in
each module docstring.
"""
