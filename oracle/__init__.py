"""Oracle: a plain, slow, FP64 CPU restatement of the low-rank Fourier–Galerkin method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import anything under ``oracle/``.  The product library
(``paper_1902_07455_gb300``) never imports it, and this package never imports the product.  The two share
no code; only the seeded input generators in ``synthetic/`` serve both.

Modules
-------
``fourier_galerkin``  full-format GaNi discretisation (Sec. 2.2.1, 2.2.2, 2.3): DFT matrices, Fourier
                      gradient/divergence, Laplacian preconditioner, PCG, homogenised coefficient.
``lowrank``           CP (d=2), Tucker and tensor-train formats (Sec. 3.1, App. A): Hadamard products, sums,
                      mode-wise DFT, rank truncation, the truncated operator of Eq. (Pls_lowrank) and the
                      minimal-residual iteration of Sec. 3.3.
``expsum``            exponential-sum approximation of 1/x used to give the preconditioner a low-rank form
                      (the paper states that preconditioning is an element-wise product that raises the
                      rank, Sec. 3.2, Table "operations", but does not say how the inverse Laplacian is put
                      in low-rank form; we use sinc quadrature of 1/x = int_0^inf exp(-t x) dt).

Every function cites the section or equation of arXiv:1902.07455 it restates.  Floating point is FP64
(complex128 in Fourier space) throughout.
"""
