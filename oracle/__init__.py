"""Plain FP64 CPU oracle for the Jacobian-free Newton-Krylov multigrid method of
Kothari, Kopanicakova & Krause, "A Multigrid Preconditioner for Jacobian-free
Newton-Krylov Methods" (arXiv:2103.13890).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import anything from this package.  The
product path (``paper_2103_13890_gb300``) never imports it and shares no code
with it: the only thing both sides use is the seeded input generators in
``workloads``, which contain none of the method's arithmetic.

Every function is a direct, slow restatement of a definition in the paper
(section / equation / algorithm cited in its docstring) or of a reading of the
paper where it is silent.  Numpy array operations over all elements are used as
the vectorised form of "for every element"; nothing is blocked, fused or
reordered beyond what the cited definition states.

Modules
-------
fem       Q1 finite-element residuals F(u) for the three problems, the discrete
          Bratu energy, the manufactured load vector, the assembled analytic
          Jacobian and the vector-Jacobian products.
transfer  Prolongation I, restriction R = I^T and projection P = 2^-d I^T.
splitmix  The SplitMix64 counter-based generator (random power-method start).
jfnk      FD Jacobian action, Chebyshev smoother, power method, coarse GMRES,
          the V-cycle of Algorithm 1, FGMRES(m), line search and inexact Newton.
adjoint   Adjoint solve and gradient with respect to the coefficient field.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
against closed forms, invariants, brute force or independent formulations,
except where a function's docstring says "parity unpinned".
"""
