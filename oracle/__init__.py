"""Oracle for phi_l(-tau*A) v with A a Kronecker sum -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, obviously-correct CPU float64 statement of what the
GPU library computes.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
product path (the ``paper_2211_00696_gb300`` package and its CUDA library) never
imports or calls anything here, and nothing here imports the product path: the two
share no code.  Inputs come from the standalone ``workloads`` module.

Contents (paper: Croci & Munoz-Matute, "Exploiting Kronecker structure in exponential
integrators", arXiv 2211.00696):

* ``phi``        -- the plain definition of phi_l (Sec. 2.1, Eq. (3)) evaluated four
                    independent ways: O1 dense augmented-matrix exponential, O2 spectral
                    (sine / Fourier transforms, symmetric operators only), O3 sparse
                    augmented action (scipy's expm_multiply), O4 mpmath at 50 digits.
* ``planner``    -- Algorithms 3 (quaderr), 4 (quadnodes) and 5 (setup_quadrature) of
                    Sec. 3.2-3.3, the Theorem 3.2 / Corollary 3.3 bounds, and the
                    Gauss-Legendre / Clenshaw-Curtis rules on [0, 1].
* ``quadrature`` -- Algorithms 1 and 6 (fixed quadrature + scaling and modified
                    squaring) restated step by step with library matrix exponentials;
                    used to check the reading of the paper and intermediate results.
* ``selector``   -- the measured error criterion, the cost-minimising (s, m) search that
                    labels the learned selector's training data, and a float64 statement
                    of the selector network with its analytic gradients.
* ``erk``        -- exponential Euler and Runge-Kutta steps (Eq. (RK), Table RK), every
                    tableau entry applied as its own phi-action supplied by the caller.

Parity status: every function here is pinned by tests under ``tests/`` against
closed forms, invariants, the paper's tables or brute force (see each docstring).
"""
