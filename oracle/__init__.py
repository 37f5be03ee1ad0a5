"""Plain FP64 CPU oracle of the SBP-SAT anisotropic elastic wave scheme (Almquist & Dunham).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run anything
in this package.  The CUDA product path never calls it and shares no code with it
(the two meet only in the seeded input generators of ``workloads``).

The oracle assembles every operator of the paper as an explicit sparse matrix, built from
the 1-D operators by Kronecker products exactly as written in Sec. 4.3-4.7, and applies
the SATs of Sec. 5-6 term by term.  It is slow by design: no blocking, fusion or reordering.

Modules
-------
sbp1d   1-D diagonal-norm SBP operators H, D_x and the fully compatible D_xx^FC(b) (Sec. 4).
scheme  metric (Sec. 3.2-3.3), transformed stiffness, the discrete elastic operator
        (Sec. 4.6-4.7), boundary SATs (Sec. 5), interface SATs (Sec. 6), leapfrog and RK4
        time stepping, discrete energy, CFL time step (Sec. 7), Ricker wavelet and
        discrete delta point sources (Sec. 7.4).
scheme3d the same operator and boundary SATs in three dimensions on one curvilinear block
        (Sec. 3.3 with eq. surfj_app_3d, Sec. 4.3-4.7 and 5 for d = 3), leapfrog and energy.
adjoint discrete adjoint of the leapfrog scheme with explicit transposes, receiver misfit and its
        gradient with respect to density and stiffness (Sec. 5.2 remark, Theorems 3 and 5).

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py``.
"""
