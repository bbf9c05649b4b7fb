"""Plain FP64 CPU oracle for the Sakurai-Sugiura eigensolver with shifted CG.

TEST INFRASTRUCTURE ONLY.  This package is a slow, obviously-correct numpy
restatement of the method (complex128 throughout) that the CUDA path is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it;
the product library never calls it and shares no code with it (the only
common dependency is the seeded input generator module ``synthetic``).

Modules, each citing the passage of the paper it restates:

* ``wilson``    -- the Hermitian fermion matrix A = gamma5 (I - kappa D)
                   (Section 4) and the free-field closed form used to pin it;
* ``contour``   -- quadrature nodes and weights on the circle C (Section 2.1)
                   and on the line pair L+- (Section 3), the filter function
                   (Eq. 3);
* ``shifted_cg``-- the shifted CG method with a real seed shift
                   (Section 2.2, Eq. 5 and the residual collinearity);
* ``moments``   -- the quadrature moments s_hat_k (Eq. 2), block form;
* ``rayleigh_ritz`` -- Rayleigh-Ritz extraction (Section 2.1) and the
                   core-rectangle acceptance (Section 3);
* ``hankel``    -- the moment-based (Hankel pencil) extraction (Section 2.1),
                   used as an independent cross-check;
* ``ss``        -- the whole pipeline.

Parity status of every function is stated in its module header.
"""
