"""CPU FP64 oracle for the divergence-free VEM Stokes discretization and its
BDDC-preconditioned CG solve (Bevilacqua, Dassi, Zampini, Scacchi,
"BDDC preconditioners for virtual element approximations of the
three-dimensional Stokes equations").

TEST INFRASTRUCTURE ONLY.  Plain NumPy/SciPy, written for readability, not
speed.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it.  It shares no code with the CUDA library;
both read their inputs from the ``synth`` package.

Modules
-------
poly    scaled monomials, polynomial algebra, quadrature rules
vem     DOFs (Sec. 3, D1-D5), face/element projectors, local matrices
        A_K (Eq. discreteA), B_K, load (Eq. discreteF), global assembly and
        the bordered direct solve of the saddle system (Eq. MatrixForm);
        the reduced scheme (the remark after the convergence theorem)
bddc    interface classification, primal constraints (Sec. 5.1), change of
        basis, deluxe scaling on faces (Sec. 6) and optionally on edges,
        the adaptive coarse space (Sec. 6), BDDC apply (Eq. BDDCprec), PCG
        and the Lanczos condition-number estimate
"""
