"""Plain FP64 CPU oracle of the leap-frog scheme on unstructured triangle meshes.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline (and its ``--impl reference`` arm) may import anything from this package.  The
product path (the C-ABI library in ``paper_1812_01448_gb300``) never calls it, and this package
never imports the product path: the two share no code.

Written with numpy and scipy.sparse in float64, arrays in the caller's numbering, one
vectorised pass per operation, following the paper (Fadeev, "Numerical simulation of 2D
electrodynamic problems with unstructured triangular meshes"):

* ``mesh``       field placement and mesh symbols (Fig. 1, Fig. 2): edges, R(i)/L(i), A(j,q)
* ``geometry``   circumcentres O_j, midpoints C_i, |e_i|, S_j, |O_R O_L| (eqs. 3, 4, 7)
* ``operators``  L_B (eq. 3) and L_E (eq. 4) as sparse matrices, the metric of eq. 7
* ``leapfrog``   the time step (eqs. 5, 6, 14, 15), energies (eqs. 7, 8), div E flux
* ``spectral``   power iteration for rho(M) (Section 2, "complex time" method), stability
                 bound (eq. 20), dense eigenvalues for small meshes
* ``rcm``        locality reordering (motivated by the "Divide and conqueror" section)
* ``mlp``        the learned spectral-radius predictor's forward and backward passes

Parity status per function is stated in each module header.
"""
