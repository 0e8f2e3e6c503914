"""Plain, slow FP64 CPU oracle of the LOR-preconditioned solver.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library (no kernels, headers, tables or helpers); both sides
receive their inputs from ``paper_1908_07071_gb300.synthetic``, which holds no
solver arithmetic.

Modules (each function cites the passage of the paper it follows):
  basis   -- GLL / Gauss-Legendre rules and Lagrange bases (Sections 2, 3.1)
  mesh    -- multilinear and isoparametric (curved) element maps (Sections 2, 5.2)
  cg      -- Q_p stiffness by dense quadrature, load vector (Eq. (fem), (system))
  lor     -- K_h, element-structured hierarchy, ordered ILU(0), vertex patches,
             coarse space, additive Schwarz B (Sections 3.1-3.4, Eq. (as), (patch))
  dg      -- interior-penalty and BR2 forms, B_DG (Eq. (ip), (br2), (dg-as))
  krylov  -- PCG / flexible CG and the Lanczos condition estimate
  learned -- FP64 reference of the per-patch convolutional smoother and its
             gradients (the learned form)
  ordering     -- MDF and RCM orderings for ILU(0) (Section 3.4)
  single_patch -- B(1): the whole domain as one patch (Section 4.1)
  unstructured -- vertex patches on unstructured quadrilateral meshes (Section 4.2)

Parity status: every function is pinned by a `-m "not gpu"` test against
closed forms, textbook special cases or invariants, except where a module
header says "parity unpinned".
"""
