"""Oracle for the matrix-free isogeometric Karhunen-Loeve operator (arXiv 2011.13861).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
CPU implementation in float64 (NumPy/SciPy) of what the GPU path computes.  It
exists to check the CUDA library and nothing else: only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  The product path (the C-ABI library and
its Python binding) never imports, calls or links anything here, and this
package imports nothing from the product package.

Modules
-------
bspline      univariate B-splines, Greville abscissae, Gauss-Legendre, the
             univariate matrices Z_k, M_k and the collocation matrix B~_k
             (Sec. 2.3, Sec. 3.5 eq. univariate_mass_matrix, Sec. 4.2
             eq. interpolation_matrix, Sec. 4.3 eq. univariate_mass_matrix2).
ibq          the interpolation-based-quadrature discretisation written out
             densely (Sec. 4.1-4.4.1), the generalized eigenproblem, and the
             matrix-free application of Algorithm 1 step by step.
kernels      the covariance kernels (Sec. 3.1; formulas fixed by the readings
             stated there).
galerkin     brute-force standard Galerkin with tensor Gauss quadrature on
             tiny meshes (Sec. 5.1) -- used to pin the IBQ exactness property.
closed_form  closed-form eigenvalues of the 1D exponential kernel
             (the analytic solution cited in the Remark of Sec. 6.1).

Every function is pinned by a ``-m "not gpu"`` test in ``tests/`` against
something other than itself (closed forms, textbook special cases,
invariants, brute force).  No function here is "parity unpinned".  Among them:

* kernels.kernel_matrix in d >= 2 (Sec. 3.1): kernel values at offsets of known
  Euclidean length (Pythagorean triples and quadruples) and the invariance of the
  exp and gauss spectra under a 30-degree rotation of the domain, which the
  separable kernel must not show
  (test_kernel_values_at_pythagorean_offsets, test_euclidean_kernels_are_rotation_invariant);
* mlp.forward / mlp.backward with the roundings off: the same network built from
  torch.nn Linear and Tanh layers in float64 and its autograd gradients
  (test_mlp_forward_and_backward_match_torch_nn); the bfloat16 rounding against
  torch's conversion, Adam against torch.optim.Adam.
"""
