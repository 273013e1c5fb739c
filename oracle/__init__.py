"""Plain CPU FP64 oracle for the Closest Point Method multigrid solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) may import, call, link or execute anything in this
package.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

The oracle is written from Chen & Macdonald, "The Closest Point Method and
multigrid solvers for elliptic equations on surfaces" (arXiv 1307.4354):

* ``geometry``  closest-point functions cp(x) (Sec. 2.1) for circle, sphere,
  torus (Sec. 4.5.4) and ellipsoid (Newton on the secular equation).
* ``band``      the computational band on a uniform grid (Sec. 3.1, Fig. 3.1,
  Table 4.1), the ghost ring of Laplacian neighbours, stencil bases.
* ``interp``    tensor-product barycentric Lagrange interpolation E_p
  (Sec. 3.1, Eq. 3.1-3.2), assembled as a sparse matrix.
* ``operators`` the discrete Laplacian L, the operator M in the
  Macdonald-Brandman-Ruuth form (Eq. 2.10, Remark 3.2) and in the paper's form
  (Eq. 3.3), A = cI - M, the shifted Laplacian cI - L (Sec. 4.2).
* ``multigrid`` closest-point restriction/prolongation (Sec. 4.3), Jacobi
  smoothers (Eq. 4.1, Eq. 4.2, Sec. 4.4), the V-cycle (Algorithm 4.1) and the
  outer defect-correction loop.
* ``mlp``       the per-point network of the learned smoother in FP64
  (forward, analytic backward) -- no counterpart in the paper.

Everything is plain numpy / scipy.sparse in float64, no blocking, fusion or
reordering beyond the definitions.  Parity-unpinned parts are listed in the
module headers.
"""
