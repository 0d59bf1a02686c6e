"""Plain FP64 CPU oracle for the periodized Stokes boundary-integral apply.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library (``paper_1912_04501_gb300``) never imports it,
and it imports nothing from the product.  The two share no code; the only
module both sides read is ``paper_1912_04501_gb300.workloads``, which draws
seeded body descriptions and holds none of the method's arithmetic.

Everything here is written from Wang, Nazockdast & Barnett, "An integral
equation method for the simulation of doubly-periodic suspensions of rigid
bodies in a shearing viscous flow" (arXiv 1912.04501), in numpy float64, as
slow and as literal as the paper's definitions allow:

* ``geometry``  -- trapezoidal boundary quadrature (Sec. 6), lattice (Sec. 7).
* ``kernels``   -- Stokeslet, pressure and traction kernels (Eqs. Gv, Gp, Gt).
* ``periodic``  -- near image sum, wall discrepancy, MFS proxy fit and the
                   periodizing correction (Sec. 4.2, Sec. 6.1, Sec. 6.2).
* ``close``     -- close-evaluation correction (Sec. 6.3), by its definition:
                   the exact integral of the trigonometric interpolant.
* ``barycentric`` -- the same integral by the paper's special quadrature
                   (Sec. 6.3): compensated barycentric rules for the Cauchy
                   integrals the single-layer traction reduces to.
* ``bie``       -- the Nystrom operator with rigid completion and pressure
                   fix (Eq. BIEdiscretized, Sec. 5, Sec. 6.2 remark), GMRES,
                   velocity extraction, effective viscosity and forward Euler
                   (Sec. 3, Sec. 7); the same operator with the paper's own
                   per-node doubled-cell periodizer (Def. Gnear) and its
                   contour-deformation effective viscosity (Sec. 6.4), as
                   cross-checks of the 3 x 3 image reading.
* ``mlp``       -- the warm-start network (no counterpart in the paper): a
                   per-node perceptron, its loss gradient and Adam, from their
                   definitions.

Pins against values fixed by the paper and by the mathematics live in
``tests/test_oracle_*.py``.
"""
