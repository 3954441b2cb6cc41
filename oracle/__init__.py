"""FP64 CPU oracle for the dynamic-formulation EMD misfit -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import anything from this package.  The product path (the CUDA library and its Python
binding) never imports, links or calls it, and this package imports nothing from the
product path: the two share no code.

Contents:

* ``emd_oracle`` -- the method as the paper states it, in float64 numpy, step by step:
  Mainini decomposition (Sec. 2.1), the discrete gradient / divergence (Sec. 2.2), the
  primal prox with ``shrink`` and the dual ascent (Eqs. of Sec. 2.2), and PDHG with
  linesearch (Algorithm 1).  Also the 1D closed form of W1 and the adjoint source.
* ``exact`` -- exact linear programs that pin the PDHG result on tiny grids: the
  Kantorovich transport LP with the anisotropic Manhattan cost and the min-cost flow
  on the grid graph (Sec. 2.1, Eqs. for K(mu, nu) and OT(mu, nu)), solved with
  ``scipy.optimize.linprog``.

* ``multigrid`` -- the two-grid strategy of Sec. 2.2 (closing paragraph) and Sec. 3.3:
  restriction of both gathers in time, a coarse Algorithm 1 solve, sinc interpolation
  of its solution onto the fine grid and a warm-started fine solve.

Parity status: every function is pinned by ``tests/test_oracle_pins.py`` and
``tests/test_oracle_mg_pins.py`` (closed forms,
library routines, exact LPs, invariants, hand-worked fixtures).  The fixed-iteration PDHG
trajectory has no closed form; it is pinned step by step (each step checked against the
defining minimisation / test of the paper) and at convergence by the LPs and the 1D
closed form.
"""
