"""FP64 CPU oracle for the Hermite half step of the 3-D scalar wave equation.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the package
``paper_1609_09841_gb300`` and its CUDA library) imports, links or runs this
package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA path.

The oracle follows the paper (Vargas, Chan, Hagstrom, Warburton, "GPU
Acceleration of Hermite Methods for the Simulation of Wave Propagation",
arXiv:1609.09841) step by step:

* Eq. 2   -- scaled-derivative degrees of freedom at each node;
* Eq. 3   -- the cell polynomial in scaled coordinates, coefficients = the
             scaled derivatives at the cell centre;
* Alg. 1/2 -- tensor Hermite interpolation, H applied along x1, then x2, x3;
* Alg. 3  -- differentiation of the coefficients (applied twice for the
             Laplacian of the wave equation);
* Alg. 4 / Eq. 4 -- local evolution over half a time step (classical RK4,
             identical to a q = 4 Taylor series for this linear problem);
* Sec. 2  -- truncation to the dual-node data and alternation of grids.

Modules: ``hermite`` (the half step, its adjoint, norms, energy),
``exact`` (closed-form solutions sampled as scaled derivatives) and
``symbol`` (Fourier symbol and stability limit of the half step).

Parity status: every function is pinned by ``tests/test_oracle_*.py``.
``hermite.energy`` (the paper defines no energy; this one is the wave
equation's quadratic invariant on the interpolants) is pinned by quadrature
of an independently built interpolant and by a closed form.
"""
