"""FP64 CPU oracle for the Taylor-expansion FMM in layered media (arXiv 1902.05875).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) imports, links or executes anything in this package.  Only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` may use it.

The oracle is a plain, slow, readable restatement of the paper:

* ``medium``      -- layered medium, the k_z branch, the interface problem for
                     the densities sigma (Sec. 2, Appendix A);
* ``sommerfeld``  -- contour quadrature of Sommerfeld integrals and their
                     derivatives (Sec. 2, eqs. for u^up/u^down, Sec. 3.3);
* ``dcim``        -- two-level DCIM sampling and GPOF fits (Sec. 3.3, Steps 1-3);
* ``derivs``      -- the Cartesian recurrence for D^k e^{ikR}/R at complex R
                     (Sec. 3.3, eq. ``recurrsion``, corrected form);
* ``direct``      -- FP64 direct sum of the DCIM-approximated layered Green's
                     function (Sec. 3.2, eq. ``totalinteraction``), in C;
* ``cross``       -- cross-layer components and their image fits (Sec. 3.3);
* ``alg2``        -- Algorithm 2's tables of Sommerfeld integrals on a grid,
                     interpolated and assembled into Cartesian derivatives
                     (Sec. 4.2, eqs. ``sysdifferential``, ``symmetricdetable``);
* ``tefmm``       -- the CPU TE-FMM (Algorithm 1 and the component loop of
                     Sec. 3, with Algorithm 2's tables as an option).

It shares no code with the CUDA path.
"""
