"""Plain FP64 CPU oracle of the spectral-multigrid Poisson solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
Python binding) imports, links or executes anything in this package.  Only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.

It is written directly from the paper (Mandal, Gressel, Ziegler & Mignone,
"A fast spectral-multigrid Poisson solver in non-Cartesian geometries"):

* ``geometry``  -- cell faces, volume-weighted centroids, volumes, face areas
  and the directional Laplacian coefficients (Sec. 2.1.1, 2.1.2).
* ``dft``       -- naive O(N^2) azimuthal DFT and its Hermitian inverse
  (Sec. 2.2, Eqs. fourier_decomposition and Hermitian_symmetry).
* ``operator``  -- the per-mode 2-D Helmholtz operator (Eqs. helmholz_sph /
  helmholz_cyl, eigenv_sph / eigenv_cyl) as a sparse matrix and as a stencil.
* ``mg``        -- the paper's multigrid: WKB over-relaxation parameter
  (App. A), alternating approximate line smoother (Sec. 3.2, Algorithm 1),
  area-weighted restriction and prolongation (Sec. 3.1), V-cycle.
* ``green``     -- azimuthal Fourier modes of the continuous Green's function
  and of its radial derivative (Eqs. DGF_bc_sph, DGF_bc_cyl, Sec. 4.2).
* ``dgf``       -- discrete Green's function tables by the auxiliary-grid and
  the extended-domain constructions (Sec. 4.2).
* ``james``     -- screening mass (Eqs. charge_sph, charge_cyl), boundary
  potential (Eqs. theta_left..theta_top) and the seven-step solve (Sec. 5.1).
* ``closed_forms`` -- analytic potentials used as pins (Sec. 6.1.1, App. A).

The result of the method is the exact solution of the discrete system; the
multigrid scheme only changes how fast it is reached.  ``james.solve`` therefore
solves each mode with a sparse direct factorisation, which is that definition
written out; ``mg`` is the paper's iteration, pinned against it on small grids
and used as the per-stage reference for the GPU kernels.
"""
