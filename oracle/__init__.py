"""FP64 CPU oracle for the curved-element RKDG Euler right-hand side.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the method of Siebenborn, Schulz & Schmidt, "A curved-element
unstructured discontinuous Galerkin method on GPUs for the Euler equations"
(arXiv 1208.4772), Section 2, written out in its 2D form on triangles.  Only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The product path
(the CUDA library and its binding) never imports, links or executes anything
here, and nothing here imports the product package.

Modules
-------
basis       orthonormal hierarchical Dubiner basis and its gradient (Sec. 2)
nodes       warp & blend collocation nodes (Sec. 2, nodes after Warburton 2006)
quadrature  Gauss rules: collapsed-coordinate volume cubature, edge Gauss
operators   V, V^-1, I_cub, D_r, D_s, I_g (Sec. 2 operator definitions)
geometry    isoparametric element map and its factors (Sec. 2 change of
            variables, Sec. 3 isoparametric curving)
euler       2D Euler flux, perfect-gas pressure, local Lax-Friedrichs flux,
            wall / farfield ghost states (Sec. 5 Euler system, Sec. 2 F*)
dg          semi-discrete right-hand side (eq. semidiscrete), mass matrix
            (eq. mass), Persson-Peraire sensor and artificial viscosity
            (Sec. 2), SSP-RK3 stage update, residual norms
cases       closed-form isentropic vortex used by the convergence pins

Parity status of each function is stated in its docstring; every function
listed above is pinned by ``tests/test_oracle_*.py`` against closed forms,
library routines, invariants or brute force.  The paper prints no values
for the artificial-viscosity right-hand side; it is pinned by closed forms
(the sensor's modal ratio, the gradient exact on linear states, a constant
viscous flux cancelling) in ``tests/test_oracle_av_pins.py`` and
``tests/test_oracle_tet_av.py``.
"""
