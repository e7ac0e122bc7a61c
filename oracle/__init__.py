"""Plain FP64 CPU oracle for the relativistic lattice Boltzmann step of
Gabbana, Mendoza, Succi & Tripiccione, "Towards a unified lattice kinetic
scheme for relativistic hydrodynamics" (arXiv:1703.04605).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA path.

Modules (each function cites the passage it follows):

* ``groups``     -- Table I (App. C): the 84 full-symmetric velocity groups.
* ``special``    -- Bessel K_nu in extended precision (``decimal``) and in
                    FP64 (scipy), rest-frame moments of the weight, Eq. 36-41.
* ``quadrature`` -- weights w_k of a 6-group (second-order) or 11-group
                    (third-order) stencil from Eq. 47/52 (square
                    moment-matching form, extended precision), the 2D fold.
* ``polynomials``-- the 2nd-order orthonormal polynomials (App. A) and the
                    projections b^(k) (App. B, three misprints corrected).
* ``equilibrium``-- the discrete equilibrium Eq. 16 by two independent routes.
* ``third_order``-- the third-order equilibrium: orthonormal polynomials of
                    degree <= 3 (Gram-Schmidt in extended precision) and
                    projections from the closed-form moments up to rank 3.
* ``lattice``    -- one lattice step: moments (Eq. 4-5/18), Landau frame
                    (Eq. 19-20), EOS inversion (Eq. 28-29), AW collision and
                    exact streaming (Eq. 49).

Equation numbers count the numbered equations of the paper in order of
appearance (Eq. 1 = relativistic Boltzmann equation, Eq. 49 = the lattice
update with v0 n_i dt displacements).
"""
