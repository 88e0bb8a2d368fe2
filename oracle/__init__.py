"""Independent FP64 CPU oracle for the PUFE hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this
package; only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` may use it.  It shares no code
with the CUDA library: every formula here is written from the paper
(Pask & Sukumar, "Partition of unity finite element method for quantum
mechanical materials calculations") in plain NumPy/SciPy, slow and direct.

Modules
-------
fe         1D cubic Lagrange / linear shape functions, tensor products,
           Gauss-Legendre rules (Sec. 2 eq. pum; Sec. 5.1 trilinear PU;
           Sec. 6.2 higher-order FE).
enrich     Slater-type radial x real spherical harmonic x C^3 cutoff
           enrichments with the periodic image sum (Sec. 5.1, eqs. Psitilde
           and Psi).  Gradients by complex-step differentiation.
mesh       periodic hexahedral mesh, FE/PU numbering, enriched-node sets,
           per-element basis lists (Sec. 4 eqs. pufebasis, psih).
quadrature element quadrature rules: fixed classes, p-adaptive and the
           recursive 5^3 vs 8^3 scheme (Sec. 5.2).
assemble   H and S by element quadrature (Sec. 4 eq. disceig3d), density at
           quadrature points (Sec. 3 eq. rhoe) and the adjoint of V -> H.
potential  periodic local potential of Gaussian ionic charges (Sec. 3,
           localized ionic charges generating V_I).
eig        generalized eigensolve and occupations.
pu1d       the 1D L2-projection example of the supplementary material.

Parity status per function is stated in each module header.
"""
