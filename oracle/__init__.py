"""FP64 CPU oracle for the finite-element Kohn-Sham slab hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or link this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the CUDA
library: it assembles sparse global matrices cell by cell from exact quadrature and
runs the textbook Chebyshev, Lanczos, conjugate-gradient and dense Rayleigh-Ritz
steps, in float64 with numpy / scipy.

Paper sections followed (Ramakrishnan, Sai Gautam, Motamarri, "Real-space methods for
ab initio modeling of surfaces and interfaces under external potential bias"):

* basis.py      -- GLL nodes and Lagrange basis of Section 2.3 (FE discretization).
* mesh.py       -- periodic-x/y, bounded-z hexahedral mesh of Section 2.3 / Fig. CEF.
* assembly.py   -- K_IJ and the overlap M of Section 2.3; H = -1/2 Laplacian + V_eff
                   (Eq. Veff and Hloc).
* potentials.py -- V_loc - V_sm, smeared charges b (Eq. Governing equations),
                   sawtooth V_app (Section 2.2.1), CPD constraint values
                   (Eq. governing_equations APD).
* poisson.py    -- the Poisson problem (Eq. Poissons equation) with the CEF
                   (Eq. governing_equations CEF) and CPD / L-CPD boundary conditions,
                   the electrostatic energy (Eq. electrostatics Energy, Eq. KS DFT
                   variational problem cef) and the dipole of Section 3.1.
* chefsi.py     -- Chebyshev-filtered subspace iteration for H u = eps M u
                   (Section 2.3 points to prior work for the eigensolver; the scaled
                   three-term filter of Zhou & Saad, J. Comput. Phys. 2006, Lanczos
                   bounds of Zhou & Li 2011, Householder QR + dense eigh).
* kpoint.py     -- the Bloch k-point Hamiltonian (Section 2.1, Bloch's theorem in x, y).
* quadpot.py    -- the potential term integrated by Gauss quadrature (the consistent
                   cell-matrix form of V in Section 2.3), V given at Gauss points.
* analysis.py, projectors.py, scf.py -- analysis outputs, synthetic nonlocal projectors
                   and the self-consistent closure (their module headers cite the
                   passages).

Parity status: every function above is pinned by tests/test_oracle_*.py against
closed forms, patch tests, brute force or textbook identities, except the readings
listed as "parity unpinned" in the module headers (sawtooth return ramps, the L-CPD
off-patch boundary, the Gaussian width convention and the lumped mass choice).
"""
