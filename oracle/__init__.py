"""FP64 CPU oracle for one RPMD / adQTB time step on a periodic water box.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or runs
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` do.  It shares no
code, constants table or helper with the CUDA library; the two meet only in
the seeded input generator ``paper_2212_03137_b300.workloads``.

Everything is plain numpy in float64, written step by step in the order of the
paper (Plé et al., "Routine molecular dynamics simulations including nuclear
quantum effects", arXiv 2212.03137):

* ``normal_modes``  - Eqs. (2), (4), (10)-(11): transfer matrix, frequencies,
  mode <-> bead transforms and the force projection;
* ``water``         - the interatomic potential V (a q-SPC/Fw-style flexible
  water with LJ and damped-shifted-force Coulomb; the paper's own force fields
  are AMOEBA-family and are not used here);
* ``neighbor``      - centroid cell assignment and Verlet list (Sec. III.A.3:
  one list on centroids shared by all beads);
* ``rpmd``          - BAOAB in normal modes with the PILE/TRPMD friction
  (Sec. III.A.1, Eqs. (16)-(17)) and the estimators of Eqs. (3), (6);
* ``qtb``           - the adQTB colored noise, spectra and gamma(omega)
  adaptation (Sec. II.B Eqs. (12)-(15); Sec. III.B Eqs. (21)-(26));
* ``philox``        - Philox4x32-10 (Salmon et al., SC'11) and Box-Muller,
  the random numbers both sides draw from the same counters;
* ``respa``         - BAOAB-RESPA multiple time stepping and ring-polymer
  contraction of the slow (nonbonded) forces (Sec. III.A.2, Eqs. (18)-(20));
* ``bar``           - the path-integral Bennett acceptance ratio and its
  single-bead variant (Sec. V, Perspective 2, Eqs. (27)-(28); Appendix A);
* ``gradients``     - dU_P/dx and dU_P/dtheta (analytic) for the force-field
  parameters theta = (eps, sigma, q_O, k_b, k_theta), and the gradient of a
  K-step trajectory average by central differences of whole trajectories.

Parity pins live in ``tests/test_oracle_*.py``.  Parity unpinned: the finite
time-step behaviour of the adQTB spectrum estimator at omega*dt ~ 1 (the
paper gives no formula for its finite-dt corrections); it is compared
oracle-vs-GPU under the same definition only.
"""
