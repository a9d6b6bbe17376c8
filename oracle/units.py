"""Physical constants in the oracle's unit system (kcal/mol, Angstrom, amu, ps, e, K).

None of these are printed in the paper; they are CODATA-derived readings.
"""
KB = 8.314462618 / 4184.0                                 # Boltzmann, kcal/mol/K
HBAR = 1.054571817e-34 * 6.02214076e23 / 4184.0 * 1e12     # hbar, kcal/mol * ps
COULOMB = 332.0637133                                      # k_e, kcal*A/(mol*e^2)
ACC = 418.4                                                # (kcal/mol)/amu -> A^2/ps^2
CM1_TO_RAD_PS = 2.0 * 3.141592653589793 * 2.99792458e10 * 1e-12  # cm^-1 -> rad/ps
