"""Physical constants and Cu data for the oracle (test infrastructure only).

CODATA 2018 exact/recommended values.  Cu values that the paper prints are cited; the
ones it leaves to earlier work are textbook values, marked as such.
"""
import math

E_CHARGE = 1.602176634e-19        # C
M_E = 9.1093837015e-31            # kg
AMU = 1.66053906660e-27           # kg
EPS0 = 8.8541878128e-12           # F/m
K_B = 1.380649e-23                # J/K
HBAR = 1.054571817e-34            # J s
K_B_EV = K_B / E_CHARGE           # eV/K

M_CU = 63.546 * AMU               # kg (textbook atomic mass of Cu)

# Sec. 2.3.1: evaporation energy printed by the paper; boiling point and the
# atmospheric pressure are not printed (textbook values).
E_VAP_EV = 3.43
T_BOIL = 2835.0
P_ATM = 101325.0

# Sec. 2.1: Lorentz number printed by the paper.
LORENTZ = 2.0e-8                  # W Ohm K^-2

# Sec. 2.3.3 (Eq. 14): ionization potential of Cu (first ionization, textbook; not printed).
XI_CU_EV = 7.726
# Second ionization energy of Cu (Cu+ -> Cu2+, textbook; not printed): the threshold of the
# Cu2+ channels of Table colls (Cu+ + e -> Cu2+ + 2e; Cu + e -> Cu2+ + 3e at XI_CU_EV + XI2_CU_EV).
XI2_CU_EV = 20.292

# Sec. 2.3.2: maximum SP number density n_max = 1e-6 per cubic Angstrom.
N_MAX = 1e-6 * 1e30               # m^-3

# Emission constants in eV / nm units.
Q_IMAGE_EVNM = E_CHARGE / (16.0 * math.pi * EPS0) * 1e9          # e^2/(16 pi eps0) in eV nm
HB2_2M_EVNM2 = HBAR ** 2 / (2.0 * M_E) / E_CHARGE * 1e18         # hbar^2/(2 m_e) in eV nm^2
GAMOW_G = 2.0 / math.sqrt(HB2_2M_EVNM2)                           # 2 sqrt(2 m)/hbar in eV^-1/2 nm^-1
SOMMERFELD_Z = E_CHARGE ** 3 * M_E / (2.0 * math.pi ** 2 * HBAR ** 3)  # A m^-2 eV^-2
