"""Surface processes of the step (test infrastructure only).

  evaporation   Clausius-Clapeyron flux (Sec. 2.3.1):
                phi_vap = p_atm / sqrt(2 pi m k_B T) * exp[E_vap/k_B (1/T_b - 1/T)],
                cooling P_vap = E_vap phi_vap (the k_B T term dropped, as the paper does);
  weights       injection weight (Sec. 2.3.2): w = min(ceil(max(1, sqrt(n_cell/n_max N_inj/w_min))) w_min, w_max)
                (the text says "floor", the formula ceil: the formula is taken);
  sputtering    Sec. 2.3.3: yields and energies from fitted data that is not available:
                a Yamamura-type stand-in Y(E) = Q s_n(E/E_TF) (1 - sqrt(E_th/E))^s and the
                Thompson energy law f(E) ~ E/(E+U_s)^3 truncated at E_cap; directions uniform
                over the hemisphere about the face normal (cos(theta) ~ U(0,1));
  bombardment   P_bom = (E_b - E_s)/(A dt_heat) (Sec. 2.3.3).

Velocities of evaporated atoms: flux-weighted half-Maxwellian (Sec. 2.3.1: "sampled from
the Maxwell-Boltzmann distribution based on the surface temperature"): normal speed
sqrt(-2 k T/m ln U), tangential components Box-Muller with sigma = sqrt(kT/m).
"""
import math

import numpy as np

from . import constants as C

# stand-in sputtering parameters (Cu -> Cu), an input table
SPUTTER = {"Q": 10.7, "E_TF": 11.9e3, "E_th": 25.0, "s": 2.5, "U_s": 3.43, "E_cap": 100.0}

SPUT_FRAC_BITS = 24      # sputter accumulator: real atoms in units of 2^-24
ENERGY_FRAC_BITS = 20    # bombardment energy accumulators: eV in units of 2^-20


def evaporation_flux(T):
    """phi_vap [m^-2 s^-1] of Sec. 2.3.1."""
    T = np.asarray(T, dtype=np.float64)
    pre = C.P_ATM / np.sqrt(2.0 * math.pi * C.M_CU * C.K_B * T)
    return pre * np.exp(C.E_VAP_EV / C.K_B_EV * (1.0 / C.T_BOIL - 1.0 / T))


def injection_weight_units(n_cell, N_inj, w_min, w_max_units):
    """Weight in units of w_min from the geometric-mean rule of Sec. 2.3.2."""
    r = (n_cell / C.N_MAX) * (N_inj / w_min)
    return int(min(math.ceil(max(1.0, math.sqrt(r))), w_max_units))


def nuclear_stopping(eps):
    se = math.sqrt(eps)
    return 3.441 * se * math.log(eps + 2.718) / (1.0 + 6.355 * se + eps * (6.882 * se - 1.708))


def sputter_yield(E, prm=SPUTTER):
    if E <= prm["E_th"]:
        return 0.0
    return prm["Q"] * nuclear_stopping(E / prm["E_TF"]) * (1.0 - math.sqrt(prm["E_th"] / E)) ** prm["s"]


def thompson_energy(U, prm=SPUTTER):
    """Inverse CDF of the Thompson law truncated at E_cap: F(E) = (E/(E+U_s))^2."""
    Us, Ec = prm["U_s"], prm["E_cap"]
    Fc = (Ec / (Ec + Us)) ** 2
    s = math.sqrt(U * Fc)
    return Us * s / (1.0 - s)
