"""Plain FP64 CPU oracle of the vacuum-arc PIC-MCC step (Koitermaa et al., arXiv:2402.08404).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or link anything
in this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  The oracle shares no code, tables or constants with the CUDA library;
each function cites the passage of the paper it restates.  Equations are cited by their
LaTeX label (the paper numbers them only when typeset), sections by number and title:
Sec. 2.1 "FEM solution of electric field and heating", Sec. 2.2 "PIC-MCC particle
simulation", Sec. 2.3.1 "Simulation model", Sec. 2.3.2 "Dynamic weighting",
Sec. 2.3.3 "Ion bombardment effects", Sec. 2.3.4 "Direct field ionization".

Modules
-------
constants  physical constants (CODATA 2018) and Cu data used by the step
philox     Philox4x32-10 counter-based generator (Salmon et al., SC'11)
grid       staircased tip geometry, exposed faces, Dirichlet nodes (Sec. 2.1, Fig. domains)
field      7-point Poisson operator and direct solve, node field E = -grad(phi) (eq:poi, eq:bcf1-3)
particles  CIC gather, leapfrog push, DDA boundary test, stable cell sort, fixed-point deposit (Sec. 2.2)
collide    impact ionization MCC with SP splitting (eq:colp, eq:du, Sec. 2.3.2) and ADK field ionization (eq:dfi)
elastic    elastic e-Cu and Cu-Cu collisions (eq:newv, eq:du) and Cu+-Cu charge exchange (Table colls)
merge      superparticle merging in over-full cells (Sec. 2.3.2)
coulomb    binary Coulomb collisions e-e, e-Cu+, Cu+-Cu+ (Table colls, the cited small-angle method)
emission   general thermal-field emission current and Nottingham heat (Sec. 2.3.1)
surface    Clausius-Clapeyron evaporation, injection weights, sputtering, bombardment heat (Sec. 2.3.1-2.3.3)
heat       tip heat equation with Wiedemann-Franz conductivity and current continuity (eq:heat, eq:cont)
circuit    RC circuit of the gap and the Shockley-Ramo gap current (Sec. 2.3.1, circuit passage)
mlp        FP64 forward/backward of the emission surrogate MLP (no counterpart in the paper)
step       one coupled PIC-MCC step in the paper's order (Sec. 2.3.1, Fig. newpic)
"""
